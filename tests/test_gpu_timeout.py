"""The bounded wait of the bulk-copy sparse product, exercised without any
fault: a one-shot test knob leaves one pipeline stage unfilled, so a warp's
wait on its mbarrier runs out (about two seconds); the kernel records the
timeout and returns, the solve reports AMG_ERR_CUDA with the reason, and the
next solve in the same process succeeds."""
import os
import subprocess
import sys

import pytest

pytestmark = pytest.mark.gpu

CHILD = r"""
import sys
sys.path.insert(0, "tests"); sys.path.insert(0, ".")
import torch
import paper_1902_01715_gb300 as A
import workloads as W
from _problems import gpu_problem
A.build(); A.lib()
d = gpu_problem(A, W.beam(32, 8, 8))
S = A.Solver(d["rowptr"], d["col"], d["vals"], d["V0"], vcycle_prec="fp32")
try:
    S.solve(d["f"], 1e-8)
    print("NO-ERROR")
except A.AmgError as e:
    assert e.code == A.AMG_ERR_CUDA and "bulk-copy" in str(e), str(e)
    print("TIMEOUT-REPORTED")
x, its, rel, rc = S.solve(d["f"], 1e-8)
assert rc == 0 and rel[0] <= 1e-8
print("RECOVERED", its[0])
"""


def test_bulk_copy_wait_timeout_is_reported():
    import torch
    assert torch.cuda.is_available(), "GPU tests need a CUDA device"
    env = dict(os.environ, AMG_MAP="8", AMG_BULK_STALL_ONCE="1")
    r = subprocess.run([sys.executable, "-c", CHILD], env=env, capture_output=True, text=True, timeout=600,
                       cwd=os.path.dirname(os.path.dirname(os.path.abspath(__file__))))
    assert r.returncode == 0, r.stdout + r.stderr
    assert "TIMEOUT-REPORTED" in r.stdout and "RECOVERED" in r.stdout, r.stdout + r.stderr
