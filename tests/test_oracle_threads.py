"""The oracle's OpenMP loops split only independent rows, chunks and entries:
the hierarchy and the PCG solution are the same bits whatever the number of
threads (checked by hashing every level in child processes run with one and
with four threads)."""
import os
import subprocess
import sys

import pytest

CHILD = r"""
import hashlib, sys
sys.path.insert(0, "tests"); sys.path.insert(0, ".")
import numpy as np
import oracle as orc
import workloads as W
from _problems import oracle_problem
p = W.beam(24, 6, 6) if sys.argv[1] == "beam" else W.slab(24, 24, 4)
K, V0, f, nm = oracle_problem(orc, p)
H = orc.Hierarchy(K, V0, orc.default_params(3, n_coarse=300))
h = hashlib.sha256()
for k in range(H.nlev):
    A = H.matrix(k, "A")
    h.update(A.rowptr.tobytes()); h.update(A.col.tobytes()); h.update(A.val.tobytes())
    if k < H.nlev - 1:
        for w in ("G", "P"):
            M = H.matrix(k, w)
            h.update(M.rowptr.tobytes()); h.update(M.col.tobytes()); h.update(M.val.tobytes())
        h.update(H.cf(k).tobytes()); h.update(H.V(k).tobytes())
        h.update(np.float64(H.info(k)["omega"]).tobytes())
x, it, rr, rc = H.pcg(f, 1e-10)
h.update(x.tobytes())
print("HASH", it, h.hexdigest())
"""


@pytest.mark.parametrize("name", ["beam", "slab"])
def test_oracle_bits_independent_of_threads(name):
    root = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
    out = []
    for nt in ("1", "4"):
        env = dict(os.environ, OMP_NUM_THREADS=nt)
        r = subprocess.run([sys.executable, "-c", CHILD, name], env=env, cwd=root, capture_output=True,
                           text=True, timeout=600)
        assert r.returncode == 0, r.stdout + r.stderr
        out.append([ln for ln in r.stdout.splitlines() if ln.startswith("HASH")][0])
    assert out[0] == out[1], out
