"""The coarse end of the V-cycle as one persistent kernel (vtail.cu, opt-in
through AMG_VTAIL_LEVEL) against the same V-cycle with one launch per
product: the same bits, in FP64 and FP32 and for both block sizes, for the
V-cycle alone and for whole solves."""
import os

import numpy as np
import pytest

import workloads as W
from _problems import gpu_problem

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def A():
    import torch
    assert torch.cuda.is_available(), "GPU tests need a CUDA device"
    import paper_1902_01715_gb300 as lib_
    lib_.build()
    lib_.lib()
    return lib_


def _solver(A, d, block, prec, fused):
    if fused:
        os.environ["AMG_VTAIL_LEVEL"] = "1"
    else:
        os.environ.pop("AMG_VTAIL_LEVEL", None)
    try:
        if block == 1:
            rp, col, val = A.bsr_to_scalar(d["rowptr"], d["col"], d["vals"])
        else:
            rp, col, val = d["rowptr"], d["col"], d["vals"]
        return A.Solver(rp, col, val, d["V0"], block=block, vcycle_prec=prec)
    finally:
        os.environ.pop("AMG_VTAIL_LEVEL", None)


@pytest.mark.parametrize("block", [3, 1])
@pytest.mark.parametrize("prec", ["fp64", "fp32"])
def test_fused_vcycle_equals_separate_launches(A, block, prec):
    import torch
    d = gpu_problem(A, W.beam(32, 8, 8))
    Sf = _solver(A, d, block, prec, True)
    Ss = _solver(A, d, block, prec, False)
    assert Sf.stats()["vcycle_fused_level"] == 1 and Ss.stats()["vcycle_fused_level"] == -1
    assert Sf.nlev >= 3
    y = torch.tensor(np.random.default_rng(61).normal(size=d["f"].numel()), device="cuda")
    for _ in range(2):
        assert torch.equal(Sf.vcycle(y), Ss.vcycle(y))
    xf, itf, rf, rcf = Sf.solve(d["f"], 1e-10)
    xs, its, rs, rcs = Ss.solve(d["f"], 1e-10)
    assert rcf == 0 and rcs == 0 and itf == its
    assert torch.equal(xf, xs)
