"""Programmatic dependent launch (a kernel may be scheduled while the one
before it runs, and waits for it in-kernel) against plain stream-ordered
launches (AMG_NO_PDL): the same hierarchy and the same bits, for the set-up,
the V-cycle alone and whole solves, in FP64 and FP32 and for both block
sizes.  The slab's level-0 Galerkin product has 5,445 rows and takes the
by-rows numeric product; the beam's smaller products take the nine-lane one."""
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


def _with_pdl(on, fn):
    if on:
        os.environ.pop("AMG_NO_PDL", None)
    else:
        os.environ["AMG_NO_PDL"] = "1"
    try:
        return fn()
    finally:
        os.environ.pop("AMG_NO_PDL", None)


@pytest.mark.parametrize("name,block,prec", [("beam", 3, "fp64"), ("beam", 3, "fp32"), ("slab", 3, "fp64"),
                                             ("beam", 1, "fp64")])
def test_programmatic_launch_same_bits(A, name, block, prec):
    import torch
    prob = W.beam(32, 8, 8) if name == "beam" else W.slab(32, 32, 4)
    d = gpu_problem(A, prob)
    if block == 1:
        rp, col, val = A.bsr_to_scalar(d["rowptr"], d["col"], d["vals"])
    else:
        rp, col, val = d["rowptr"], d["col"], d["vals"]
    make = lambda: A.Solver(rp, col, val, d["V0"], block=block, vcycle_prec=prec)
    Sp = _with_pdl(True, make)
    Sq = _with_pdl(False, make)
    assert Sp.nlev == Sq.nlev
    for k in range(Sp.nlev):
        for which in ("A", "G", "P") if k < Sp.nlev - 1 else ("A",):
            a, b = Sp.level_matrix(k, which), Sq.level_matrix(k, which)
            for u, v in zip(a, b):
                assert np.array_equal(u, v), (k, which)
    y = torch.tensor(np.random.default_rng(67).normal(size=d["f"].numel()), device="cuda")
    zp = _with_pdl(True, lambda: Sp.vcycle(y))
    zq = _with_pdl(False, lambda: Sq.vcycle(y))
    assert torch.equal(zp, zq)
    xp, itp, rp_, rcp = _with_pdl(True, lambda: Sp.solve(d["f"], 1e-10))
    xq, itq, rq_, rcq = _with_pdl(False, lambda: Sq.solve(d["f"], 1e-10))
    assert rcp == 0 and rcq == 0 and itp == itq
    assert torch.equal(xp, xq)
