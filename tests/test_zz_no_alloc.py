"""amg_vcycle_noalloc (the V-cycle entry point that allocates nothing, for
callers whose process cannot allocate device memory while the preconditioner
runs) against amg_vcycle, through the C ABI.  This file is collected last so
that a run stopping at the first failure has run every other test first."""
import ctypes as C

import numpy as np
import pytest

import workloads as W

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def A():
    import torch
    assert torch.cuda.is_available(), "GPU tests need a CUDA device"
    import paper_1902_01715_gb300 as lib_
    lib_.build()
    lib_.lib()
    return lib_


def _solver(A, p, **over):
    d = A.fe_assemble(p.nx, p.ny, p.nz, p.hx, p.hy, p.hz, p.nu, p.E, p.clamp_axis)
    V0 = A.fe_rbm(p.nx, p.ny, p.nz, p.hx, p.hy, p.hz, p.clamp_axis, d["nfree"])
    return A.Solver(d["rowptr"], d["col"], d["vals"], V0, **over), d["nfree"]


@pytest.mark.parametrize("prec", ["fp64", "fp32"])
def test_noalloc_vcycle_matches_vcycle_twice(A, prec):
    import torch
    S, nf = _solver(A, W.beam(32, 8, 8), vcycle_prec=prec)
    L = A.lib()
    y = torch.tensor(np.random.default_rng(51).normal(size=3 * nf), device="cuda")
    z_ref = torch.empty_like(y)
    A.check(L.amg_vcycle(S._h, C.c_void_p(y.data_ptr()), C.c_void_p(z_ref.data_ptr())), "amg_vcycle")
    ref = z_ref.cpu().numpy()
    tol = 1e-12 if prec == "fp64" else 1e-6
    for _ in range(2):  # two calls in a row share (and reset) the static scratch
        z = torch.full_like(y, float("nan"))
        A.check(L.amg_vcycle_noalloc(S._h, C.c_void_p(y.data_ptr()), C.c_void_p(z.data_ptr())),
                "amg_vcycle_noalloc")
        got = z.cpu().numpy()
        assert np.all(np.isfinite(got))
        assert np.abs(got - ref).max() <= tol * np.abs(ref).max()


def test_noalloc_large_coarse_level(A):
    """A last level of 3,630 dofs (a 10^3 cube kept whole): the coarse solve is
    one product with the level's explicit inverse and needs no scratch."""
    import torch
    S, nf = _solver(A, W.cube16(10), n_coarse=4000)
    assert S.nlev == 1
    L = A.lib()
    y = torch.tensor(np.random.default_rng(52).normal(size=3 * nf), device="cuda")
    z_ref = torch.empty_like(y)
    A.check(L.amg_vcycle(S._h, C.c_void_p(y.data_ptr()), C.c_void_p(z_ref.data_ptr())), "amg_vcycle")
    z = torch.full_like(y, float("nan"))
    A.check(L.amg_vcycle_noalloc(S._h, C.c_void_p(y.data_ptr()), C.c_void_p(z.data_ptr())),
            "amg_vcycle_noalloc")
    assert torch.equal(z, z_ref)
    # one level: the V-cycle is the exact solve K z = y
    rp, col, val = S.level_matrix(0, "A")
    K = np.zeros((3 * nf, 3 * nf))
    for I in range(nf):
        for k in range(rp[I], rp[I + 1]):
            J = col[k]
            K[3 * I:3 * I + 3, 3 * J:3 * J + 3] = val[k].reshape(3, 3)
    zn, yn = z.cpu().numpy(), y.cpu().numpy()
    assert np.linalg.norm(K @ zn - yn) <= 1e-9 * np.linalg.norm(yn)
