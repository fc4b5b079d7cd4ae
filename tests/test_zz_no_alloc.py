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


def _default_pool():
    """(used, used_high, reset_high) of this device's default stream-ordered
    memory pool, the pool every device allocation of the library comes from,
    read through the CUDA driver API."""
    import torch
    cu = C.CDLL("libcuda.so.1")
    cu.cuDeviceGet.argtypes = [C.POINTER(C.c_int), C.c_int]
    cu.cuDeviceGetDefaultMemPool.argtypes = [C.POINTER(C.c_void_p), C.c_int]
    cu.cuMemPoolGetAttribute.argtypes = [C.c_void_p, C.c_int, C.c_void_p]
    cu.cuMemPoolSetAttribute.argtypes = [C.c_void_p, C.c_int, C.c_void_p]
    dev, pool = C.c_int(), C.c_void_p()
    assert cu.cuDeviceGet(C.byref(dev), torch.cuda.current_device()) == 0
    assert cu.cuDeviceGetDefaultMemPool(C.byref(pool), dev.value) == 0
    USED_CURRENT, USED_HIGH = 7, 8  # CU_MEMPOOL_ATTR_USED_MEM_CURRENT / _HIGH

    def get(attr):
        v = C.c_uint64()
        assert cu.cuMemPoolGetAttribute(pool, attr, C.byref(v)) == 0
        return v.value

    def reset_high():
        z = C.c_uint64(0)
        assert cu.cuMemPoolSetAttribute(pool, USED_HIGH, C.byref(z)) == 0

    return (lambda: get(USED_CURRENT)), (lambda: get(USED_HIGH)), reset_high


@pytest.mark.parametrize("prec", ["fp64", "fp32"])
def test_noalloc_vcycle_matches_vcycle_twice(A, prec):
    import torch
    S, nf = _solver(A, W.beam(32, 8, 8), vcycle_prec=prec)
    L = A.lib()
    y = torch.tensor(np.random.default_rng(51).normal(size=3 * nf), device="cuda")
    z_ref = torch.empty_like(y)
    A.check(L.amg_vcycle(S._h, C.c_void_p(y.data_ptr()), C.c_void_p(z_ref.data_ptr())), "amg_vcycle")
    zs = [torch.full_like(y, float("nan")) for _ in range(2)]
    used, used_high, reset_high = _default_pool()
    torch.cuda.synchronize()
    before = used()
    reset_high()
    for z in zs:  # two calls in a row share (and reset) the static scratch
        A.check(L.amg_vcycle_noalloc(S._h, C.c_void_p(y.data_ptr()), C.c_void_p(z.data_ptr())),
                "amg_vcycle_noalloc")
    torch.cuda.synchronize()
    # nothing was taken from the pool, not even temporarily
    assert used() == before and used_high() <= before
    # the same kernels in the same order as amg_vcycle: the same bits
    for z in zs:
        assert torch.equal(z, z_ref)


CHILD_TIMEOUT = r"""
import ctypes as C
import sys
sys.path.insert(0, "tests"); sys.path.insert(0, ".")
import torch
import paper_1902_01715_gb300 as A
import workloads as W
from _problems import gpu_problem
A.build(); L = A.lib()
d = gpu_problem(A, W.beam(32, 8, 8))
S = A.Solver(d["rowptr"], d["col"], d["vals"], d["V0"], vcycle_prec="fp32")
y = torch.randn(d["f"].numel(), dtype=torch.float64, device="cuda")
z = torch.empty_like(y)
rc = L.amg_vcycle_noalloc(S._h, C.c_void_p(y.data_ptr()), C.c_void_p(z.data_ptr()))
msg = L.amg_last_error().decode()
assert rc == A.AMG_ERR_CUDA and "bulk-copy" in msg, (rc, msg)
print("TIMEOUT-REPORTED")
z2, z3 = torch.empty_like(y), torch.empty_like(y)
assert L.amg_vcycle_noalloc(S._h, C.c_void_p(y.data_ptr()), C.c_void_p(z2.data_ptr())) == 0
assert L.amg_vcycle(S._h, C.c_void_p(y.data_ptr()), C.c_void_p(z3.data_ptr())) == 0
assert torch.equal(z2, z3)
print("RECOVERED")
"""


def test_noalloc_reports_bulk_copy_timeout():
    """With the bulk-copy sparse product pinned and the one-shot stall knob
    set, a pipeline wait inside amg_vcycle_noalloc runs out (bounded, no
    fault): the call reports AMG_ERR_CUDA with the reason instead of returning
    a partly written z, and the next call succeeds."""
    import os
    import subprocess
    import sys
    import torch
    assert torch.cuda.is_available(), "GPU tests need a CUDA device"
    env = dict(os.environ, AMG_MAP="8", AMG_BULK_STALL_ONCE="1")
    r = subprocess.run([sys.executable, "-c", CHILD_TIMEOUT], env=env, capture_output=True, text=True,
                       timeout=600, cwd=os.path.dirname(os.path.dirname(os.path.abspath(__file__))))
    assert r.returncode == 0, r.stdout + r.stderr
    assert "TIMEOUT-REPORTED" in r.stdout and "RECOVERED" in r.stdout, r.stdout + r.stderr


def test_noalloc_rejects_other_device(A):
    """The scratch address is looked up per device: a call whose current
    device is not the handle's is refused.  (Runs only with two GPUs.)"""
    import torch
    if torch.cuda.device_count() < 2:
        pytest.skip("needs two GPUs")
    S, nf = _solver(A, W.beam(16, 4, 4))
    y = torch.zeros(3 * nf, dtype=torch.float64, device="cuda")
    z = torch.empty_like(y)
    with torch.cuda.device(1):
        rc = A.lib().amg_vcycle_noalloc(S._h, C.c_void_p(y.data_ptr()), C.c_void_p(z.data_ptr()))
    assert rc == A.AMG_ERR_ARG


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
