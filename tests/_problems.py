"""Builds one seeded workload on both sides: the oracle assembles its own K, f
and rigid-body modes on the CPU, the GPU library its own on the device.  The
two share only the workload description (workloads.Problem)."""
import numpy as np

import workloads as W


def oracle_problem(orc, p: W.Problem, col=0):
    K, nm = orc.assemble(p.nx, p.ny, p.nz, p.hx, p.hy, p.hz, p.nu, p.E, p.clamp_axis)
    V0 = orc.rbm(p.nx, p.ny, p.nz, p.hx, p.hy, p.hz, nm)
    if p.load == "body":
        f = orc.load_body(p.nx, p.ny, p.nz, p.hx, p.hy, p.hz, p.body, nm)
    elif p.load == "end_shear":
        f = orc.load_end_shear(p.nx, p.ny, p.nz, p.hx, p.hy, p.hz, p.shear_total, nm)
    elif p.load == "top_pressure":
        f = orc.load_top_pressure(p.nx, p.ny, p.nz, p.hx, p.hy, p.hz, p.pressure, nm)
    else:
        f = nodal_to_free(p, nm, col)
    return K, V0, f, nm


def nodal_to_free(p: W.Problem, nm, col=0):
    """Scatter the top-face nodal forces of load case `col` onto free dofs."""
    nfree = int((nm >= 0).sum())
    f = np.zeros(3 * nfree)
    NX, NY = p.nx + 1, p.ny + 1
    for iy in range(NY):
        for ix in range(NX):
            I = nm[ix + NX * (iy + NY * p.nz)]
            if I >= 0:
                f[3 * I:3 * I + 3] += p.nodal[col, ix + NX * iy]
    return f


def gpu_problem(A, p: W.Problem, col=0):
    """(rowptr, col, vals, Ke0, V0 (n, 6), f) as CUDA tensors from the library."""
    d = A.fe_assemble(p.nx, p.ny, p.nz, p.hx, p.hy, p.hz, p.nu, p.E, p.clamp_axis)
    n = d["nfree"]
    V0 = A.fe_rbm(p.nx, p.ny, p.nz, p.hx, p.hy, p.hz, p.clamp_axis, n)
    if p.load == "body":
        f = A.fe_load(p.nx, p.ny, p.nz, p.hx, p.hy, p.hz, p.clamp_axis, "body", g=p.body, nfree=n)
    elif p.load == "end_shear":
        f = A.fe_load(p.nx, p.ny, p.nz, p.hx, p.hy, p.hz, p.clamp_axis, "end_shear",
                      g=[p.shear_total], nfree=n)
    elif p.load == "top_pressure":
        f = A.fe_load(p.nx, p.ny, p.nz, p.hx, p.hy, p.hz, p.clamp_axis, "top_pressure",
                      p=p.pressure, nfree=n)
    else:
        f = A.fe_load(p.nx, p.ny, p.nz, p.hx, p.hy, p.hz, p.clamp_axis, "top_nodal",
                      p=np.ascontiguousarray(p.nodal[col]).reshape(-1), nfree=n)
    d.update(V0=V0, f=f)
    return d


SMALL = {
    "cube": lambda: W.cube16(16),
    "beam": lambda: W.beam(32, 8, 8),
    "slab": lambda: W.slab(32, 32, 4),
}


def rel(a, b):
    a, b = np.asarray(a), np.asarray(b)
    den = np.abs(b).max() if b.size else 0.0
    return float(np.abs(a - b).max() / den) if den > 0 else float(np.abs(a - b).max() if a.size else 0.0)


def compare_hierarchies(S, H):
    """GPU hierarchy S (library handle) against the oracle's H, level by level:
    the C/F split and the patterns of A_k, G_k, P_k, R_k bit for bit, their
    values within 1e-13 relative, omega_k, lambda_1 and the refinement passes
    exactly, the test spaces within 1e-12 relative."""
    assert S.nlev == H.nlev, (S.nlev, H.nlev)
    for k in range(H.nlev):
        go, oo = S.level_info(k), H.info(k)
        assert go["nr"] == oo["nr"] and go["nnzb_A"] == oo["nnzb_A"], k
        Ao = H.matrix(k, "A")
        rp, col, val = S.level_matrix(k, "A")
        assert np.array_equal(rp, Ao.rowptr) and np.array_equal(col, Ao.col[:Ao.nnzb]), k
        assert rel(val, Ao.val[:Ao.nnzb]) <= 1e-13, k
        if k == H.nlev - 1:
            continue
        assert go["npasses"] == oo["npasses"], k
        assert go["omega"] == oo["omega"] and go["lmax"] == oo["lmax"], k
        assert np.array_equal(S.level_cf(k), H.cf(k)), k
        for which in ("G", "P", "R"):
            Mo = H.matrix(k, which)
            rp, col, val = S.level_matrix(k, which)
            assert np.array_equal(rp, Mo.rowptr) and np.array_equal(col, Mo.col[:Mo.nnzb]), (k, which)
            assert rel(val, Mo.val[:Mo.nnzb]) <= 1e-13, (k, which)
        assert rel(S.level_testspace(k), H.V(k)) <= 1e-12, k
