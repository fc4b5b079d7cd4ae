"""Batched right-hand sides (block SpMM V-cycle, per-column convergence masks)
and the adjoint gradient, through the C ABI, against the oracle and finite
differences."""
import numpy as np
import pytest

import workloads as W
from _problems import gpu_problem, nodal_to_free, oracle_problem

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def A():
    import torch
    assert torch.cuda.is_available(), "GPU tests need a CUDA device"
    import paper_1902_01715_gb300 as lib_
    lib_.build()
    lib_.lib()
    return lib_


def _batched_problem(A, orc, n=8, k=5):
    import torch
    p = W.cube_batched(n, k)
    K, V0, f0, nm = oracle_problem(orc, p, 0)
    F = np.column_stack([nodal_to_free(p, nm, c) for c in range(k)])
    d = gpu_problem(A, p, 0)
    Fg = torch.tensor(F, device="cuda")
    return p, K, V0, F, d, Fg


def test_batched_fp64_matches_oracle_per_column(A, orc):
    p, K, V0, F, d, Fg = _batched_problem(A, orc)
    H = orc.Hierarchy(K, V0)
    S = A.Solver(d["rowptr"], d["col"], d["vals"], d["V0"])
    X, its, rel, rc = S.solve(Fg, 1e-12)
    assert rc == 0 and len(its) == F.shape[1]
    Xn = X.cpu().numpy()
    for c in range(F.shape[1]):
        xo, ito, _, _ = H.pcg(F[:, c], 1e-12)
        assert np.linalg.norm(Xn[:, c] - xo) <= 1e-10 * np.linalg.norm(xo), c
        assert rel[c] <= 1e-12
        # the same column alone through the single right-hand-side path
        x1, it1, _, _ = S.solve(Fg[:, c].contiguous(), 1e-12)
        assert abs(it1[0] - its[c]) <= 1
        assert np.linalg.norm(x1.cpu().numpy() - Xn[:, c]) <= 1e-10 * np.linalg.norm(xo)


@pytest.mark.parametrize("prec", ["fp32", "bf16gp"])
def test_batched_mixed_reaches_tolerance(A, orc, prec):
    p, K, V0, F, d, Fg = _batched_problem(A, orc, n=10, k=8)
    S = A.Solver(d["rowptr"], d["col"], d["vals"], d["V0"], vcycle_prec=prec)
    X, its, rel, rc = S.solve(Fg, 1e-8)
    assert rc == 0
    Xn = X.cpu().numpy()
    # rel[c] is the library's FP64 true residual of column c (restarted from
    # it when above rtol); the oracle's K gives the same value to rounding
    for c in range(F.shape[1]):
        true_rel = np.linalg.norm(F[:, c] - K.matvec(Xn[:, c])) / np.linalg.norm(F[:, c])
        assert rel[c] <= 1e-8, (c, rel[c])
        assert abs(true_rel - rel[c]) <= 1e-10, (c, true_rel, rel[c])


def test_batched_masks_freeze_finished_columns(A, orc):
    import torch
    p, K, V0, F, d, Fg = _batched_problem(A, orc, n=8, k=4)
    G = Fg.clone()
    G[:, 1] = 0.0            # converged at the start
    G[:, 2] *= 1e6           # scale must not matter for the relative test
    S = A.Solver(d["rowptr"], d["col"], d["vals"], d["V0"])
    X, its, rel, rc = S.solve(G, 1e-8)
    assert rc == 0
    assert its[1] == 0 and float(X[:, 1].abs().max()) == 0.0
    X0, its0, _, _ = S.solve(Fg[:, 2].contiguous(), 1e-8)
    assert abs(its[2] - its0[0]) <= 1
    assert torch.allclose(X[:, 2] / 1e6, X0, rtol=1e-7, atol=0)
    S2 = A.Solver(d["rowptr"], d["col"], d["vals"], d["V0"], maxit=2)
    X2, its2, rel2, rc2 = S2.solve(Fg, 1e-8)
    assert rc2 == A.AMG_ERR_NOT_CONVERGED and max(its2) == 2


def _simp(A, n, rho):
    import torch
    p = W.cube_simp(n)
    p.rho = rho
    p.E = rho ** 3
    d = gpu_problem(A, p)
    return p, d


def test_adjoint_gradient_against_oracle_and_fd(A, orc):
    import torch
    n = 6
    p0 = W.cube_simp(n)
    rho = p0.rho.copy()
    p, d = _simp(A, n, rho)
    S = A.Solver(d["rowptr"], d["col"], d["vals"], d["V0"], n_coarse=300)
    conn = A.fe_conn(p.nx, p.ny, p.nz, p.clamp_axis)
    rho_t = torch.tensor(rho, device="cuda", requires_grad=True)
    E = rho_t ** 3
    u = A.LinearSolve.apply(S, d["f"], E, d["Ke0"], conn, 1e-12)
    L = torch.dot(d["f"], u)                     # compliance f^T u
    L.backward()
    g = rho_t.grad.cpu().numpy()
    # adjoint solve reuses the hierarchy and equals the forward solve (K = K^T)
    lam, _, _, _ = S.adjoint(d["f"], 1e-12)
    assert torch.equal(lam, u.detach())
    # oracle: dL/drho_e = -3 rho_e^2 u_e^T Ke0 u_e with the oracle's solution
    K, V0, f, nm = oracle_problem(orc, p)
    H = orc.Hierarchy(K, V0, orc.default_params(3, n_coarse=300))
    uo, _, _, _ = H.pcg(f, 1e-12)
    Ke0 = orc.ke0(p.nu, p.hx, p.hy, p.hz)
    NX, NY = p.nx + 1, p.ny + 1
    go = np.zeros(p.ne)
    for e in range(p.ne):
        ex, ey, ez = e % p.nx, (e // p.nx) % p.ny, e // (p.nx * p.ny)
        ue = np.zeros(24)
        for a in range(8):
            I = nm[(ex + (a & 1)) + NX * ((ey + ((a >> 1) & 1)) + NY * (ez + ((a >> 2) & 1)))]
            if I >= 0:
                ue[3 * a:3 * a + 3] = uo[3 * I:3 * I + 3]
        go[e] = -3.0 * rho[e] ** 2 * (ue @ Ke0 @ ue)
    assert np.abs(g - go).max() <= 1e-8 * np.abs(go).max()
    # central finite differences on 32 seeded elements (the element count of
    # the 128^3 compliance workload's check; here each perturbed solve is cheap)
    for e in W.fd_elements(p, 32):
        h = 1e-4 * rho[e]
        vals = []
        for sgn in (1.0, -1.0):
            r2 = rho.copy()
            r2[e] += sgn * h
            p2, d2 = _simp(A, n, r2)
            S2 = A.Solver(d2["rowptr"], d2["col"], d2["vals"], d2["V0"], n_coarse=300)
            x2, _, _, _ = S2.solve(d2["f"], 1e-12)
            vals.append(float(torch.dot(d2["f"], x2)))
        fd = (vals[0] - vals[1]) / (2 * h)
        assert abs(fd - g[e]) <= 1e-5 * abs(g[e]) + 1e-12 * np.abs(g).max(), (e, fd, g[e])
