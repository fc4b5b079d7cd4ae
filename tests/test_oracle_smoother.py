"""Pins of the oracle's aFSAI smoother (Sec. 3.1, Algorithm 3): unit diagonal of
G A G^T, the full-pattern special case (exact inverse Cholesky factor), the
first adaptive step against brute force, the Lanczos estimate against a dense
eigensolver, the omega_alpha closed form of Sec. 3.1.1 and rho(S) < 1."""
import os

import numpy as np
import pytest

import workloads as W

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


def dense_to_bsr(orc, D, b):
    n = D.shape[0] // b
    rowptr = np.arange(n + 1, dtype=np.int32) * n
    col = np.tile(np.arange(n, dtype=np.int32), n)
    val = D.reshape(n, b, n, b).transpose(0, 2, 1, 3).reshape(n * n, b, b)
    return orc.Bsr(rowptr, col, val)


def small_problem(orc, n=4, b=3, lognormal=True):
    p = W.beam(n, 3, 2) if lognormal else W.cube16(n)
    K, nm = orc.assemble(p.nx, p.ny, p.nz, p.hx, p.hy, p.hz, p.nu, p.E, p.clamp_axis)
    if b == 1:
        K = orc.to_scalar(K)
    return K


@pytest.mark.parametrize("b", [1, 3])
def test_unit_diagonal_and_lower_structure(orc, b):
    A = small_problem(orc, b=b)
    G = orc.afsai(A, None, 4, 4 if b == 1 else 2, 1e-3, 64 if b == 1 else 24)
    Gd, Ad = G.todense(), A.todense()
    S = Gd @ Ad @ Gd.T
    assert np.abs(np.diag(S) - 1.0).max() <= 1e-14 * 16
    assert np.array_equal(Gd, np.tril(Gd))
    assert np.all(np.diag(Gd) > 0)


def test_full_pattern_is_inverse_cholesky(orc):
    rng = np.random.default_rng(7)
    n, b = 5, 3
    X = rng.normal(size=(n * b, n * b))
    D = X @ X.T + n * b * np.eye(n * b)
    A = dense_to_bsr(orc, D, b)
    G = orc.afsai(A, None, 10, 10, 0.0, 24)
    L = np.linalg.cholesky(D)
    assert np.allclose(G.todense(), np.linalg.inv(L), rtol=0, atol=1e-12 * np.abs(np.linalg.inv(L)).max())
    Gd = G.todense()
    assert np.abs(Gd @ D @ Gd.T - np.eye(n * b)).max() <= 1e-12


def _row_system(Ad, rowpat, i):
    """Dense FSAI row on pattern Q (indices < i): gh, psi."""
    Q = np.array(rowpat, dtype=int)
    if len(Q):
        gh = np.linalg.solve(Ad[np.ix_(Q, Q)], -Ad[Q, i])
        psi = Ad[i, i] + Ad[i, Q] @ gh
    else:
        gh, psi = np.zeros(0), Ad[i, i]
    return gh, psi


@pytest.mark.parametrize("b", [1, 3])
def test_first_step_brute_force(orc, b):
    """One step adding one node: the chosen node maximises the squared gradient
    2 (A gt)_j of the row functional, summed over the node's dofs and rows."""
    A = small_problem(orc, b=b)
    Ad = A.todense()
    G = orc.afsai(A, None, 1, 1, 0.0, 24)
    nn = A.nr
    for I in range(nn):
        # dense unit-diagonal rows before the step: own lower dofs only
        gts = []
        for c in range(b):
            i = b * I + c
            Q = [b * I + e for e in range(c)]
            gh, _ = _row_system(Ad, Q, i)
            gt = np.zeros(Ad.shape[0])
            gt[Q] = gh
            gt[i] = 1.0
            gts.append(gt)
        grads = np.array([Ad @ gt for gt in gts])  # (b, n)
        best, bscore = None, 0.0
        for J in range(I):
            sc = np.sum(grads[:, b * J:b * J + b] ** 2)
            if sc > bscore * (1 + 1e-12) and sc > 0:
                best, bscore = J, sc
        cols = G.col[G.rowptr[I]:G.rowptr[I + 1]]
        if best is None:
            assert list(cols) == [I]
            continue
        assert list(cols) == [best, I]
        # values: scaled solution of the pattern system
        blk = G.val[G.rowptr[I]:G.rowptr[I + 1]]
        for c in range(b):
            i = b * I + c
            Q = [b * best + e for e in range(b)] + [b * I + e for e in range(c)]
            gh, psi = _row_system(Ad, Q, i)
            row = np.concatenate([blk[0][c], blk[1][c][:c]])
            assert np.allclose(row, gh / np.sqrt(psi), rtol=1e-10, atol=1e-12)
            assert np.isclose(blk[1][c][c], 1 / np.sqrt(psi), rtol=1e-12)


def test_rows_solve_their_pattern_systems(orc):
    A = small_problem(orc, n=5)
    Ad = A.todense()
    G = orc.afsai(A, None, 4, 2, 1e-3, 24)
    b = 3
    for I in range(A.nr):
        cols = G.col[G.rowptr[I]:G.rowptr[I + 1]]
        blk = G.val[G.rowptr[I]:G.rowptr[I + 1]]
        assert cols[-1] == I and np.all(np.diff(cols) > 0)
        for c in range(b):
            i = b * I + c
            Q = [b * J + e for J in cols[:-1] for e in range(b)] + [b * I + e for e in range(c)]
            gh, psi = _row_system(Ad, Q, i)
            row = np.concatenate([blk[k][c] for k in range(len(cols) - 1)] + [blk[-1][c][:c]])
            assert np.allclose(row, gh / np.sqrt(psi), rtol=1e-9, atol=1e-12)
            assert np.all(blk[-1][c][c + 1:] == 0)


def test_eps_stops_after_first_step(orc):
    A = small_problem(orc)
    G = orc.afsai(A, None, 4, 2, 1e9, 24)
    assert np.diff(G.rowptr).max() <= 3  # one step of at most two nodes + diagonal


def test_lanczos_exact_when_space_is_small(orc):
    rng = np.random.default_rng(8)
    n, b = 6, 3   # 18 dofs <= 20 Lanczos steps
    X = rng.normal(size=(n * b, n * b))
    D = X @ X.T + 0.5 * np.eye(n * b)
    A = dense_to_bsr(orc, D, b)
    G = orc.afsai(A, None, 1, 1, 0.0, 24)
    GT = orc.transpose(G)
    lam = orc.lanczos_lmax(A, G, GT, 20, 123, 0)
    Gd = G.todense()
    ev = np.linalg.eigvalsh(Gd @ D @ Gd.T)
    assert abs(lam - ev[-1]) <= 1e-10 * ev[-1]


def test_lanczos_underestimates_slightly(orc):
    A = small_problem(orc, n=6)
    G = orc.afsai(A, None, 4, 2, 1e-3, 24)
    GT = orc.transpose(G)
    lam = orc.lanczos_lmax(A, G, GT, 20, 20190205, 0)
    Gd, Ad = G.todense(), A.todense()
    lmax = np.linalg.eigvalsh(Gd @ Ad @ Gd.T)[-1]
    assert lam <= lmax * (1 + 1e-12)
    assert lam >= 0.97 * lmax


def test_omega_alpha_golden():
    """Sec. 3.1.1: omega_alpha = 2 omega / (2 + alpha omega); the paper's example
    omega = 0.922, alpha = 5 gives 0.279."""
    vals = {}
    for line in open(os.path.join(GOLDEN, "omega_alpha.txt")):
        line = line.split("#")[0].strip()
        if line:
            k, v = line.split("=")
            vals[k.strip()] = float(v)
    w, a = vals["omega"], vals["alpha"]
    assert round(2 * w / (2 + a * w), 3) == vals["omega_alpha"]


def test_omega_alpha_by_lanczos(orc):
    """Shifting the 10 largest eigenvalues of G A G^T by alpha (A' = A +
    alpha G^{-1} U U^T G^{-T}) turns the Lanczos omega into 2 omega/(2+alpha omega)."""
    rng = np.random.default_rng(9)
    n, b = 6, 3
    X = rng.normal(size=(n * b, n * b))
    D = X @ X.T + 1.0 * np.eye(n * b)
    A = dense_to_bsr(orc, D, b)
    G = orc.afsai(A, None, 1, 1, 0.0, 24)
    GT = orc.transpose(G)
    Gd = G.todense()
    w = 2.0 / orc.lanczos_lmax(A, G, GT, 20, 5, 0)
    ev, U = np.linalg.eigh(Gd @ D @ Gd.T)
    U = U[:, -10:]
    alpha = 5.0
    Gi = np.linalg.inv(Gd)
    D2 = D + alpha * Gi @ U @ U.T @ Gi.T
    D2 = 0.5 * (D2 + D2.T)
    w2 = 2.0 / orc.lanczos_lmax(dense_to_bsr(orc, D2, b), G, GT, 20, 5, 0)
    assert abs(w2 - 2 * w / (2 + alpha * w)) <= 1e-10


def test_smoother_setup_loop_and_convergence(orc):
    A = small_problem(orc, n=5)
    G, GT, om, lm, npass = orc.smoother_setup(A, orc.default_params(3), 0)
    assert npass == 0 or om < 0.95
    assert om == min(1.0, 0.95 * 2.0 / lm)
    Gd, Ad = G.todense(), A.todense()
    S = np.eye(Ad.shape[0]) - om * Gd.T @ Gd @ Ad
    assert np.abs(np.linalg.eigvals(S)).max() < 1.0
    # an unreachable omega_bar forces the refinement passes
    G2, _, om2, lm2, np2 = orc.smoother_setup(A, orc.default_params(3, omega_bar=10.0), 0)
    assert np2 >= 1 and G2.nnzb > G.nnzb
    assert np.abs(np.diag(G2.todense() @ Ad @ G2.todense().T) - 1).max() < 1e-13


def _afsai_dense(Ad, b, k, rho, eps, maxg, start=None):
    """aFSAI straight from its definition on a dense matrix: per node row, k
    steps; candidates are lower nodes outside the pattern adjacent to the
    pattern or to the row's node; the rho nodes with the largest summed squared
    gradient 2 (A gt)_j are added; stop when every row's psi decreased by at
    most eps of its previous value."""
    n = Ad.shape[0] // b
    adj = [set(J for J in range(n) if np.any(Ad[b * I:b * I + b, b * J:b * J + b] != 0)) for I in range(n)]
    pats = []
    for I in range(n):
        pat = sorted(start[I]) if start is not None else []

        def rows(pat):
            gts, psis = [], []
            for c in range(b):
                i = b * I + c
                Q = [b * J + e for J in pat for e in range(b)] + [b * I + e for e in range(c)]
                gh, psi = _row_system(Ad, Q, i)
                gt = np.zeros(Ad.shape[0])
                gt[Q] = gh
                gt[i] = 1.0
                gts.append(gt)
                psis.append(psi)
            return gts, np.array(psis)

        gts, psi = rows(pat)
        for _ in range(k):
            if len(pat) >= maxg:
                break
            cand = sorted(J for K in pat + [I] for J in adj[K] if J < I and J not in pat)
            cand = sorted(set(cand))
            sc = {J: sum(np.sum((Ad @ gt)[b * J:b * J + b] ** 2) for gt in gts) for J in cand}
            order = sorted((J for J in cand if sc[J] > 0), key=lambda J: (-sc[J], J))
            pick = order[:min(rho, maxg - len(pat))]
            if not pick:
                break
            pat = sorted(pat + pick)
            old = psi
            gts, psi = rows(pat)
            if np.all(old - psi <= eps * old):
                break
        pats.append(pat)
    return pats


@pytest.mark.parametrize("b,k,rho,eps", [(3, 3, 2, 0.0), (3, 4, 2, 1e-3), (1, 3, 4, 1e-3), (3, 2, 1, 0.0)])
def test_multistep_patterns_brute_force(orc, b, k, rho, eps):
    A = small_problem(orc, n=4, b=b)
    Ad = A.todense()
    G = orc.afsai(A, None, k, rho, eps, 24)
    ref = _afsai_dense(Ad, b, k, rho, eps, 24)
    for I in range(A.nr):
        assert list(G.col[G.rowptr[I]:G.rowptr[I + 1] - 1]) == ref[I], I
    # a continuation call grows from the given pattern
    G2 = orc.afsai(A, G, 2, rho, eps, 24)
    start = [list(G.col[G.rowptr[I]:G.rowptr[I + 1] - 1]) for I in range(A.nr)]
    ref2 = _afsai_dense(Ad, b, 2, rho, eps, 24, start=start)
    for I in range(A.nr):
        assert list(G2.col[G2.rowptr[I]:G2.rowptr[I + 1] - 1]) == ref2[I], I
