"""Pins of the oracle's test-space generation (Sec. 3.2, Algorithm 4): the step
length minimises the Rayleigh quotient along the search direction (brute
force), the Ritz step solves the generalised eigenproblem (scipy), and SRQCG
converges to the smallest eigenvectors of the pencil (A, (G^T G)^{-1})."""
import numpy as np
import pytest
import scipy.linalg as sla

from test_oracle_smoother import small_problem


def rq(S, z):
    return (z @ S @ z) / (z @ z)


def test_line_min_brute_force(orc):
    rng = np.random.default_rng(11)
    printed = 0
    for trial in range(200):
        n = 8
        X = rng.normal(size=(n, n))
        S = X @ X.T + 0.1 * np.eye(n)
        z, p = rng.normal(size=n), rng.normal(size=n)
        a, b, c, d, e, f = p @ S @ z, p @ S @ p, p @ z, p @ p, z @ S @ z, z @ z
        al = orc.rq_line_min(a, b, c, d, e, f)
        grid = np.linspace(-50, 50, 20001)
        vals = [(e + 2 * g * a + g * g * b) / (f + 2 * g * c + g * g * d) for g in grid]
        assert rq(S, z + al * p) <= min(vals) + 1e-12 * abs(min(vals))
        # stationary point: the quotient's derivative vanishes
        h = 1e-6 * max(1.0, abs(al))
        der = (rq(S, z + (al + h) * p) - rq(S, z + (al - h) * p)) / (2 * h)
        assert abs(der) <= 1e-5 * abs(rq(S, z)) / max(1.0, abs(al))
        de_bf, bc_ad, af_ce = d * e - b * f, b * c - a * d, a * f - c * e
        delta = de_bf ** 2 - 4 * bc_ad * af_ce
        if abs(al - (de_bf + np.sqrt(delta)) / (2 * bc_ad)) <= 1e-9 * max(1, abs(al)):
            printed += 1
    # the root printed in Algorithm 4 is the minimiser in the generic case
    assert printed >= 190


def test_gen_eig_matches_scipy(orc):
    rng = np.random.default_rng(12)
    for t in (1, 4, 10):
        X = rng.normal(size=(t, t))
        H = X + X.T
        Y = rng.normal(size=(t, t))
        M = Y @ Y.T + t * np.eye(t)
        lam, U = orc.gen_eig(H, M)
        ref = sla.eigh(H, M, eigvals_only=True)
        assert np.allclose(lam, ref, rtol=0, atol=1e-12 * np.abs(ref).max())
        assert np.allclose(H @ U, M @ U @ np.diag(lam), atol=1e-11 * np.abs(H).max())
        assert np.allclose(U.T @ M @ U, np.eye(t), atol=1e-12)
        for j in range(t):
            assert U[np.argmax(np.abs(U[:, j])), j] > 0


def test_gen_eig_equal_diagonal_and_repeated_eigenvalues(orc):
    """Pivots with C_pp = C_qq (the 45-degree rotation, d = 0 in the rotation
    formula, with either sign of C_pq) and a pencil with a repeated eigenvalue."""
    for off in (0.5, -0.5):
        H = np.array([[1.0, off], [off, 1.0]])
        lam, U = orc.gen_eig(H, np.eye(2))
        assert np.allclose(lam, [0.5, 1.5], rtol=0, atol=1e-15)
        assert np.allclose(H @ U, U @ np.diag(lam), atol=1e-15)
    rng = np.random.default_rng(14)
    Q, _ = np.linalg.qr(rng.normal(size=(6, 6)))
    H = Q @ np.diag([1.0, 2.0, 2.0, 2.0, 3.0, -1.0]) @ Q.T
    H = (H + H.T) / 2
    lam, U = orc.gen_eig(H, np.eye(6))
    assert np.allclose(lam, [-1.0, 1.0, 2.0, 2.0, 2.0, 3.0], rtol=0, atol=1e-13)
    assert np.allclose(U.T @ U, np.eye(6), atol=1e-13)
    assert np.allclose(H @ U, U @ np.diag(lam), atol=1e-13)


def test_mgs_orthonormal(orc):
    V = np.random.default_rng(13).normal(size=(500, 7))
    Q = orc.mgs(V)
    assert np.allclose(Q.T @ Q, np.eye(7), atol=1e-13)
    # same column spaces, column by column
    for j in range(1, 8):
        ang = sla.subspace_angles(Q[:, :j], V[:, :j])
        assert ang.max() < 1e-10


def _pencil(orc, A, G):
    Gd, Ad = G.todense(), A.todense()
    return Ad, np.linalg.inv(Gd.T @ Gd), Gd


def test_srqcg_converges_to_eigenvectors(orc):
    A = small_problem(orc, n=3, lognormal=False)
    G = orc.afsai(A, None, 2, 2, 1e-3, 24)
    GT = orc.transpose(G)
    Ad, M, Gd = _pencil(orc, A, G)
    n, t = Ad.shape[0], 4
    V0 = np.random.default_rng(14).normal(size=(n, t))
    ev, X = sla.eigh(Ad, M)
    # one column: conjugate-gradient minimisation of the Rayleigh quotient
    # converges to the lowest eigenvector of the pencil (A, (G^T G)^{-1})
    v1 = orc.srqcg(A, G, GT, V0[:, :1], kmax=200, k_ritz=1)
    assert sla.subspace_angles(v1, X[:, :1]).max() < 1e-6
    # a block: the lower Ritz pairs converge.  (Algorithm 4 minimises each
    # column's quotient without orthogonality constraints between Ritz steps,
    # so the top column keeps being pulled towards the span of the others and
    # lags; the paper runs n_rq = 10 iterations.)
    V = orc.srqcg(A, G, GT, V0, kmax=60, k_ritz=1)
    rv, Y = sla.eigh(V.T @ Ad @ V, V.T @ M @ V)
    assert np.allclose(rv[:t - 1], ev[:t - 1], rtol=1e-8, atol=0)
    W_ = V @ Y[:, :t - 1]
    res = Ad @ W_ - M @ W_ @ np.diag(rv[:t - 1])
    assert np.abs(res).max() <= 1e-6 * np.abs(Ad).max() * np.abs(W_).max()
    assert np.allclose(V.T @ V, np.eye(t), atol=1e-13)


def test_srqcg_lowest_ritz_value_decreases(orc):
    A = small_problem(orc, n=4)
    G = orc.afsai(A, None, 4, 2, 1e-3, 24)
    GT = orc.transpose(G)
    Ad, M, Gd = _pencil(orc, A, G)
    n, t = Ad.shape[0], 6
    V0 = np.random.default_rng(15).normal(size=(n, t))
    # after a Ritz step the first column holds the lowest Ritz vector and its
    # line minimisation can only lower it, so the lowest Ritz value of the
    # block never increases and stays above the pencil's lowest eigenvalue
    prev = np.inf
    for kmax in range(0, 12):
        V = orc.srqcg(A, G, GT, V0, kmax=kmax, k_ritz=1)
        s = sla.eigh(V.T @ Ad @ V, V.T @ M @ V, eigvals_only=True)[0]
        assert s <= prev * (1 + 1e-10)
        prev = s
    lowest = sla.eigh(Ad, M, eigvals_only=True)[0]
    assert prev >= lowest * (1 - 1e-10)


def test_padding_generator_statistics(orc):
    u = orc.uniform_pm1(20190205, range(20000))
    assert u.min() >= -1.0 and u.max() < 1.0
    assert abs(u.mean()) < 0.02 and abs(u.var() - 1 / 3) < 0.01
    assert len(np.unique(u)) == len(u)
