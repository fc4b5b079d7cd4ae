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


def _mgs_plain(V):
    """Modified Gram-Schmidt in column order, then unit columns."""
    V = V.copy()
    for j in range(V.shape[1]):
        for i in range(j):
            V[:, j] -= (V[:, i] @ V[:, j]) * V[:, i]
        V[:, j] /= np.linalg.norm(V[:, j])
    return V


def _line_min_plain(a, b, c, d, e, f):
    """The stationary points of rq(alpha) = (e + 2 alpha a + alpha^2 b) /
    (f + 2 alpha c + alpha^2 d), i.e. the roots of (bc - ad) alpha^2 +
    (bf - de) alpha + (af - ce) = 0, and the one with the smaller quotient."""
    qa, qb, qc = b * c - a * d, b * f - d * e, a * f - c * e
    if qa == 0.0:
        return -qc / qb if qb != 0.0 else 0.0
    disc = qb * qb - 4 * qa * qc
    if disc < 0:
        return 0.0
    roots = [(-qb + s * np.sqrt(disc)) / (2 * qa) for s in (1.0, -1.0)]
    return min(roots, key=lambda al: (e + 2 * al * a + al * al * b) / (f + 2 * al * c + al * al * d))


def _srqcg_plain(S, Gd, V0, kmax, k_ritz):
    """Algorithm 4 as printed, with the dense S = G A G^T applied afresh
    wherever the algorithm names S Z_i, S P_i (no recurrences), the Rayleigh
    quotient of a column z as z^T S z / z^T z, f_i = 1 after a Ritz step, the
    Ritz vectors from scipy (ascending, each signed by its largest entry) and
    a column with p^T S p <= 0 left as it is."""
    n, t = V0.shape
    Z = _mgs_plain(V0 - S @ V0)
    P = np.empty_like(Z)
    f = np.ones(t)
    for i in range(t):
        z = Z[:, i]
        q = z @ S @ z
        P[:, i] = 2 * (S @ z - q * z)
    for k in range(1, kmax + 1):
        if k_ritz > 0 and k % k_ritz == 0:
            lam, U = sla.eigh(Z.T @ S @ Z, Z.T @ Z)
            for j in range(t):
                if U[np.argmax(np.abs(U[:, j])), j] < 0:
                    U[:, j] = -U[:, j]
            Z = Z @ U
            f[:] = 1.0
        for i in range(t):
            z, p = Z[:, i].copy(), P[:, i].copy()
            a, b, c, d, e = p @ S @ z, p @ S @ p, p @ z, p @ p, z @ S @ z
            if not b > 0:
                continue
            alpha = _line_min_plain(a, b, c, d, e, f[i])
            z = z + alpha * p
            fi = z @ z
            q = (z @ S @ z) / fi
            g = 2 * (S @ z - q * z) / fi
            beta = -(g @ S @ p) / b
            P[:, i] = g + beta * p
            Z[:, i] = z
            f[i] = fi
    return _mgs_plain(Gd.T @ Z)


@pytest.mark.parametrize("b", [1, 3])
def test_srqcg_matches_plain_algorithm4(orc, b):
    """The oracle's SRQCG (S Z and S P carried by recurrences, fused
    multiply-adds, fixed-order sums) against Algorithm 4 restated in numpy with
    S applied afresh each time: the same test space up to rounding."""
    A = small_problem(orc, n=3, b=b)
    G = orc.afsai(A, None, 2, 2 if b == 3 else 4, 1e-3, 24 if b == 3 else 64)
    GT = orc.transpose(G)
    Gd, Ad = G.todense(), A.todense()
    S = Gd @ Ad @ Gd.T
    n, t = Ad.shape[0], 4
    V0 = np.random.default_rng(16).normal(size=(n, t))
    for kmax in (0, 1, 10):
        V = orc.srqcg(A, G, GT, V0, kmax=kmax, k_ritz=1)
        Vp = _srqcg_plain(S, Gd, V0, kmax, 1)
        assert np.abs(V - Vp).max() <= 1e-9, (kmax, np.abs(V - Vp).max())
    # and without Ritz steps (k_ritz = 0: pure per-column CG on the quotient)
    V = orc.srqcg(A, G, GT, V0, kmax=10, k_ritz=0)
    Vp = _srqcg_plain(S, Gd, V0, 10, 0)
    assert np.abs(V - Vp).max() <= 1e-9


def test_coarse_test_space_starts_from_injection(orc):
    """A coarser level's test space is SRQCG on that level (its A and G)
    started from the finer level's test space restricted to the coarse nodes,
    in increasing fine-node order (the coarse numbering of P's columns)."""
    import workloads as W
    from _problems import oracle_problem
    p = W.beam(24, 6, 6)
    K, V0, f, nm = oracle_problem(orc, p)
    prm = orc.default_params(3, n_coarse=300)
    H = orc.Hierarchy(K, V0, prm)
    assert H.nlev >= 3
    for k in range(H.nlev - 2):
        cf = H.cf(k)
        C = np.flatnonzero(cf == 1)
        # P's C rows are identity blocks onto the coarse nodes numbered by
        # increasing fine index
        P = H.matrix(k, "P")
        for j, I in enumerate(C):
            assert P.rowptr[I + 1] - P.rowptr[I] == 1 and P.col[P.rowptr[I]] == j
            assert np.array_equal(P.val[P.rowptr[I]], np.eye(3))
        rows = (3 * C[:, None] + np.arange(3)).reshape(-1)
        Vin = H.V(k)[rows]
        A1, G1, GT1 = H.matrix(k + 1, "A"), H.matrix(k + 1, "G"), H.matrix(k + 1, "GT")
        V1 = orc.srqcg(A1, G1, GT1, Vin, kmax=prm.n_rq, k_ritz=prm.k_ritz)
        assert np.array_equal(V1, H.V(k + 1)), k
