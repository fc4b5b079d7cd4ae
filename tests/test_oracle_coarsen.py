"""Pins of the oracle's coarsening (Sec. 3.3): the affinity SoC (its scalar
formula, range, symmetry and invariances), the theta filter, and the MIS
against brute force and against an independent parallel (Luby-style) rule."""
import itertools

import numpy as np
import pytest

from test_oracle_smoother import small_problem


def rand_V(n, t, seed):
    return np.random.default_rng(seed).normal(size=(n, t))


@pytest.mark.parametrize("b", [1, 3])
def test_soc_range_symmetry_invariance(orc, b):
    A = small_problem(orc, b=b)
    n = A.nr * b
    V = rand_V(n, 10, 21)
    s = orc.soc(A, V)
    assert np.all(s >= 0) and np.all(s <= 1 + 1e-15)
    pos = {}
    for I in range(A.nr):
        for k in range(A.rowptr[I], A.rowptr[I + 1]):
            pos[(I, A.col[k])] = k
    for (I, J), k in pos.items():
        assert s[k] == s[pos[(J, I)]]
        if I == J:
            assert s[k] == 0
    # invariant under an orthogonal change of the test-space basis
    Q, _ = np.linalg.qr(np.random.default_rng(22).normal(size=(10, 10)))
    assert np.allclose(orc.soc(A, V @ Q), s, rtol=1e-12, atol=1e-14)
    # invariant under scaling the rows of one node
    sc = np.repeat(np.random.default_rng(23).uniform(0.1, 10, size=A.nr), b)
    assert np.allclose(orc.soc(A, V * sc[:, None]), s, rtol=1e-12, atol=1e-14)


def test_soc_scalar_formula(orc):
    """b = 1 is the paper's affinity (v_i^T v_j)^2 / ((v_i^T v_i)(v_j^T v_j))."""
    A = small_problem(orc, b=1)
    V = rand_V(A.nr, 10, 24)
    s = orc.soc(A, V)
    for I in range(A.nr):
        for k in range(A.rowptr[I], A.rowptr[I + 1]):
            J = A.col[k]
            if J == I:
                continue
            vi, vj = V[I], V[J]
            assert np.isclose(s[k], (vi @ vj) ** 2 / ((vi @ vi) * (vj @ vj)), rtol=1e-12)


def test_soc_collinear_blocks_are_one(orc):
    A = small_problem(orc, b=3)
    rng = np.random.default_rng(25)
    base = rng.normal(size=(3, 10))
    V = np.zeros((A.nr * 3, 10))
    for I in range(A.nr):
        Q, _ = np.linalg.qr(rng.normal(size=(3, 3)))
        V[3 * I:3 * I + 3] = rng.uniform(0.5, 2) * Q @ base
    s = orc.soc(A, V)
    off = np.array([A.col[k] != I for I in range(A.nr) for k in range(A.rowptr[I], A.rowptr[I + 1])])
    assert np.allclose(s[off], 1.0, rtol=1e-12)


def test_filter_keeps_theta_largest(orc):
    A = small_problem(orc, n=5)
    s = orc.soc(A, rand_V(A.nr * 3, 10, 26))
    theta = 5
    kept, strong = orc.filter_soc(A, s, theta)
    for I in range(A.nr):
        ks = range(A.rowptr[I], A.rowptr[I + 1])
        offd = [k for k in ks if A.col[k] != I]
        order = sorted(offd, key=lambda k: (-s[k], A.col[k]))
        assert set(k for k in offd if kept[k]) == set(order[:theta])
    pos = {(I, A.col[k]): k for I in range(A.nr) for k in range(A.rowptr[I], A.rowptr[I + 1])}
    for (I, J), k in pos.items():
        assert strong[k] == (kept[k] or kept[pos[(J, I)]])


def _graph(A, strong):
    adj = [set() for _ in range(A.nr)]
    for I in range(A.nr):
        for k in range(A.rowptr[I], A.rowptr[I + 1]):
            if strong[k] and A.col[k] != I:
                adj[I].add(int(A.col[k]))
    return adj


def _luby_fixed_weights(adj):
    """Parallel rounds: an undecided node whose (degree, -index) beats every
    undecided neighbour joins C; neighbours of C become F."""
    n = len(adj)
    w = [(len(adj[i]), -i) for i in range(n)]
    state = [-1] * n
    while -1 in state:
        winners = [i for i in range(n) if state[i] == -1 and
                   all(state[j] != -1 or w[i] > w[j] for j in adj[i])]
        for i in winners:
            state[i] = 1
        for i in winners:
            for j in adj[i]:
                if state[j] == -1:
                    state[j] = 0
    return state


def test_mis_independent_maximal_and_parallel_equal(orc):
    for n, seed in ((4, 27), (5, 28)):
        A = small_problem(orc, n=n)
        s = orc.soc(A, rand_V(A.nr * 3, 10, seed))
        _, strong = orc.filter_soc(A, s, 3)
        cf = orc.mis(A, strong)
        adj = _graph(A, strong)
        C = {i for i in range(A.nr) if cf[i] == 1}
        for i in C:
            assert not (adj[i] & C)                       # independent
        for i in range(A.nr):
            assert i in C or (adj[i] & C)                 # maximal
        assert list(cf) == _luby_fixed_weights(adj)


def test_mis_brute_force_tiny_graphs(orc):
    """On tiny random graphs the result is the greedy maximal independent set
    in (degree desc, index asc) order, found here by exhaustive search: the
    lexicographically first maximal independent set in that order."""
    rng = np.random.default_rng(29)
    for trial in range(30):
        n = int(rng.integers(2, 9))
        M = np.triu(rng.random((n, n)) < 0.35, 1)
        M = M | M.T
        rowptr = [0]
        col = []
        for i in range(n):
            cs = sorted(set(np.nonzero(M[i])[0].tolist()) | {i})
            col += cs
            rowptr.append(len(col))
        A = orc.Bsr(np.array(rowptr), np.array(col), np.zeros((len(col), 1, 1)))
        strong = np.array([1 if col[k] != i else 0 for i in range(n)
                           for k in range(rowptr[i], rowptr[i + 1])], np.uint8)
        cf = orc.mis(A, strong)
        order = sorted(range(n), key=lambda i: (-M[i].sum(), i))
        best = None
        for bits in itertools.product([0, 1], repeat=n):
            S = [i for i in range(n) if bits[i]]
            if any(M[i, j] for i in S for j in S):
                continue
            if any(not bits[i] and not any(M[i, j] for j in S) for i in range(n)):
                continue
            key = [bits[i] for i in order]
            if best is None or key > best[0]:
                best = (key, bits)
        assert list(cf) == list(best[1])
