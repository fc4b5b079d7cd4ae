"""Oracle utilities against values fixed outside the oracle: the published
SplitMix64 output sequence, and the fixed-order inner product against the
exact (rational) inner product within the rounding bound of its summation
tree."""
from fractions import Fraction

import numpy as np
import pytest


def test_splitmix64_published_sequence(orc):
    # the first outputs of the SplitMix64 generator started from state 0
    # (Steele, Lea, Flood 2014; the reference implementation's sequence)
    assert orc.splitmix64(0, 0) == 0xE220A8397B1DCDAF
    assert orc.splitmix64(0, 1) == 0x6E789E6AA1B965F4
    assert orc.splitmix64(0, 2) == 0x06C45D188009454F


def test_uniform_pm1_range_and_exactness(orc):
    u = orc.uniform_pm1(20190205, range(20000))
    assert u.min() >= -1.0 and u.max() < 1.0
    # 53-bit fractions doubled minus one: multiples of 2^-52
    assert np.all(np.ldexp(u + 1.0, 52) == np.round(np.ldexp(u + 1.0, 52)))
    assert abs(u.mean()) < 0.02


def _exact(x, y):
    return sum((Fraction(float(a)) * Fraction(float(b)) for a, b in zip(x, y)), Fraction(0))


@pytest.mark.parametrize("n", [1, 31, 32, 1023, 1024, 1025, 40000])
def test_dot_within_summation_bound(orc, n):
    """Each term passes through at most 32 fused multiply-adds, 5 exchange
    additions, ceil(nchunks / 32) chunk additions and 5 more exchanges: the
    error is at most gamma_k * sum |x_i y_i| with k that many roundings."""
    g = np.random.default_rng(n)
    x, y = g.normal(size=n), g.normal(size=n)
    d = orc.dot(x, y)
    ex = _exact(x, y)
    nch = (n + 1023) // 1024
    k = 32 + 5 + (nch + 31) // 32 + 5
    u = 2.0 ** -53
    bound = k * u / (1 - k * u) * float(np.sum(np.abs(x * y)))
    assert abs(Fraction(d) - ex) <= Fraction(bound)


def test_dot_special_cases(orc):
    assert orc.dot(np.zeros(0), np.zeros(0)) == 0.0
    x = np.zeros(5000)
    x[3071] = 3.5
    y = np.arange(5000, dtype=np.float64)
    assert orc.dot(x, y) == 3.5 * 3071.0
    # small integers: every partial sum is exact
    a = np.arange(1, 3001, dtype=np.float64)
    assert orc.dot(a, a) == float(sum(i * i for i in range(1, 3001)))
    # one fused multiply-add per term: x*y + 0 is the correctly rounded product
    p, q = 1.0 + 2.0 ** -30, 1.0 - 2.0 ** -30
    assert orc.dot(np.array([p]), np.array([q])) == float(Fraction(p) * Fraction(q))


@pytest.mark.parametrize("m", [1, 2, 7, 40])
def test_chol_factor_and_solve(orc, m):
    """The dense Cholesky factor reproduces M, its solve matches a direct
    solve within the conditioning bound, and a matrix that is not positive
    definite is refused."""
    rng = np.random.default_rng(100 + m)
    X = rng.normal(size=(m, m))
    M = X @ X.T + m * np.eye(m)
    rc, L = orc.chol(M)
    assert rc == 0
    assert np.allclose(np.triu(L, 1), 0.0)
    assert np.all(np.diag(L) > 0)
    assert np.abs(L @ L.T - M).max() <= 1e-13 * np.abs(M).max()
    b = rng.normal(size=m)
    x = orc.chol_solve(L, b)
    xr = np.linalg.solve(M, b)
    assert np.linalg.norm(x - xr) <= 1e-12 * np.linalg.cond(M) * np.linalg.norm(xr)
    if m > 1:
        Mbad = M.copy()
        Mbad[m - 1, m - 1] = -1.0
        rc2, _ = orc.chol(Mbad)
        assert rc2 != 0
