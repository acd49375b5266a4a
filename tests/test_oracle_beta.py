"""Pins for the oracle's regularised incomplete beta I_x(a,b) and its inverse (paper §3.3).

Pinned by closed forms, by the binomial identity for integer parameters, by symmetry, by a
library that is run (scipy.special.betainc / betaincinv, never copied) and by brute-force
bisection on the library CDF.
"""

import math

import numpy as np
import pytest
import scipy.special as sp

GRID_AB = [0.1, 0.13, 0.26, 0.5, 1.0, 1.7, 3.0, 9.9, 25.0, 50.0, 89.1, 100.0]
GRID_P = [2.0 ** -24, 1e-6, 1e-3, 0.01, 0.1, 0.3, 0.5, 0.7, 0.9, 0.99, 0.999, 1 - 2.0 ** -24]


def close(x, y, rel=1e-12, abs_=1e-300):
    return abs(x - y) <= max(rel * max(abs(x), abs(y)), abs_)


@pytest.mark.parametrize("x", [1e-12, 1e-4, 0.1, 0.37, 0.5, 0.9, 0.999999])
def test_betainc_closed_forms(oracle, x):
    assert close(oracle.betainc(1.0, 1.0, x), x)
    for a in (0.13, 0.5, 2.0, 9.9):
        assert close(oracle.betainc(a, 1.0, x), x ** a)
    for b in (0.26, 0.5, 3.0, 89.1):
        assert close(oracle.betainc(1.0, b, x), -math.expm1(b * math.log1p(-x)), 1e-11)
    assert close(oracle.betainc(0.5, 0.5, x), 2.0 / math.pi * math.asin(math.sqrt(x)), 1e-12)


@pytest.mark.parametrize("a,b", [(1, 1), (2, 3), (3, 2), (5, 7), (10, 1), (1, 12), (20, 30)])
def test_betainc_integer_binomial_identity(oracle, a, b):
    # I_x(a,b) = P[Binomial(a+b-1, x) >= a] for integer a, b.
    n = a + b - 1
    for x in (0.01, 0.2, 0.45, 0.5, 0.8, 0.97):
        s = sum(math.comb(n, j) * x ** j * (1 - x) ** (n - j) for j in range(a, n + 1))
        assert close(oracle.betainc(a, b, x), s, 1e-11, 1e-15)


@pytest.mark.parametrize("a", GRID_AB)
@pytest.mark.parametrize("b", GRID_AB[::3])
def test_betainc_symmetry_and_library(oracle, a, b):
    # dyadic x so that 1 - x is exact (near 1 the density can exceed 1e6)
    for x in (2.0 ** -27, 2.0 ** -7, 0.1875, 0.5, 0.8125, 1 - 2.0 ** -7):
        v = oracle.betainc(a, b, x)
        w = oracle.betainc(b, a, 1.0 - x)
        assert abs(v + w - 1.0) < 1e-13
        assert close(v, sp.betainc(a, b, x), 1e-11, 1e-15)


@pytest.mark.parametrize("u", [2.0 ** -24, 1e-5, 0.05, 0.3, 0.5, 0.77, 0.999, 1 - 2.0 ** -24])
def test_betaincinv_closed_forms(oracle, u):
    x, st = oracle.betaincinv(1.0, 1.0, u)
    assert st == 0 and close(x, u)
    for a in (0.13, 0.5, 2.0, 9.9):
        x, _ = oracle.betaincinv(a, 1.0, u)
        assert close(x, u ** (1.0 / a), 1e-11)
    for b in (0.26, 0.5, 3.0, 89.1):
        x, _ = oracle.betaincinv(1.0, b, u)
        assert close(x, -math.expm1(math.log1p(-u) / b), 1e-11)
    x, _ = oracle.betaincinv(0.5, 0.5, u)
    assert close(x, math.sin(math.pi * u / 2) ** 2, 1e-11)


@pytest.mark.parametrize("a", GRID_AB)
@pytest.mark.parametrize("b", GRID_AB)
def test_betaincinv_grid_against_library(oracle, a, b):
    for p in GRID_P:
        x, st = oracle.betaincinv(a, b, p)
        assert st == 0
        ref = sp.betaincinv(a, b, p)
        # relative agreement in x, or in 1-x near the upper end
        ok = close(x, ref, 1e-10, 1e-300) or abs((1 - x) - (1 - ref)) <= 1e-10 * (1 - ref)
        assert ok, (a, b, p, x, ref)
        # round trip through the oracle's own forward function; x itself carries a rounding
        # error of ~1 ulp, which the density f(x) (large near a U-shaped end) amplifies
        if 0.0 < x < 1.0:
            pp = oracle.betainc(a, b, x)
            dens = math.exp((a - 1) * math.log(x) + (b - 1) * math.log1p(-x) - sp.betaln(a, b))
            assert abs(pp - p) <= 1e-12 * max(p, 1 - p) + 1e-15 + 4e-16 * dens * x


def test_betaincinv_bisection_brute_force(oracle):
    # Plain bisection of the library CDF (80 halvings of [0,1]) for workload-shaped parameters.
    rng = np.random.default_rng(3)
    for _ in range(40):
        s, m = rng.uniform(0.3, 1.2), rng.uniform(3, 10)
        k = (m - 1) / s ** 2 - 1
        a, b = k / m, (1 - 1 / m) * k
        p = rng.uniform(0.001, 0.999)
        lo, hi = 0.0, 1.0
        for _ in range(80):
            mid = 0.5 * (lo + hi)
            if sp.betainc(a, b, mid) < p:
                lo = mid
            else:
                hi = mid
        x, _ = oracle.betaincinv(a, b, p)
        assert abs(x - 0.5 * (lo + hi)) <= 1e-12 + 1e-9 * x


def test_betaincinv_monotone_and_limits(oracle):
    ps = np.linspace(0.0, 1.0, 401)
    for a, b in [(0.13, 0.26), (9.9, 89.1), (2.0, 5.0)]:
        xs = [oracle.betaincinv(a, b, p)[0] for p in ps]
        assert xs[0] == 0.0 and xs[-1] == 1.0
        assert all(x2 >= x1 for x1, x2 in zip(xs, xs[1:]))


def test_betaincinv_tiny_lower_tail(oracle):
    # a = 0.13: x ~ (p a B(a,b))^(1/a) is ~1e-55, far below binary32 but a normal double.
    a, b, p = 0.13, 0.26, 2.0 ** -24
    x, st = oracle.betaincinv(a, b, p)
    lnB = math.lgamma(a) + math.lgamma(b) - math.lgamma(a + b)
    approx = math.exp((math.log(p) + math.log(a) + lnB) / a)
    assert st == 0 and 1e-70 < x < 1e-40
    assert close(x, approx, 1e-6)  # small-x form is exact to O(x)
