"""Pins for the oracle's moment matching and secondary-uncertainty loss (paper §3.3).

Loss = max_l * InvCDF_beta(z; alpha, beta) must have mean mu and standard deviation sigma when
sigma_beta is within its bound, and standard deviation sigma_beta_max (1 - 2^-20) max_l when
clamped. Checked by quadrature of the quantile function (deterministic, tight) and by Philox
sampling (statistical, 5 standard errors).
"""

import math

import numpy as np
import pytest


def quad_moments(oracle, mean, sd, mx, n=4000):
    # E[g(Q(U))] = integral_0^1 g(Q(u)) du by Gauss-Legendre on [0,1] split into 40 panels,
    # with the endpoint panels graded, where the quantile function is least smooth.
    nodes, weights = np.polynomial.legendre.leggauss(n // 40)
    edges = np.concatenate([[0.0], np.geomspace(1e-12, 1e-2, 12), np.linspace(0.02, 0.98, 15),
                            1 - np.geomspace(1e-2, 1e-12, 12), [1.0]])
    m1 = m2 = 0.0
    for lo, hi in zip(edges[:-1], edges[1:]):
        u = 0.5 * (hi - lo) * nodes + 0.5 * (hi + lo)
        w = 0.5 * (hi - lo) * weights
        loss = np.array([oracle.su_loss(mean, sd, mx, float(v))[0] for v in u])
        m1 += float(np.dot(w, loss))
        m2 += float(np.dot(w, loss * loss))
    return m1, math.sqrt(max(m2 - m1 * m1, 0.0))


@pytest.mark.parametrize("s,m", [(0.3, 3.0), (1.2, 3.0), (0.3, 10.0), (1.2, 10.0), (0.7, 5.5)])
def test_moment_matching_quadrature(oracle, s, m):
    mean = 1.6e5
    sd, mx = s * mean, m * mean
    rc, a, b = oracle.beta_moments(mean, sd, mx)
    assert rc == 0
    # Beta(a,b) has mean a/(a+b) and variance ab/((a+b)^2 (a+b+1)); scaled by max_l.
    assert math.isclose(a / (a + b) * mx, mean, rel_tol=1e-13)
    var = a * b / ((a + b) ** 2 * (a + b + 1))
    assert math.isclose(math.sqrt(var) * mx, sd, rel_tol=1e-13)
    m1, sdq = quad_moments(oracle, mean, sd, mx)
    assert math.isclose(m1, mean, rel_tol=2e-6)
    assert math.isclose(sdq, sd, rel_tol=2e-5)


def test_moment_matching_philox_sample(oracle):
    mean, sd, mx = 2.0e5, 1.6e5, 1.1e6
    n = 60_000
    losses = np.array([oracle.su_loss(mean, sd, mx, oracle.su_uniform(42, i, 0, 0))[0]
                       for i in range(n)])
    se = sd / math.sqrt(n)
    assert abs(losses.mean() - mean) < 5 * se
    # variance of the sample variance for a bounded variable: use a loose 5% band
    assert abs(losses.std() / sd - 1.0) < 0.05
    assert losses.min() >= 0.0 and losses.max() <= mx


def test_clamped_standard_deviation(oracle):
    # sigma_beta > sigma_beta_max = sqrt(mu_b (1 - mu_b)) -> clamped just below the bound.
    mean, mx = 1.0, 2.0
    sd = 1.5  # sigma_b = 0.75 > 0.5
    rc, a, b = oracle.beta_moments(mean, sd, mx)
    assert rc == 1
    mu_b = 0.5
    sb = math.sqrt(mu_b * (1 - mu_b)) * (1 - 2.0 ** -20)
    var = a * b / ((a + b) ** 2 * (a + b + 1))
    assert math.isclose(math.sqrt(var), sb, rel_tol=1e-9)
    assert math.isclose(a / (a + b), mu_b, rel_tol=1e-12)
    m1, sdq = quad_moments(oracle, mean, sd, mx, n=2000)
    assert math.isclose(m1, mean, rel_tol=1e-4)
    assert math.isclose(sdq, sb * mx, rel_tol=1e-3)


def test_zero_sigma_is_the_mean(oracle):
    # sigma = 0 leaves only primary uncertainty: the loss is the mean, whatever the uniform.
    for u in (2.0 ** -24, 0.3, 1 - 2.0 ** -24):
        v, st = oracle.su_loss(123456.0, 0.0, 999999.0, u)
        assert v == 123456.0 and st == 0


def test_invalid_records(oracle):
    assert oracle.beta_moments(5.0, 1.0, 5.0)[0] == -1  # max must exceed the mean
    assert oracle.beta_moments(-1.0, 1.0, 5.0)[0] == -1
    assert oracle.beta_moments(1.0, -1.0, 5.0)[0] == -1
