"""The stopping rule of the inversion's continued fraction (DLMF 8.17.22), studied in binary64.

The device sums K(c, d, z) in blocks of four terms and stops once the last four terms changed K
by at most kCfStop relatively, or by as much as moves the root's ln x by kCfStop (tol_g = kCfStop
c / y, capped at 1e-4).  Because the fraction gains orders of magnitude over four terms, the error
left is far below the last change.  This test runs that rule in binary64 on the roots of the
ELT value law and of extreme shapes (alpha, beta log-uniform on [0.1, 100]) and checks the error
it leaves in ln x against the exact K that scipy's incomplete beta gives: I_x = P K / c with
P = z^c (1 - z)^d / B(c, d).  A relative error e in K moves ln x by e y K / c on either side of
the threshold z = (c + 1) / (c + d + 2) (y = 1 - x of the tail solved).
"""

import os
import re

import numpy as np
import pytest

scipy_special = pytest.importorskip("scipy.special")

HERE = os.path.dirname(os.path.abspath(__file__))
IBETA = os.path.join(HERE, "..", "paper_1310_2274_b300", "csrc", "ara_ibeta.cuh")


def cf_stop():
    m = re.search(r"constexpr float kCfStop = ([0-9.eE+-]+)f;", open(IBETA).read())
    assert m, "kCfStop not found"
    return float(m.group(1))


def d_coef(n, c, d, z):
    """d_n of DLMF 8.17.22 (n >= 1)."""
    if n % 2 == 1:
        m = (n - 1) // 2
        return -(c + m) * (c + d + m) * z / ((c + 2 * m) * (c + 2 * m + 1))
    m = n // 2
    return m * (d - m) * z / ((c + 2 * m - 1) * (c + 2 * m))


def summed(c, d, z, tol, tol_g, n_max=400):
    """K = 1 / (1 + d_1 / (1 + d_2 / ...)) by the forward recurrence in blocks of four terms,
    stopped by the device's rule; returns (K, terms)."""
    a2, a1, b2, b1 = 1.0, 1.0, 0.0, 1.0  # A_{n-2}, A_{n-1}, B_{n-2}, B_{n-1}; T_n = A_n / B_n
    prev = None
    n = 0
    while True:
        for _ in range(4):
            n += 1
            dn = d_coef(n, c, d, z)
            an, bn = a1 + dn * a2, b1 + dn * b2
            s = 1.0 / abs(an)
            a2, a1, b2, b1 = a1 * s, an * s, b1 * s, bn * s
        k = b1 / a1
        if prev is not None and abs(k - prev) <= max(tol * abs(prev), tol_g * abs(prev) / abs(k)):
            return k, n
        if n >= n_max:
            return k, n
        prev = k


def roots(a0, b0, u):
    """The tail below the mean, as the inversion solves it, and the fraction's side."""
    p0 = scipy_special.betainc(a0, b0, a0 / (a0 + b0))
    flip = u > p0
    a = np.where(flip, b0, a0)
    b = np.where(flip, a0, b0)
    p = np.where(flip, 1.0 - u, u)
    x = scipy_special.betaincinv(a, b, p)
    lower = x < (a + 1.0) / (a + b + 2.0)
    c = np.where(lower, a, b)
    d = np.where(lower, b, a)
    z = np.where(lower, x, 1.0 - x)
    return c, d, z, 1.0 - x


def value_law(n, rng):
    from paper_1310_2274_b300 import synth
    elts = synth.paper_elts(16)
    mu = np.concatenate([e.mean / e.max_exposure for e in elts])
    sd = np.concatenate([e.sd / e.max_exposure for e in elts])
    keep = sd > 0
    mu, sd = mu[keep], sd[keep]
    nu = mu * (1.0 - mu) / sd ** 2 - 1.0
    i = rng.integers(0, mu.size, n)
    return mu[i] * nu[i], (1.0 - mu[i]) * nu[i]


@pytest.mark.parametrize("law", ["elt_value_law", "extreme_shapes"])
def test_fraction_stop_leaves_under_1e7_in_ln_x(law):
    rng = np.random.default_rng(17)
    n = 1500
    if law == "elt_value_law":
        a0, b0 = value_law(n, rng)
    else:
        a0, b0 = 10.0 ** rng.uniform(-1, 2, n), 10.0 ** rng.uniform(-1, 2, n)
    u = (np.floor(rng.random(n) * 2 ** 23) * 2 + 1) * 2.0 ** -24  # the uniform grid of the draws
    c, d, z, y = roots(a0, b0, u)
    # the exact fraction: I_z(c, d) = z^c (1 - z)^d / (c B(c, d)) K
    ln_pref = c * np.log(z) + d * np.log1p(-z) - scipy_special.betaln(c, d)
    k_exact = scipy_special.betainc(c, d, z) * c / np.exp(ln_pref)
    stop = cf_stop()
    worst, terms, terms_tight = 0.0, 0, 0
    for i in range(n):
        tol_g = min(stop * c[i] / y[i], 1e-4)
        k, m = summed(c[i], d[i], z[i], stop, tol_g)
        worst = max(worst, abs(k / k_exact[i] - 1.0) * y[i] * k_exact[i] / c[i])
        terms += m
        terms_tight += summed(c[i], d[i], z[i], 1.2e-7, 0.0)[1]
    assert worst <= 1e-7, worst  # under the binary32 rounding of ln x itself
    assert terms < terms_tight  # and it stops earlier than a plain 1.2e-7 bound on K
