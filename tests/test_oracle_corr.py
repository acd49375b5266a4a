"""Pins for the oracle's combination of independent and correlated standard deviations (paper
§3.1-3.2): the normal distribution against scipy, the two extreme cases the paper names
(sigma_I = 0 and sigma_C = 0), the marginal uniformity of the combined uniform, the correlation
the combination implies between two records of one occurrence, and the run with sigma_C = 0
against the single-SD run."""

import numpy as np
import scipy.special as sp
import scipy.stats as st

import oracle
from paper_1310_2274_b300 import synth


def test_norm_cdf_and_quantile_against_scipy():
    xs = np.concatenate([np.linspace(-37, 8, 451), [0.0, 1e-12, -1e-12]])
    for x in xs:
        # Phi's relative condition number is about x^2 in the lower tail: rounding x / sqrt 2
        # alone moves the value by ~1e-16 (1 + x^2) relative
        tol = 4e-16 * (1.0 + x * x) * sp.ndtr(x)
        assert abs(oracle.norm_cdf(x) - sp.ndtr(x)) <= tol + 1e-300, x
    ps = np.concatenate([10.0 ** -np.arange(1, 300, 7), np.linspace(0.01, 0.99, 99),
                         1 - 10.0 ** -np.arange(1, 15)])
    for p in ps:
        q = oracle.norm_quantile(p)
        assert abs(q - sp.ndtri(p)) <= 1e-13 * max(1.0, abs(q)), (p, q, sp.ndtri(p))
    assert oracle.norm_quantile(0.5) == 0.0
    assert abs(oracle.norm_quantile(0.975) - 1.959963984540054) <= 1e-14
    # symmetry and round trip
    for p in (1e-9, 0.01, 0.2, 0.4999):
        assert abs(oracle.norm_quantile(p) + oracle.norm_quantile(1 - p)) <= 1e-9 * abs(oracle.norm_quantile(p)) + 1e-15
        assert abs(oracle.norm_cdf(oracle.norm_quantile(p)) - p) <= 1e-14 * p


def test_combination_extremes():
    rng = np.random.default_rng(1)
    for zp, ze in rng.uniform(1e-6, 1 - 1e-6, size=(50, 2)):
        # sigma_C = 0: the program/occurrence uniform, exactly
        assert oracle.su_combine(zp, ze, 3.0, 0.0) == zp
        # sigma_I = 0: the occurrence uniform (through Phi(Phi^-1(ze)))
        assert abs(oracle.su_combine(zp, ze, 0.0, 5.0) - ze) <= 1e-14
        # equal SDs: v = (vp + ve) / sqrt 2, written with scipy
        want = sp.ndtr((sp.ndtri(zp) + sp.ndtri(ze)) / np.sqrt(2.0))
        assert abs(oracle.su_combine(zp, ze, 2.0, 2.0) - want) <= 1e-13


def test_combined_uniform_is_uniform_and_correlates_records():
    rng = np.random.default_rng(2)
    n = 40_000
    zp1, zp2, ze = rng.uniform(size=(3, n))
    # two records of one occurrence: independent parts differ, the correlated part is shared
    wi1, wc1, wi2, wc2 = 0.7, 0.3, 0.4, 0.6
    z1 = np.array([oracle.su_combine(a, c, wi1, wc1) for a, c in zip(zp1, ze)])
    z2 = np.array([oracle.su_combine(b, c, wi2, wc2) for b, c in zip(zp2, ze)])
    for z in (z1, z2):
        assert st.kstest(z, "uniform").pvalue > 1e-3
    # normal scores correlate by c1 c2, c = w_c / sqrt(w_i^2 + w_c^2)
    c1 = wc1 / np.hypot(wi1, wc1)
    c2 = wc2 / np.hypot(wi2, wc2)
    r = np.corrcoef(sp.ndtri(z1), sp.ndtri(z2))[0, 1]
    assert abs(r - c1 * c2) <= 4.0 / np.sqrt(n)


def test_correlated_uniform_is_shared_and_distinct_from_elt_uniforms():
    u = oracle.su_uniform_corr(42, 17, 3)
    assert u == oracle.su_uniform_corr(42, 17, 3)
    assert u != oracle.su_uniform_corr(42, 17, 4) and u != oracle.su_uniform_corr(42, 18, 3)
    # word 0 of counter (k, i_lo, 0xFFFFFFFF, i_hi), key (seed_lo, seed_hi)
    w = oracle.philox4x32_10([3, 17, 0xFFFFFFFF, 0], [42, 0])
    assert u == ((2 * (int(w[0]) >> 9) + 1) * 2.0 ** -24)


def test_run_with_zero_correlated_sd_equals_single_sd_run():
    w = synth.tiny(200)
    e = w.elts[0]
    zero = synth.Elt(e.event_ids, e.mean, e.sd, e.max_exposure, np.zeros(e.n))
    a, _ = oracle.run(w.yet, [e], w.terms, 42)
    b, _ = oracle.run(w.yet, [zero], w.terms, 42)
    np.testing.assert_array_equal(a, b)


def test_run_with_split_sd_keeps_the_loss_moments():
    # sigma = sigma_I + sigma_C feeds the beta moments, and the combined uniform is U(0,1), so a
    # record's losses keep its mean: one event in every trial, one record
    n_trials = 4000
    offsets = np.arange(n_trials + 1, dtype=np.int64)
    yet = synth.Yet(offsets, np.zeros(n_trials, np.int32), np.zeros(n_trials, np.float32), 1)
    e = synth.Elt(np.array([0], np.int32), np.array([1e5]), np.array([3e4]), np.array([6e5]),
                  np.array([5e4]))
    terms = synth.Terms(0.0, 1e12, 0.0, 1e15)
    y, _ = oracle.run(yet, [e], terms, 42)
    se = y.std() / np.sqrt(n_trials)
    assert abs(y.mean() - 1e5) <= 5 * se
    assert abs(y.std() - 8e4) <= 0.05 * 8e4  # sigma = 3e4 + 5e4
