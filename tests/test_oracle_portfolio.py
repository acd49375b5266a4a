"""Pins for the oracle's portfolio run (Algorithm 1's loops over programs and layers): a layer's
year losses depend on its own ELTs and terms alone, an ELT's secondary-uncertainty draws are keyed
by the ELT (not by its place in a layer), so with terms that pass losses through, a layer's year
loss is the sum of its ELTs' year losses, and layers with the same ELTs in another order agree up
to the order of summation."""

import numpy as np

import oracle
from paper_1310_2274_b300 import synth

IDENT = synth.Terms(0.0, np.inf, 0.0, np.inf)


def workload():
    yet = synth.make_yet(300, 60, 10_000, seed=1)
    elts = [synth.make_elt(1500, 10_000, seed=s) for s in (2, 3, 4, 5)]
    return yet, elts


def test_layers_are_independent_and_ordered():
    yet, elts = workload()
    t = synth.TERMS_TINY
    pf = [[((0, 1), t), ((2,), t)], [((1, 3), IDENT)]]
    m = oracle.run_portfolio(yet, elts, pf, 42)
    assert m.shape == (3, 300)
    # the same layers in another portfolio, one at a time and in reverse program order
    rev = oracle.run_portfolio(yet, elts, [pf[1], [pf[0][1]], [pf[0][0]]], 42)
    np.testing.assert_array_equal(rev[0], m[2])
    np.testing.assert_array_equal(rev[1], m[1])
    np.testing.assert_array_equal(rev[2], m[0])
    assert np.count_nonzero(m[0]) > 100


def test_pass_through_terms_make_year_losses_additive_over_elts():
    yet, elts = workload()
    m = oracle.run_portfolio(yet, elts, [[((0,), IDENT), ((3,), IDENT), ((0, 3), IDENT),
                                          ((3, 0), IDENT)]], 42)
    scale = np.maximum(m[2], 1.0)
    # same draws for ELT 0 and ELT 3 in every layer: sums agree up to binary64 rounding
    assert np.max(np.abs(m[0] + m[1] - m[2]) / scale) <= 1e-12
    assert np.max(np.abs(m[3] - m[2]) / scale) <= 1e-12
    assert np.count_nonzero(m[0]) > 100 and np.count_nonzero(m[1]) > 100


def test_trial_selection_selects_columns():
    yet, elts = workload()
    t = synth.TERMS_TINY
    pf = [[((0, 2), t), ((1,), t)]]
    full = oracle.run_portfolio(yet, elts, pf, 42)
    pick = np.array([5, 0, 299, 17])
    part = oracle.run_portfolio(yet, elts, pf, 42, trials=pick)
    np.testing.assert_array_equal(part, full[:, pick])
