"""Parity at the paper's scale, in the benchmark's launch configuration.

800,000 trials x 1,000 events, 16 ELTs of 20,000-200,000 records over a 2,000,000-event
catalogue: the full YLT is computed on the GPU by the same ara_run call the benchmark times; the
oracle recomputes a seeded sample of trials one by one; properties that hold at any size are
checked on the rest.  The precision workload (800,000 x 100 x 1) is checked on its seeded
10,000-trial subset in both accumulation modes.
"""

import numpy as np
import pytest

from paper_1310_2274_b300 import synth

pytestmark = pytest.mark.gpu

YLT_TOL = 1e-5


@pytest.fixture(scope="module")
def paper(ara):
    w = synth.paper()
    c = ara.Context(seed=42)
    yet, elts, layer = c.stage_workload(w)
    ylt = c.run(yet, layer, 0, w.yet.n_trials)
    yield w, c, (yet, elts, layer), ylt
    c.close()


def test_paper_scale_sampled_trials(oracle, paper):
    w, c, (yet, elts, layer), ylt = paper
    pick = synth.subset_trials(w.yet.n_trials, 48, seed=7)
    pick = np.unique(np.concatenate([pick, [0, w.yet.n_trials - 1]]))
    o, nc = oracle.run(w.yet, w.elts, w.terms, 42, trials=pick, elt_handles=elts)
    assert nc == 0
    scale = np.maximum(np.maximum(np.abs(o), w.terms.agg_ret), 1.0)
    assert np.max(np.abs(ylt[pick] - o) / scale) <= YLT_TOL
    # the sample is not degenerate: the layer pays in these trials
    assert np.count_nonzero(o) >= len(pick) // 2


def test_paper_scale_newton_path_sampled(ara, oracle, paper):
    w, c, (yet, elts, layer), ylt_table = paper
    c.set_option(ara.OPT_INVERSION, ara.INV_NEWTON)
    try:
        ylt = c.run(yet, layer, 0, w.yet.n_trials)
    finally:
        c.set_option(ara.OPT_INVERSION, ara.INV_TABLE)
    pick = synth.subset_trials(w.yet.n_trials, 24, seed=11)
    o, _ = oracle.run(w.yet, w.elts, w.terms, 42, trials=pick, elt_handles=elts)
    scale = np.maximum(np.maximum(np.abs(o), w.terms.agg_ret), 1.0)
    assert np.max(np.abs(ylt[pick] - o) / scale) <= YLT_TOL
    # the two inversions agree everywhere to well inside the tolerance
    scale_all = np.maximum(ylt, w.terms.agg_ret)
    assert np.max(np.abs(ylt - ylt_table) / scale_all) <= 2e-6
    st = c.stats()
    assert st["uncertified"] <= 0.005 * sum(e.n for e in w.elts)


def test_paper_scale_properties(paper):
    w, c, _, ylt = paper
    assert ylt.shape == (800_000,)
    assert np.all(np.isfinite(ylt))
    assert np.all(ylt >= 0.0) and np.all(ylt <= w.terms.agg_lim)
    # fewer than 1% of the years sit on a bound, so the 1-in-1000 tail is not a block of ties
    at_bounds = np.count_nonzero((ylt == 0.0) | (ylt == w.terms.agg_lim))
    assert at_bounds < 0.01 * ylt.size
    assert c.not_converged() == 0


def test_paper_scale_hits_bit_exact(oracle, paper):
    w, c, (yet, elts, layer), _ = paper
    t0 = 123_456
    gh, _ = c.trace(yet, layer, t0, 3)
    oh, _ = oracle.trace(w.yet, w.elts, w.terms, 42, np.arange(t0, t0 + 3), elt_handles=elts)
    for f in ("k", "j", "rec"):
        np.testing.assert_array_equal(gh[f], oh[f])
    np.testing.assert_array_equal(gh["trial"] + t0, oh["trial"])
    np.testing.assert_array_equal(gh["u"].astype(np.float64), oh["u"])
    assert gh["k"].size > 2000  # ~880 hits per trial at this scale


def test_paper_scale_risk_measures_on_identical_ylt(oracle, paper):
    w, c, _, ylt = paper
    np.testing.assert_array_equal(c.rank(ylt), oracle.rank(ylt))
    gp, gt = c.risk_measures(ylt, w.rps)
    op, ot = oracle.risk(ylt, w.rps)
    np.testing.assert_array_equal(gp, op)
    np.testing.assert_allclose(gt, ot, rtol=1e-12)


def test_precision_workload_subset(ara, oracle):
    w = synth.precision()
    pick = synth.subset_trials(w.yet.n_trials, 10_000, seed=7)
    o, _ = oracle.run(w.yet, w.elts, w.terms, 42, trials=pick, elt_handles=[0])
    with ara.Context(seed=42) as c:
        yet, elts, layer = c.stage_workload(w)
        assert elts == [0]
        for mode in (ara.ACC_FP64, ara.ACC_KAHAN32):
            c.set_option(ara.OPT_PRECISION, mode)
            g = c.run(yet, layer, 0, w.yet.n_trials)
            scale = np.maximum(np.maximum(np.abs(o), w.terms.agg_ret), 1.0)
            assert np.max(np.abs(g[pick] - o) / scale) <= YLT_TOL, mode
