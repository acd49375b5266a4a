"""Pins for the oracle's event-level outputs (Algorithm 1 with the terms of §2.3 applied after
every event): per occurrence, the loss after occurrence terms and the increment of the year's net
aggregate loss.  Checked against the per-hit trace (a second route through the oracle), the
telescoping of the increments to the year loss, the bounds a clamp implies, the retention and
limit regions, and the identity aggregate terms."""

import numpy as np

import oracle
from paper_1310_2274_b300 import synth


def ragged_workload(seed=4, n=300):
    w = synth.tiny(200)
    rng = np.random.default_rng(seed)
    lens = rng.choice([0, 1, 1, 2, 7, 40, 90], size=n)
    offsets = np.zeros(n + 1, dtype=np.int64)
    np.cumsum(lens, out=offsets[1:])
    ids = rng.integers(0, w.yet.catalog_size, size=int(offsets[-1]), dtype=np.int32)
    yet = synth.Yet(offsets, ids, np.zeros(ids.shape[0], np.float32), w.yet.catalog_size)
    return yet, w.elts, w.terms, lens


def test_run_events_agrees_with_run():
    yet, elts, terms, _ = ragged_workload()
    y0, e0, _ = oracle.run(yet, elts, terms, 42, with_oep=True)
    y1, e1, olt, inc, nc = oracle.run_events(yet, elts, terms, 42)
    assert nc == 0
    np.testing.assert_array_equal(y0, y1)
    np.testing.assert_array_equal(e0, e1)
    assert olt.shape == inc.shape == (int(yet.offsets[-1]),)


def test_occurrence_losses_against_the_hit_trace():
    yet, elts, terms, lens = ragged_workload(n=80)
    _, oep, olt, _, _ = oracle.run_events(yet, elts, terms, 42)
    hits, _ = oracle.trace(yet, elts, terms, 42, np.arange(80))
    for i in range(80):
        for k in range(int(lens[i])):
            sel = (hits["trial"] == i) & (hits["k"] == k)
            l = sum(float(v) for v in hits["loss"][sel])  # layer order, left to right
            o = min(max(l - terms.occ_ret, 0.0), terms.occ_lim)
            assert olt[yet.offsets[i] + k] == o, (i, k)
        seg = olt[yet.offsets[i]:yet.offsets[i + 1]]
        assert oep[i] == (seg.max() if seg.size else 0.0)


def test_increments_telescope_and_obey_the_clamps():
    yet, elts, terms, lens = ragged_workload()
    ylt, _, olt, inc, _ = oracle.run_events(yet, elts, terms, 42)
    assert np.all(inc >= 0.0)
    assert np.all(inc <= olt * (1 + 1e-15) + 1e-9)
    for i in range(len(lens)):
        a, b = yet.offsets[i], yet.offsets[i + 1]
        # the year's net loss is the sum of its increments (each is a difference of consecutive
        # partial results, so only their rounding separates the two)
        assert abs(inc[a:b].sum() - ylt[i]) <= 1e-12 * max(ylt[i], 1.0) + 1e-9
        cum_after = np.cumsum(olt[a:b])
        cum_before = cum_after - olt[a:b]
        # nothing is paid until the running sum passes the retention, nothing once the limit is
        # used up (small margins keep the cumulative sums' rounding out of the check)
        below = cum_after <= terms.agg_ret * (1 - 1e-12)
        above = cum_before >= (terms.agg_ret + terms.agg_lim) * (1 + 1e-12)
        assert np.all(inc[a:b][below] == 0.0)
        assert np.all(inc[a:b][above] == 0.0)
    assert np.count_nonzero(inc) > 100


def test_identity_aggregate_terms_pass_occurrence_losses_through():
    yet, elts, terms, _ = ragged_workload(seed=5)
    ident = synth.Terms(terms.occ_ret, terms.occ_lim, 0.0, np.inf)
    ylt, _, olt, inc, _ = oracle.run_events(yet, elts, ident, 42)
    # inc_k = (S_{k-1} + o_k) - S_{k-1} in binary64: o_k up to the rounding of the running sum
    cum = np.concatenate([[0.0], np.cumsum(olt)])
    tol = 2.0 ** -52 * np.maximum(cum[1:], 1.0) * 2
    assert np.all(np.abs(inc - olt) <= tol)
    assert np.count_nonzero(olt) > 100


def test_limit_crossing_pays_the_rest_of_the_limit():
    # one trial whose occurrences overrun a small aggregate layer: nothing before the retention,
    # the part of the crossing occurrence above it, whole occurrences, the rest of the limit at
    # the occurrence that exhausts it, then nothing
    yet, elts, terms, lens = ragged_workload(seed=6)
    _, _, olt0, _, _ = oracle.run_events(yet, elts, terms, 42)
    i = int(np.argmax(lens))
    a, b = yet.offsets[i], yet.offsets[i + 1]
    o = olt0[a:b]
    nz = np.flatnonzero(o)
    assert nz.size >= 6
    cum = np.cumsum(o)
    lo = float(cum[nz[1]] - 0.5 * o[nz[1]])   # retention: half-way through occurrence nz[1]
    hi = float(cum[nz[4]] - 0.25 * o[nz[4]])  # retention + limit: 3/4 through occurrence nz[4]
    t2 = synth.Terms(terms.occ_ret, terms.occ_lim, lo, hi - lo)
    ylt, _, olt, inc, _ = oracle.run_events(yet, elts, t2, 42, trials=np.array([i]))
    np.testing.assert_array_equal(olt, o)
    tol = 1e-12 * hi
    assert abs(ylt[0] - (hi - lo)) <= tol
    assert np.all(inc[:nz[1]] == 0.0)
    assert abs(inc[nz[1]] - 0.5 * o[nz[1]]) <= tol
    for k in (nz[2], nz[3]):
        assert abs(inc[k] - o[k]) <= tol
    assert abs(inc[nz[4]] - 0.75 * o[nz[4]]) <= tol
    assert np.all(inc[nz[4] + 1:] == 0.0)
    assert np.count_nonzero(inc) == 4


def test_selected_trials_are_concatenated_in_selection_order():
    yet, elts, terms, lens = ragged_workload()
    _, _, olt, inc, _ = oracle.run_events(yet, elts, terms, 42)
    pick = np.array([17, 3, 250, 3])
    _, _, o2, i2, _ = oracle.run_events(yet, elts, terms, 42, trials=pick)
    want_o = np.concatenate([olt[yet.offsets[t]:yet.offsets[t + 1]] for t in pick])
    want_i = np.concatenate([inc[yet.offsets[t]:yet.offsets[t + 1]] for t in pick])
    np.testing.assert_array_equal(o2, want_o)
    np.testing.assert_array_equal(i2, want_i)
