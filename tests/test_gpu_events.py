"""Event-level outputs on the device against the FP64 oracle: the OEP year table (each year's
largest occurrence loss) and the per-occurrence outputs (occurrence loss after occurrence terms,
increment of the year's net aggregate loss), on 3,000 trials of the paper-scale layer (2,000,000
event catalogue, 16 ELTs) and on a ragged YET with empty trials."""

import numpy as np
import pytest

from paper_1310_2274_b300 import synth

pytestmark = pytest.mark.gpu

TOL = 1e-5  # the binary32 occurrence results against binary64, as for the year losses
N = 3000


@pytest.fixture(scope="module")
def staged(ara, oracle):
    w = synth.paper(n_trials=N)
    c = ara.Context(seed=42)
    yet, elts, layer = c.stage_workload(w)
    ref = oracle.run_events(w.yet, w.elts, w.terms, 42, elt_handles=elts)
    yield c, w, yet, elts, layer, ref
    c.close()


def n_occ(w, t0, n):
    return int(w.yet.offsets[t0 + n] - w.yet.offsets[t0])


def check_against_oracle(w, terms, got, ref, t0=0, n=None):
    n = w.yet.n_trials if n is None else n
    ylt, oep, olt, inc = got
    o_ylt, o_oep, o_olt, o_inc, _ = ref
    a, b = w.yet.offsets[t0], w.yet.offsets[t0 + n]
    o_olt, o_inc = o_olt[a:b], o_inc[a:b]
    # occurrence losses: binary32 against binary64, relative to the retention they cancel against
    assert np.max(np.abs(olt - o_olt) / np.maximum(np.maximum(o_olt, terms.occ_ret), 1.0),
                  initial=0.0) <= TOL
    assert np.max(np.abs(oep - o_oep[t0:t0 + n]) /
                  np.maximum(np.maximum(o_oep[t0:t0 + n], terms.occ_ret), 1.0)) <= TOL
    assert np.max(np.abs(ylt - o_ylt[t0:t0 + n]) /
                  np.maximum(np.maximum(np.abs(o_ylt[t0:t0 + n]), terms.agg_ret), 1.0)) <= TOL
    # increments: an error in the running sum moves value between neighbouring increments, so
    # they are compared on the scale of the year's total occurrence loss
    lens = np.diff(w.yet.offsets[t0:t0 + n + 1])
    scale = np.maximum(np.maximum(np.repeat(seg_sums(o_olt, lens), lens), terms.agg_ret), 1.0)
    assert np.max(np.abs(inc - o_inc) / scale, initial=0.0) <= 2 * TOL
    # the device's own increments add up to its year losses
    assert np.all(np.abs(seg_sums(inc, lens) - ylt) <= 1e-12 * np.maximum(ylt, 1.0) + 1e-6)


def seg_sums(x, lens):
    """Per-trial sums of a per-occurrence array (trials of length lens, in order)."""
    out = np.zeros(len(lens))
    nz = lens > 0
    if x.size:
        out[nz] = np.add.reduceat(x, np.r_[0, np.cumsum(lens)[:-1]][nz])
    return out


def test_events_match_oracle(ara, staged):
    c, w, yet, elts, layer, ref = staged
    got = c.run_events(yet, layer, 0, N, n_occ(w, 0, N))
    check_against_oracle(w, w.terms, got, ref)
    ylt, oep, olt, inc = got
    assert olt.dtype == np.float32 and inc.dtype == np.float64
    assert np.count_nonzero(inc) > 100 and np.count_nonzero(olt) > 10_000
    # the YLT and OEP of the same pass equal the band-major run's
    y_b, e_b = c.run_ep(yet, layer, 0, N)
    np.testing.assert_array_equal(ylt, y_b)
    np.testing.assert_array_equal(oep, e_b)
    # the OEP year table is the maximum of the year's occurrence losses
    for i in range(0, N, 97):
        seg = olt[w.yet.offsets[i]:w.yet.offsets[i + 1]]
        assert oep[i] == (seg.max() if seg.size else 0.0)


def test_events_on_binding_aggregate_terms(ara, oracle, staged):
    # terms placed inside the distribution of year sums: retention crossed mid-year by most
    # trials, limit exhausted by some
    c, w, yet, elts, _, ref = staged
    o_ylt, _, o_olt, _, _ = ref
    sums = seg_sums(o_olt, np.diff(w.yet.offsets))
    agg_ret, top = np.quantile(sums, [0.2, 0.7])
    terms = synth.Terms(w.terms.occ_ret, w.terms.occ_lim, float(agg_ret), float(top - agg_ret))
    layer = c.add_layer(elts, terms.occ_ret, terms.occ_lim, terms.agg_ret, terms.agg_lim)
    try:
        got = c.run_events(yet, layer, 0, N, n_occ(w, 0, N))
    finally:
        c.free_layer(layer)
    ref2 = oracle.run_events(w.yet, w.elts, terms, 42, elt_handles=elts)
    check_against_oracle(w, terms, got, ref2)
    ylt = got[0]
    assert np.count_nonzero(ylt == terms.agg_lim) > N // 10
    assert np.count_nonzero(ylt == 0.0) > N // 10


def test_event_ranges_and_device_outputs(ara, staged):
    c, w, yet, elts, layer, ref = staged
    full = c.run_events(yet, layer, 0, N, n_occ(w, 0, N))
    dev = c.run_events(yet, layer, 0, N, n_occ(w, 0, N), device=True)
    for a, b in zip(full, dev):
        np.testing.assert_array_equal(a, b.cpu().numpy())
    for t0, n in [(0, 1), (5, 129), (N - 1, 1), (1000, N - 1000)]:
        part = c.run_events(yet, layer, t0, n, n_occ(w, t0, n))
        a, b = w.yet.offsets[t0], w.yet.offsets[t0 + n]
        np.testing.assert_array_equal(part[0], full[0][t0:t0 + n])
        np.testing.assert_array_equal(part[1], full[1][t0:t0 + n])
        np.testing.assert_array_equal(part[2], full[2][a:b])
        np.testing.assert_array_equal(part[3], full[3][a:b])


def test_kahan_precision_and_increments(ara, staged):
    c, w, yet, elts, layer, ref = staged
    full = c.run_events(yet, layer, 0, 500, n_occ(w, 0, 500))
    c.set_option(ara.OPT_PRECISION, ara.ACC_KAHAN32)
    try:
        with pytest.raises(ara.AraError) as e:
            c.run_events(yet, layer, 0, 500, n_occ(w, 0, 500))
        assert e.value.status == 1
        # occurrence losses alone do not depend on the year accumulator
        _, oep, olt, inc = c.run_events(yet, layer, 0, 500, n_occ(w, 0, 500), increments=False)
    finally:
        c.set_option(ara.OPT_PRECISION, ara.ACC_FP64)
    assert inc is None
    np.testing.assert_array_equal(olt, full[2])
    np.testing.assert_array_equal(oep, full[1])


def test_events_ragged_yet_with_empty_trials(ara, oracle):
    rng = np.random.default_rng(12)
    lens = rng.choice([0, 0, 1, 2, 31, 33, 600], size=400)
    lens[-3:] = 0  # a range made only of empty trials at the end
    offsets = np.zeros(401, dtype=np.int64)
    np.cumsum(lens, out=offsets[1:])
    ids = rng.integers(0, 2_000_000, size=int(offsets[-1]), dtype=np.int32)
    yet_h = synth.Yet(offsets, ids, np.zeros(ids.shape[0], np.float32), 2_000_000)
    w = synth.Workload("ragged", yet_h, synth.paper_elts(4), synth.Terms(2e5, 2e7, 1e7, 1e9),
                       synth.RPS_PAPER)
    with ara.Context(seed=42) as c:
        yet, elts, layer = c.stage_workload(w)
        got = c.run_events(yet, layer, 0, 400, int(offsets[-1]))
        empty = c.run_events(yet, layer, 397, 3, 0)
    ref = oracle.run_events(yet_h, w.elts, w.terms, 42, elt_handles=elts)
    check_against_oracle(w, w.terms, got, ref)
    assert np.all(got[0][lens == 0] == 0.0) and np.all(got[1][lens == 0] == 0.0)
    assert empty[2].shape == (0,) and empty[3].shape == (0,)
    np.testing.assert_array_equal(empty[0], np.zeros(3))


def test_increments_are_the_formula_on_the_devices_own_sums(ara, staged):
    # S_k is the exact sum of the occurrence losses on the grid 2^e (e fixed by the longest trial
    # and OccL so that a year fits in 52 bits); the increments must be A(S_k) - A(S_k - o_k) in
    # binary64 bit for bit, including the regions where the kernel skips the formula
    c, w, yet, elts, layer, ref = staged
    max_len = int(np.diff(w.yet.offsets).max())
    for agg_ret, agg_lim in [(w.terms.agg_ret, w.terms.agg_lim), (3.0e8 + 0.3, 7.7e7 + 0.1),
                             (0.0, 1e15), (1e15, 1.0)]:
        t = synth.Terms(w.terms.occ_ret, w.terms.occ_lim, agg_ret, agg_lim)
        l2 = c.add_layer(elts, t.occ_ret, t.occ_lim, t.agg_ret, t.agg_lim)
        try:
            ylt, _, olt, inc = c.run_events(yet, l2, 0, 400, n_occ(w, 0, 400))
        finally:
            c.free_layer(l2)
        e = int(np.ceil(np.log2(float(np.float32(t.occ_lim)) * max_len))) - 52
        units = np.rint(olt.astype(np.float64) * 2.0 ** -e).astype(np.int64)
        lens = np.diff(w.yet.offsets[:401])
        trial = np.repeat(np.arange(400), lens)
        s1 = np.cumsum(units)
        first = np.r_[0, np.cumsum(lens)[:-1]]
        s1 = s1 - np.repeat(np.r_[0, s1][first], lens)  # restart at every trial
        s0 = s1 - units

        def A(s):
            return np.minimum(np.maximum(s.astype(np.float64) * 2.0 ** e - agg_ret, 0.0), agg_lim)

        np.testing.assert_array_equal(inc, A(s1) - A(s0))
        last = np.cumsum(lens) - 1
        nz = lens > 0
        np.testing.assert_array_equal(ylt[nz], A(s1[last[nz]]))
        assert trial.shape == inc.shape
