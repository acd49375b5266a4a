"""Band-major schedule of the table path against the trial-major one and the FP64 oracle.

The workload has the paper's 2,000,000-event catalogue and 16 ELTs, so a layer is cut into 31
bands of 65,536 events, on 3,000 trials (oracle-checkable).  Both schedules make the same hits,
uniforms and table evaluations, sum each event's ELT losses the same way and sum years exactly
(integer grid units), so their year losses are identical bit for bit.
"""

import numpy as np
import pytest

from paper_1310_2274_b300 import synth

pytestmark = pytest.mark.gpu

YLT_TOL = 1e-5
N = 3000


@pytest.fixture(scope="module")
def staged(ara):
    w = synth.paper(n_trials=N)
    c = ara.Context(seed=42)
    c.set_option(ara.OPT_SCHEDULE, ara.SCHED_BAND)
    yet, elts, layer = c.stage_workload(w)
    # under ARA_SCHED_BAND the layer's band-major YET copy is made by its first run (5 launches):
    # make it here, so that the tests count the launches of runs alone
    s0 = c.stats()
    c.run(yet, layer, 0, 1)
    assert c.stats()["launches"] - s0["launches"] == 2 + 5
    yield c, w, yet, elts, layer
    c.close()


def run_sched(ara, c, yet, layer, sched, t0=0, n=N):
    c.set_option(ara.OPT_SCHEDULE, sched)
    try:
        c.run(yet, layer, t0, 1)  # a layer's first band-schedule run makes its band-major YET copy
        s0 = c.stats()
        y = c.run(yet, layer, t0, n)
        s1 = c.stats()
    finally:
        c.set_option(ara.OPT_SCHEDULE, ara.SCHED_BAND)
    return y, {k: s1[k] - s0[k] for k in s0}


def scale_of(o, terms):
    return np.maximum(np.maximum(np.abs(o), terms.agg_ret), 1.0)


def test_band_schedule_matches_oracle(ara, oracle, staged):
    c, w, yet, elts, layer = staged
    g, d = run_sched(ara, c, yet, layer, ara.SCHED_BAND)
    o, nc = oracle.run(w.yet, w.elts, w.terms, 42, elt_handles=elts)
    assert nc == 0
    err = np.abs(g - o) / scale_of(o, w.terms)
    assert err.max() <= YLT_TOL, err.max()
    assert d["launches"] == 2  # band kernel + band-order finalisation
    assert d["table_evals"] > 0.99 * d["hits"]


def test_band_and_trial_schedules_agree(ara, staged):
    c, w, yet, elts, layer = staged
    gb, db = run_sched(ara, c, yet, layer, ara.SCHED_BAND)
    gt, dt = run_sched(ara, c, yet, layer, ara.SCHED_TRIAL)
    # identical work
    for k in ("hits", "table_evals", "inversions", "newton", "cf_terms"):
        assert db[k] == dt[k], k
    # the same binary32 occurrence results, summed exactly
    np.testing.assert_array_equal(gb, gt)
    assert np.count_nonzero(gb) > N // 2


def test_kahan_precision_runs_trial_major(ara, oracle, staged):
    # the Kahan-compensated binary32 year sum depends on the order of additions, so it keeps the
    # trial-major schedule (one launch) whatever the schedule option says
    c, w, yet, elts, layer = staged
    c.set_option(ara.OPT_PRECISION, ara.ACC_KAHAN32)
    try:
        g, d = run_sched(ara, c, yet, layer, ara.SCHED_BAND, 0, 500)
    finally:
        c.set_option(ara.OPT_PRECISION, ara.ACC_FP64)
    assert d["launches"] == 1
    o, _ = oracle.run(w.yet, w.elts, w.terms, 42, trials=np.arange(500), elt_handles=elts)
    assert np.max(np.abs(g - o) / scale_of(o, w.terms)) <= YLT_TOL


def test_band_results_do_not_depend_on_the_trial_range(ara, staged):
    c, w, yet, elts, layer = staged
    full, _ = run_sched(ara, c, yet, layer, ara.SCHED_BAND)
    # ranges that start inside a block's and a warp's trial tile, single trials, the last trial
    for t0, n in [(0, 1), (1, 15), (5, 129), (127, 300), (N - 1, 1), (1000, N - 1000)]:
        part, _ = run_sched(ara, c, yet, layer, ara.SCHED_BAND, t0, n)
        np.testing.assert_array_equal(part, full[t0:t0 + n])


def test_band_schedule_ragged_yet(ara, oracle):
    # empty trials, trials of one event and long trials over the paper catalogue
    rng = np.random.default_rng(9)
    lens = rng.choice([0, 0, 1, 2, 15, 16, 17, 33, 900, 2500], size=700)
    offsets = np.zeros(701, dtype=np.int64)
    np.cumsum(lens, out=offsets[1:])
    ids = rng.integers(0, 2_000_000, size=int(offsets[-1]), dtype=np.int32)
    ts = np.concatenate([np.sort(rng.uniform(0, 365, size=m)).astype(np.float32) for m in lens])
    yet_h = synth.Yet(offsets, ids, ts, 2_000_000)
    elts_h = synth.paper_elts(3)
    terms = synth.TERMS_PAPER
    with ara.Context(seed=42) as c:
        yet = c.create_yet(yet_h.offsets, yet_h.event_ids, yet_h.timestamps, 2_000_000)
        elts = [c.add_elt(yet, e.event_ids, e.mean, e.sd, e.max_exposure) for e in elts_h]
        layer = c.add_layer(elts, terms.occ_ret, terms.occ_lim, 1e7, terms.agg_lim)
        g, d = run_sched(ara, c, yet, layer, ara.SCHED_BAND, 0, 700)
        gt, _ = run_sched(ara, c, yet, layer, ara.SCHED_TRIAL, 0, 700)
    o, _ = oracle.run(yet_h, elts_h, synth.Terms(terms.occ_ret, terms.occ_lim, 1e7, terms.agg_lim),
                      42, elt_handles=elts)
    lens = np.diff(yet_h.offsets)
    assert (lens == 0).any()
    assert d["launches"] == 2
    scale = np.maximum(np.maximum(np.abs(o), 1e7), 1.0)
    assert np.max(np.abs(g - o) / scale) <= YLT_TOL
    np.testing.assert_array_equal(g, gt)
    assert np.all(g[lens == 0] == 0.0)


def run_ep_sched(ara, c, yet, layer, sched, t0=0, n=N, device=False):
    c.set_option(ara.OPT_SCHEDULE, sched)
    try:
        if device:
            import torch
            y = torch.zeros(n, dtype=torch.float64, device="cuda")
            e = torch.zeros(n, dtype=torch.float64, device="cuda")
            c.run_ep(yet, layer, t0, n, out=y, oep=e)
            return y.cpu().numpy(), e.cpu().numpy()
        return c.run_ep(yet, layer, t0, n)
    finally:
        c.set_option(ara.OPT_SCHEDULE, ara.SCHED_BAND)


def test_oep_matches_oracle_and_both_schedules_agree(ara, oracle, staged):
    # event-level output: each year's largest occurrence loss, from the same pass as the YLT
    c, w, yet, elts, layer = staged
    yb, eb = run_ep_sched(ara, c, yet, layer, ara.SCHED_BAND)
    yt, et = run_ep_sched(ara, c, yet, layer, ara.SCHED_TRIAL)
    o_y, o_e, nc = oracle.run(w.yet, w.elts, w.terms, 42, elt_handles=elts, with_oep=True)
    assert nc == 0
    scale = np.maximum(np.maximum(o_e, w.terms.occ_ret), 1.0)
    assert np.max(np.abs(eb - o_e) / scale) <= YLT_TOL
    np.testing.assert_array_equal(eb, et)  # a maximum of the same binary32 values
    assert np.count_nonzero(eb) > N // 2
    # the YLT of the same pass is the YLT of ara_run
    y, _ = run_sched(ara, c, yet, layer, ara.SCHED_BAND)
    np.testing.assert_array_equal(yb, y)
    np.testing.assert_array_equal(yt, y)
    # OEP values are binary32 occurrence results, capped by the occurrence limit
    assert np.all(eb == eb.astype(np.float32)) and np.all(eb <= w.terms.occ_lim)


def test_oep_device_output_and_trial_ranges(ara, staged):
    c, w, yet, elts, layer = staged
    y_full, e_full = run_ep_sched(ara, c, yet, layer, ara.SCHED_BAND)
    y_dev, e_dev = run_ep_sched(ara, c, yet, layer, ara.SCHED_BAND, device=True)
    np.testing.assert_array_equal(y_dev, y_full)
    np.testing.assert_array_equal(e_dev, e_full)
    for sched in (ara.SCHED_BAND, ara.SCHED_TRIAL):
        for t0, n in [(0, 1), (5, 129), (N - 1, 1), (1000, N - 1000)]:
            _, e = run_ep_sched(ara, c, yet, layer, sched, t0, n)
            np.testing.assert_array_equal(e, e_full[t0:t0 + n])


def test_oep_is_independent_of_the_year_accumulator(ara, staged):
    # Kahan year sums (trial-major) change the YLT's rounding, never the per-event maximum
    c, w, yet, elts, layer = staged
    _, e_ref = run_ep_sched(ara, c, yet, layer, ara.SCHED_BAND, 0, 500)
    c.set_option(ara.OPT_PRECISION, ara.ACC_KAHAN32)
    try:
        _, e_k = run_ep_sched(ara, c, yet, layer, ara.SCHED_BAND, 0, 500)
    finally:
        c.set_option(ara.OPT_PRECISION, ara.ACC_FP64)
    np.testing.assert_array_equal(e_k, e_ref)


def test_oep_ragged_yet_and_newton_path(ara, oracle):
    rng = np.random.default_rng(11)
    lens = rng.choice([0, 0, 1, 2, 31, 33, 600], size=500)
    offsets = np.zeros(501, dtype=np.int64)
    np.cumsum(lens, out=offsets[1:])
    ids = rng.integers(0, 2_000_000, size=int(offsets[-1]), dtype=np.int32)
    yet_h = synth.Yet(offsets, ids, np.zeros(ids.shape[0], np.float32), 2_000_000)
    elts_h = synth.paper_elts(4)
    terms = synth.Terms(2e5, 2e7, 1e7, 1e9)
    o_y, o_e, _ = oracle.run(yet_h, elts_h, terms, 42, elt_handles=[0, 1, 2, 3], with_oep=True)
    with ara.Context(seed=42) as c:
        yet = c.create_yet(yet_h.offsets, yet_h.event_ids, yet_h.timestamps, 2_000_000)
        elts = [c.add_elt(yet, e.event_ids, e.mean, e.sd, e.max_exposure) for e in elts_h]
        assert elts == [0, 1, 2, 3]
        layer = c.add_layer(elts, terms.occ_ret, terms.occ_lim, terms.agg_ret, terms.agg_lim)
        _, eb = run_ep_sched(ara, c, yet, layer, ara.SCHED_BAND, 0, 500)
        c.set_option(ara.OPT_INVERSION, ara.INV_NEWTON)
        try:
            _, en = c.run_ep(yet, layer, 0, 500)
        finally:
            c.set_option(ara.OPT_INVERSION, ara.INV_TABLE)
    scale = np.maximum(np.maximum(o_e, terms.occ_ret), 1.0)
    for e in (eb, en):
        assert np.max(np.abs(e - o_e) / scale) <= YLT_TOL
        assert np.all(e[lens == 0] == 0.0)
    assert np.count_nonzero(o_e) > 100


def test_dense_64_elt_layer_splits_events_and_overflows_the_hit_map(ara, oracle):
    # the widest layer (64 ELTs) over a 300-event catalogue that every ELT covers in full: each
    # occurrence meets 64 records, so an event's hits span two rounds (split 32 hits from its
    # first) and a chunk's 8,192 hits overflow the 512-entry hit map (events found by search);
    # trials of 0, 1, 129 and 3,000 events
    rng = np.random.default_rng(13)
    lens = np.array([0, 1, 129, 3000, 7, 0, 260, 1])
    offsets = np.zeros(lens.size + 1, dtype=np.int64)
    np.cumsum(lens, out=offsets[1:])
    ids = rng.integers(0, 300, size=int(offsets[-1]), dtype=np.int32)
    yet_h = synth.Yet(offsets, ids, np.zeros(ids.shape[0], np.float32), 300)
    elts_h = []
    for s in range(64):
        e = synth.make_elt(300, 300, seed=500 + s)
        elts_h.append(e)
    assert all(e.n == 300 for e in elts_h)
    terms = synth.Terms(1e6, 5e8, 1e8, 1e12)
    n = lens.size
    with ara.Context(seed=42) as c:
        yet = c.create_yet(yet_h.offsets, yet_h.event_ids, yet_h.timestamps, 300)
        elts = [c.add_elt(yet, e.event_ids, e.mean, e.sd, e.max_exposure) for e in elts_h]
        c.set_option(ara.OPT_BAND_WIDTH, 11)  # one band holds the whole catalogue
        layer = c.add_layer(elts, terms.occ_ret, terms.occ_lim, terms.agg_ret, terms.agg_lim)
        gb, db = run_sched(ara, c, yet, layer, ara.SCHED_BAND, 0, n)
        gt, dt = run_sched(ara, c, yet, layer, ara.SCHED_TRIAL, 0, n)
    assert db["launches"] == 2 and dt["launches"] == 1  # band kernel + finalisation; trial kernel
    assert db["hits"] == dt["hits"] == 64 * int(offsets[-1])
    np.testing.assert_array_equal(gb, gt)
    o, nc = oracle.run(yet_h, elts_h, terms, 42, elt_handles=elts)
    assert nc == 0
    scale = np.maximum(np.maximum(np.abs(o), terms.agg_ret), 1.0)
    assert np.max(np.abs(gb - o) / scale) <= YLT_TOL
    assert np.all(gb[lens == 0] == 0.0) and np.count_nonzero(gb) >= 4


def test_auto_schedule_buys_the_band_copy_once_it_pays(ara):
    """ARA_SCHED_AUTO (the default) runs trial-major (one launch) until the YET's table runs
    reach ARA_BAND_BUY_PASSES passes of its occurrences, then makes the band-major copy (5
    launches) and runs band-major (band kernel and finalisation) from then on; every run gives
    the same year losses, bit for bit."""
    w = synth.paper(n_trials=N)
    with ara.Context(seed=42) as c:
        yet, elts, layer = c.stage_workload(w)
        launches, ylts = [], []
        for _ in range(5):
            s0 = c.stats()["launches"]
            ylts.append(c.run(yet, layer, 0, N))
            launches.append(c.stats()["launches"] - s0)
        # whole-YET runs: passes 1 and 2 rent, the third reaches 3 passes and buys
        assert ara.BAND_BUY_PASSES == 3.0
        assert launches == [1, 1, 5 + 2, 2, 2], launches
        for y in ylts[1:]:
            np.testing.assert_array_equal(y, ylts[0])
        # runs over part of the trials count their share of the occurrences
        c2 = ara.Context(seed=42)
        yet2, elts2, layer2 = c2.stage_workload(w)
        got = []
        for _ in range(6):
            s0 = c2.stats()["launches"]
            c2.run(yet2, layer2, 0, N // 2)
            got.append(c2.stats()["launches"] - s0)
        c2.close()
        assert got == [1, 1, 1, 1, 1, 5 + 2], got
