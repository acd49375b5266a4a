"""Host-resident YETs: runs stream the trials they need from host memory in chunks (copy stream,
a ring of device buffers, the first chunks copied ahead when the YET is created) while earlier
chunks are validated and run.  Results must equal the
device-resident YET's trial-major runs bit for bit, for any trial range, chunk size and output
set; invalid chunks are reported after the run without any of their trials being computed."""

import numpy as np
import pytest
import torch

from paper_1310_2274_b300 import synth

pytestmark = pytest.mark.gpu

N = 3000


def pinned(a):
    t = torch.from_numpy(np.ascontiguousarray(a)).pin_memory()
    return t, t.numpy()


@pytest.fixture(scope="module")
def pair(ara):
    """The paper-scale layer (2,000,000-event catalogue, 16 ELTs) on 3,000 trials, staged on a
    resident YET in one context and on a host-resident one (page-locked arrays) in another, so
    that the ELTs have the same handles (which key their draws) in both."""
    w = synth.paper(n_trials=N)
    keep = [pinned(x) for x in (w.yet.offsets, w.yet.event_ids, w.yet.timestamps)]
    off, ids, ts = (k[1] for k in keep)
    cr = ara.Context(seed=42)
    res_yet, _, res_layer = cr.stage_workload(w)
    ch = ara.Context(seed=42)
    h_yet = ch.create_yet_host(off, ids, ts, 2_000_000)
    h_elts = [ch.add_elt(h_yet, e.event_ids, e.mean, e.sd, e.max_exposure) for e in w.elts]
    t = w.terms
    h_layer = ch.add_layer(h_elts, t.occ_ret, t.occ_lim, t.agg_ret, t.agg_lim)
    cr.set_option(ara.OPT_SCHEDULE, ara.SCHED_TRIAL)
    yield (cr, ch), w, (res_yet, res_layer), (h_yet, h_layer), keep
    ch.close()
    cr.close()


def n_occ(w, t0, n):
    return int(w.yet.offsets[t0 + n] - w.yet.offsets[t0])


@pytest.mark.parametrize("chunk", [1 << 26, 1 << 18, 1024])
def test_streamed_runs_equal_resident_runs(ara, pair, chunk):
    (cr, ch), w, (ry, rl), (hy, hl), _ = pair
    ch.set_option(ara.OPT_STREAM_CHUNK, chunk)
    try:
        for t0, n in [(0, N), (7, 1500), (N - 1, 1), (1234, 567)]:
            np.testing.assert_array_equal(ch.run(hy, hl, t0, n), cr.run(ry, rl, t0, n))
    finally:
        ch.set_option(ara.OPT_STREAM_CHUNK, 1 << 26)


def test_streamed_event_outputs_and_newton(ara, pair):
    (cr, ch), w, (ry, rl), (hy, hl), _ = pair
    ch.set_option(ara.OPT_STREAM_CHUNK, 1 << 18)
    try:
        for t0, n in [(0, N), (100, 900)]:
            got = ch.run_events(hy, hl, t0, n, n_occ(w, t0, n))
            want = cr.run_events(ry, rl, t0, n, n_occ(w, t0, n))
            for a, b in zip(got, want):
                np.testing.assert_array_equal(a, b)
        for c in (cr, ch):
            c.set_option(ara.OPT_INVERSION, ara.INV_NEWTON)
        np.testing.assert_array_equal(ch.run(hy, hl, 0, N), cr.run(ry, rl, 0, N))
    finally:
        for c in (cr, ch):
            c.set_option(ara.OPT_INVERSION, ara.INV_TABLE)
        ch.set_option(ara.OPT_STREAM_CHUNK, 1 << 26)


def test_streamed_run_matches_oracle(ara, oracle, pair):
    (_, ch), w, _, (hy, hl), _ = pair
    g = ch.run(hy, hl, 0, 800)
    o, _ = oracle.run(w.yet, w.elts, w.terms, 42, trials=np.arange(800),
                      elt_handles=list(range(16)))
    scale = np.maximum(np.maximum(np.abs(o), w.terms.agg_ret), 1.0)
    assert np.max(np.abs(g - o) / scale) <= 1e-5


def test_invalid_chunks_are_reported(ara):
    # event ids outside the catalogue in one trial (checked per chunk on the device before the
    # chunk, whose trials are then skipped), timestamps out of order in another (checked on host
    # threads during the run): the run fails and writes nothing
    rng = np.random.default_rng(3)
    lens = np.full(400, 50)
    off = np.zeros(401, dtype=np.int64)
    np.cumsum(lens, out=off[1:])
    ids = rng.integers(0, 10_000, size=int(off[-1]), dtype=np.int32)
    ts = np.tile(np.linspace(0, 365, 50, dtype=np.float32), 400)
    elt = synth.make_elt(2_000, 10_000, seed=2)
    for bad in ("id", "ts"):
        ids2, ts2 = ids.copy(), ts.copy()
        if bad == "id":
            ids2[off[300] + 7] = 10_000
        else:
            ts2[off[120] + 3] = -1.0
        with ara.Context(seed=42) as c:
            c.set_option(ara.OPT_STREAM_CHUNK, 4096)
            y = c.create_yet_host(off, ids2, ts2, 10_000)
            e = c.add_elt(y, elt.event_ids, elt.mean, elt.sd, elt.max_exposure)
            layer = c.add_layer([e], 0.0, 1e9, 0.0, 1e12)
            out = np.full(400, -7.0)
            with pytest.raises(ara.AraError) as ex:
                c.run(y, layer, 0, 400, out=out)
            assert ex.value.status == 1
            assert np.all(out == -7.0)  # outputs are written only on success
            if bad == "id":
                # ids are checked chunk by chunk on the device: a range before the bad trial runs
                assert c.run(y, layer, 0, 100).shape == (100,)
            else:
                # timestamps are checked for the whole YET on host threads: every run fails
                with pytest.raises(ara.AraError):
                    c.run(y, layer, 0, 100)


def test_host_yet_restrictions(ara, pair):
    (_, ch), w, _, (hy, hl), _ = pair
    with pytest.raises(ara.AraError):
        ch.run_portfolio(hy, [hl], 0, 10)
    with pytest.raises(ara.AraError):  # asynchronous calls (a non-default stream)
        ch.run(hy, hl, 0, 10, out=torch.zeros(10, dtype=torch.float64, device="cuda"),
               stream=torch.cuda.Stream())


def staged_host(ara, w, keep, chunk):
    """A fresh context (ELT handles 0..15, as in the resident one) with a host-resident YET
    created under the given chunk size, so its first chunks are copied ahead."""
    off, ids, ts = (k[1] for k in keep)
    c = ara.Context(seed=42)
    c.set_option(ara.OPT_STREAM_CHUNK, chunk)
    y = c.create_yet_host(off, ids, ts, 2_000_000)
    elts = [c.add_elt(y, e.event_ids, e.mean, e.sd, e.max_exposure) for e in w.elts]
    t = w.terms
    return c, y, c.add_layer(elts, t.occ_ret, t.occ_lim, t.agg_ret, t.agg_lim)


@pytest.mark.parametrize("first", [(0, N), (0, 300), (5, N - 5), (0, 1)])
def test_chunks_copied_ahead(ara, pair, first):
    # chunks of 2^18 occurrences (~262 trials): the ring of buffers wraps several times; the first
    # run uses the chunks copied ahead when it starts at trial 0 (all of them, or only the first
    # when it ends inside the second), none otherwise; later runs stream everything
    (cr, _), w, (ry, rl), _, keep = pair
    c, y, layer = staged_host(ara, w, keep, 1 << 18)
    try:
        t0, n = first
        np.testing.assert_array_equal(c.run(y, layer, t0, n), cr.run(ry, rl, t0, n))
        np.testing.assert_array_equal(c.run(y, layer, 0, N), cr.run(ry, rl, 0, N))
    finally:
        c.close()


def test_copied_ahead_chunks_of_another_yet(ara, pair):
    # two host YETs created back to back: the second one's chunks are in the ring, so the run over
    # the first streams all of its own; the second's run then finds its chunks gone and streams
    # too; a YET freed before any run waits for its copies
    (cr, _), w, (ry, rl), _, keep = pair
    off, ids, ts = (k[1] for k in keep)
    c, y, layer = staged_host(ara, w, keep, 1 << 18)
    try:
        y2 = c.create_yet_host(off, ids, ts, 2_000_000)
        np.testing.assert_array_equal(c.run(y, layer, 0, N), cr.run(ry, rl, 0, N))
        c.free_yet(y2)
        y3 = c.create_yet_host(off, ids, ts, 2_000_000)
        c.free_yet(y3)
        np.testing.assert_array_equal(c.run(y, layer, 0, 700), cr.run(ry, rl, 0, 700))
    finally:
        c.close()


@pytest.mark.parametrize("kind", ["pinned", "cuda"])
def test_elt_inputs_read_in_place(ara, pair, kind):
    # ELT arrays in page-locked host memory or on the device are read in place by the staging
    # kernel (pageable ones are copied first, as in the resident context): the same records give
    # bit-identical runs, and a bad record read in place is still rejected
    (cr, _), w, (ry, rl), _, _ = pair

    def conv(a, dt):
        t = torch.from_numpy(np.ascontiguousarray(a, dtype=dt))
        return t.pin_memory() if kind == "pinned" else t.cuda()

    def arrays(e, ids=None):
        return (conv(e.event_ids if ids is None else ids, np.int32), conv(e.mean, np.float64),
                conv(e.sd, np.float64), conv(e.max_exposure, np.float64))

    with ara.Context(seed=42) as c:
        c.set_option(ara.OPT_SCHEDULE, ara.SCHED_TRIAL)
        y = c.create_yet(w.yet.offsets, w.yet.event_ids, w.yet.timestamps, 2_000_000)
        elts = [c.add_elt(y, *arrays(e)) for e in w.elts]
        t = w.terms
        layer = c.add_layer(elts, t.occ_ret, t.occ_lim, t.agg_ret, t.agg_lim)
        np.testing.assert_array_equal(c.run(y, layer, 0, 500), cr.run(ry, rl, 0, 500))
        dup = w.elts[0].event_ids.copy()
        dup[5] = dup[4]
        with pytest.raises(ara.AraError, match="duplicate"):
            c.add_elt(y, *arrays(w.elts[0], dup))
