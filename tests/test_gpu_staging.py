"""Staging scratch: the temporaries of ELT and layer staging come from one grow-only device buffer
of the context.  An ELT larger than its first size (here 2.5M records over a 4M-event catalogue:
~100 MB of temporaries against the initial 64 MB) grows it; ELTs and layers staged after that
must come out exactly as in a context that never grew it, and the large ELT's own results must
match the FP64 oracle."""

import numpy as np
import pytest

from paper_1310_2274_b300 import synth

pytestmark = pytest.mark.gpu

CAT = 4_000_000
N = 400


def test_scratch_growth_keeps_staging_exact(ara, oracle):
    yet = synth.make_yet(N, 1000, CAT, seed=5)
    big = synth.make_elt(2_500_000, CAT, seed=6)
    small = synth.make_elt(150_000, CAT, seed=7)
    terms = synth.TERMS_PAPER
    args = (terms.occ_ret, terms.occ_lim, terms.agg_ret, terms.agg_lim)
    with ara.Context(seed=42) as a, ara.Context(seed=42) as b:
        ya = a.create_yet(yet.offsets, yet.event_ids, yet.timestamps, CAT)
        yb = b.create_yet(yet.offsets, yet.event_ids, yet.timestamps, CAT)
        # context a: the small ELT first (handle 0), then the large one grows the scratch, then
        # a layer over the small one is staged from the grown scratch
        ea0 = a.add_elt(ya, small.event_ids, small.mean, small.sd, small.max_exposure)
        ea1 = a.add_elt(ya, big.event_ids, big.mean, big.sd, big.max_exposure)
        la_small = a.add_layer([ea0], *args)
        la_big = a.add_layer([ea1], *args)
        # context b: the small ELT alone (handle 0), scratch never grown
        eb0 = b.add_elt(yb, small.event_ids, small.mean, small.sd, small.max_exposure)
        lb_small = b.add_layer([eb0], *args)
        np.testing.assert_array_equal(a.run(ya, la_small, 0, N), b.run(yb, lb_small, 0, N))
        got = a.run(ya, la_big, 0, N)
    want, _ = oracle.run(yet, [big], terms, 42, trials=np.arange(N), elt_handles=[1])
    scale = np.maximum(np.maximum(np.abs(want), terms.agg_ret), 1.0)
    assert np.max(np.abs(got - want) / scale) <= 1e-5


def test_device_resident_yet_checked_on_the_device(ara):
    """A YET whose arrays are in device memory is checked there (offsets by a kernel, timestamps
    where they are, never copied): bad offsets, ids and timestamps are rejected, and a valid one
    runs exactly as the same YET staged from host arrays (the same handles)."""
    import torch

    w = synth.tiny(300)
    y = w.yet
    dev = lambda x: torch.from_numpy(np.ascontiguousarray(x)).cuda()  # noqa: E731
    with ara.Context(seed=42) as ctx:
        h = ctx.create_yet(y.offsets, y.event_ids, y.timestamps, y.catalog_size)
        d = ctx.create_yet(dev(y.offsets), dev(y.event_ids), dev(y.timestamps), y.catalog_size)
        e_h = ctx.add_elt(h, *(getattr(w.elts[0], f) for f in ("event_ids", "mean", "sd",
                                                                "max_exposure")))
        e_d = ctx.add_elt(d, *(getattr(w.elts[0], f) for f in ("event_ids", "mean", "sd",
                                                                "max_exposure")))
        assert (e_h, e_d) == (0, 1)
        t = w.terms
        l_d = ctx.add_layer([e_d], t.occ_ret, t.occ_lim, t.agg_ret, t.agg_lim)
        # the uniforms are keyed by the ELT handle: compare with a context of host arrays in
        # which the same ELT also has handle 1
        got_d = ctx.run(d, l_d, 0, 300)
        with ara.Context(seed=42) as ref:
            rh = ref.create_yet(y.offsets, y.event_ids, y.timestamps, y.catalog_size)
            ref.add_elt(rh, *(getattr(w.elts[0], f) for f in ("event_ids", "mean", "sd",
                                                               "max_exposure")))
            r1 = ref.add_elt(rh, *(getattr(w.elts[0], f) for f in ("event_ids", "mean", "sd",
                                                                    "max_exposure")))
            rl = ref.add_layer([r1], t.occ_ret, t.occ_lim, t.agg_ret, t.agg_lim)
            np.testing.assert_array_equal(got_d, ref.run(rh, rl, 0, 300))
        # rejections, each with the caller's arrays on the device
        bad_off = y.offsets.copy()
        bad_off[7], bad_off[8] = bad_off[8], bad_off[7]  # trial 7 ends before it starts
        with pytest.raises(ara.AraError, match="decrease at trial 7"):
            ctx.create_yet(dev(bad_off), dev(y.event_ids), dev(y.timestamps), y.catalog_size)
        first = y.offsets.copy() + 1
        with pytest.raises(ara.AraError, match=r"trial_offsets\[0\] != 0"):
            ctx.create_yet(dev(first), dev(y.event_ids), dev(y.timestamps), y.catalog_size)
        ids = y.event_ids.copy()
        ids[1234] = y.catalog_size
        with pytest.raises(ara.AraError, match="event id outside"):
            ctx.create_yet(dev(y.offsets), dev(ids), dev(y.timestamps), y.catalog_size)
        ts = y.timestamps.copy()
        ts[int(y.offsets[5]) + 3] = -1.0  # below its predecessor in trial 5
        with pytest.raises(ara.AraError, match="timestamps decrease"):
            ctx.create_yet(dev(y.offsets), dev(y.event_ids), dev(ts), y.catalog_size)
        ts = y.timestamps.copy()
        ts[int(y.offsets[9])] = np.nan
        with pytest.raises(ara.AraError, match="NaN timestamp"):
            ctx.create_yet(dev(y.offsets), dev(y.event_ids), dev(ts), y.catalog_size)


def test_add_elts_stages_like_add_elt_and_is_all_or_nothing(ara):
    """ara_add_elts stages several ELTs with one check: the records, tables and uniforms are those
    of one ara_add_elt per ELT (same handles, same year losses bit for bit, with and without
    correlated SDs); a batch with a rejected ELT adds none and names it."""
    w = synth.tiny(400)
    y = w.yet
    e0 = w.elts[0]
    e1 = synth.make_elt(1_500, y.catalog_size, seed=21)
    e2 = synth.split_sd(synth.make_elt(1_000, y.catalog_size, seed=22), seed=22)
    t = w.terms
    tup = lambda e: (e.event_ids, e.mean, e.sd, e.max_exposure)  # noqa: E731
    for policy in (ara.TABLES_EAGER, ara.TABLES_ON_DEMAND):
        with ara.Context(seed=42) as a, ara.Context(seed=42) as b:
            a.set_option(ara.OPT_TABLES, policy)
            b.set_option(ara.OPT_TABLES, policy)
            ya = a.create_yet(y.offsets, y.event_ids, y.timestamps, y.catalog_size)
            yb = b.create_yet(y.offsets, y.event_ids, y.timestamps, y.catalog_size)
            ha = a.add_elts(ya, [tup(e0), tup(e1), tup(e2) + (e2.sd_corr,)])
            hb = [b.add_elt(yb, *tup(e0)), b.add_elt(yb, *tup(e1)),
                  b.add_elt(yb, *tup(e2), sd_corr=e2.sd_corr)]
            assert ha == hb == [0, 1, 2]
            la = a.add_layer(ha, t.occ_ret, t.occ_lim, t.agg_ret, t.agg_lim)
            lb = b.add_layer(hb, t.occ_ret, t.occ_lim, t.agg_ret, t.agg_lim)
            ga, gb = a.run(ya, la, 0, 400), b.run(yb, lb, 0, 400)
            np.testing.assert_array_equal(ga, gb)
            assert np.count_nonzero(ga) > 100
            assert a.stats()["uncertified"] == b.stats()["uncertified"]
            # a batch whose second ELT repeats an event id: rejected as a whole
            bad = e1.event_ids.copy()
            bad[7] = bad[3]
            with pytest.raises(ara.AraError, match="ELT 1 rejected: duplicate event id"):
                a.add_elts(ya, [tup(e0), (bad, e1.mean, e1.sd, e1.max_exposure), tup(e2)])
            assert a.add_elt(ya, *tup(e0)) == 3  # nothing of the failed batch was added
