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
