"""Pins for the oracle's Algorithm 1 loop: lookup, terms, accumulation, YLT population.

Pinned by the hand-worked term sequences in tests/golden/terms_sequences.txt (paper §2.3), by the
sigma = 0 reduction to primary uncertainty (paper §1: mean losses only; integer means make the
year loss exact), and by brute-force linear-scan lookups.
"""

import os

import numpy as np
import pytest

from paper_1310_2274_b300 import synth

GOLDEN = os.path.join(os.path.dirname(__file__), "golden", "terms_sequences.txt")


def load_term_cases():
    cases = []
    for line in open(GOLDEN):
        line = line.strip()
        if not line or line.startswith("#"):
            continue
        name, terms, losses, occ, s, y = [f.strip() for f in line.split("|")]
        t = [float(v) for v in terms.split()]
        cases.append((name, synth.Terms(*t), [float(v) for v in losses.split()],
                      [float(v) for v in occ.split()], float(s), float(y)))
    return cases


def one_trial_layer(losses):
    """One trial whose k-th event has event id k and, in a single ELT, mean loss losses[k]."""
    n = len(losses)
    yet = synth.Yet(np.array([0, n], np.int64), np.arange(n, dtype=np.int32),
                    np.arange(n, dtype=np.float32), max(n, 1))
    elt = synth.Elt(np.arange(n, dtype=np.int32), np.array(losses, np.float64),
                    np.zeros(n), np.array(losses, np.float64) * 2 + 1)
    return yet, elt


@pytest.mark.parametrize("case", load_term_cases(), ids=lambda c: c[0])
def test_golden_term_sequences(oracle, case):
    name, terms, losses, occ, s, y = case
    for l, o in zip(losses, occ):
        assert oracle.occ_terms(l, terms.occ_ret, terms.occ_lim) == o
    assert oracle.agg_terms(s, terms.agg_ret, terms.agg_lim) == y
    yet, elt = one_trial_layer(losses)
    ylt, nc = oracle.run(yet, [elt], terms, 42)
    assert nc == 0 and ylt[0] == y


def test_sigma_zero_reduction_brute_force(oracle):
    # Primary uncertainty only: every sd = 0 and integer means, so the year loss
    # f_agg(sum_k f_occ(sum_j mean_j(e_k))) is exact in binary64.
    w = synth.tiny(200)
    rng = np.random.default_rng(5)
    elts = []
    for j in range(3):
        e = synth.make_elt(1500 + 300 * j, w.yet.catalog_size, seed=20 + j)
        e.mean = np.floor(e.mean)
        e.sd = np.zeros_like(e.mean)
        elts.append(e)
    terms = synth.Terms(5e4, 3e6, 2e5, 4e7)
    ylt, _ = oracle.run(w.yet, elts, terms, 42)
    maps = [dict(zip(e.event_ids.tolist(), e.mean.tolist())) for e in elts]
    for i in range(w.yet.n_trials):
        s = 0.0
        for q in range(w.yet.offsets[i], w.yet.offsets[i + 1]):
            e = int(w.yet.event_ids[q])
            l = sum(m.get(e, 0.0) for m in maps)
            s += min(max(l - terms.occ_ret, 0.0), terms.occ_lim)
        assert ylt[i] == min(max(s - terms.agg_ret, 0.0), terms.agg_lim)
    assert rng is not None


def test_lookup_and_uniform_trace_brute_force(oracle):
    w = synth.tiny(60)
    elts = [w.elts[0], synth.make_elt(800, w.yet.catalog_size, seed=31)]
    handles = [5, 2]
    hits, ylt_t = oracle.trace(w.yet, elts, w.terms, 42, np.arange(60), elt_handles=handles)
    ylt_r, _ = oracle.run(w.yet, elts, w.terms, 42, trials=np.arange(60), elt_handles=handles)
    assert np.array_equal(ylt_t, ylt_r)
    # brute force: linear scan of each ELT for each occurrence, in loop order
    expect = []
    for i in range(60):
        for q in range(w.yet.offsets[i], w.yet.offsets[i + 1]):
            e = w.yet.event_ids[q]
            for j, elt in enumerate(elts):
                r = np.nonzero(elt.event_ids == e)[0]
                if r.size:
                    expect.append((i, q - w.yet.offsets[i], j, int(r[0])))
    got = list(zip(hits["trial"].tolist(), hits["k"].tolist(), hits["j"].tolist(),
                   hits["rec"].tolist()))
    assert got == expect
    for h in range(0, len(got), 7):
        i, k, j, r = got[h]
        u = oracle.su_uniform(42, i, k, handles[j])
        assert hits["u"][h] == u
        e = elts[j]
        loss, _ = oracle.su_loss(e.mean[r], e.sd[r], e.max_exposure[r], u)
        assert hits["loss"][h] == loss
    # about 0.2 + 0.08 hits per occurrence
    assert 0.2 < len(got) / (60 * 100) < 0.4


def test_run_is_deterministic_across_threads_and_subsets(oracle):
    w = synth.tiny(300)
    full1, _ = oracle.run(w.yet, w.elts, w.terms, 42, threads=1)
    full4, _ = oracle.run(w.yet, w.elts, w.terms, 42, threads=4)
    assert np.array_equal(full1, full4)
    pick = synth.subset_trials(300, 37, seed=9)
    sub, _ = oracle.run(w.yet, w.elts, w.terms, 42, trials=pick)
    assert np.array_equal(sub, full1[pick])
    # another seed changes the year losses
    other, _ = oracle.run(w.yet, w.elts, w.terms, 43, threads=4)
    assert not np.array_equal(other, full1)


def test_ragged_and_empty_trials(oracle):
    yet = synth.make_ragged_yet(50, 0, 40, 500, seed=3)
    elt = synth.make_elt(200, 500, seed=4)
    ylt, _ = oracle.run(yet, [elt], synth.TERMS_TINY, 42)
    empty = np.nonzero(np.diff(yet.offsets) == 0)[0]
    assert empty.size > 0 and np.all(ylt[empty] == 0.0)
    assert np.all(ylt >= 0.0) and np.all(ylt <= synth.TERMS_TINY.agg_lim)


def test_duplicate_ids_rejected(oracle):
    yet = synth.make_yet(2, 5, 100, seed=1)
    elt = synth.Elt(np.array([3, 3], np.int32), np.ones(2), np.zeros(2), np.full(2, 4.0))
    with pytest.raises(ValueError):
        oracle.run(yet, [elt], synth.TERMS_TINY, 42)


def test_oep_is_the_largest_occurrence_loss():
    # event-level output: the year's largest occurrence loss, checked against a hand-rolled loop
    # over the oracle's own per-hit trace (occurrence sums, then terms, then the maximum)
    import oracle
    from paper_1310_2274_b300 import synth

    w = synth.tiny(60)
    ylt, oep, nc = oracle.run(w.yet, w.elts, w.terms, 42, with_oep=True)
    assert nc == 0
    hits, y2 = oracle.trace(w.yet, w.elts, w.terms, 42, np.arange(60))
    np.testing.assert_array_equal(ylt, y2)
    for i in range(60):
        sel = hits["trial"] == i
        ks = np.unique(hits["k"][sel])
        o = [min(max(hits["loss"][sel & (hits["k"] == k)].sum() - w.terms.occ_ret, 0.0),
                 w.terms.occ_lim) for k in ks]
        assert oep[i] == (max(o) if o else 0.0)
    # the OEP year never exceeds the occurrence-summed year before aggregate terms
    assert np.all(oep >= 0) and np.all(oep <= w.terms.occ_lim)


def test_oep_against_the_aggregate_year_in_special_cases():
    # with identity aggregate terms the largest occurrence loss never exceeds the year's sum, and a
    # trial of one event has OEP = AEP; the OEP does not move with the aggregate terms
    import oracle
    from paper_1310_2274_b300 import synth

    w = synth.tiny(200)
    rng = np.random.default_rng(4)
    lens = rng.choice([0, 1, 1, 2, 7, 40], size=300)
    offsets = np.zeros(301, dtype=np.int64)
    np.cumsum(lens, out=offsets[1:])
    ids = rng.integers(0, w.yet.catalog_size, size=int(offsets[-1]), dtype=np.int32)
    yet = synth.Yet(offsets, ids, np.zeros(ids.shape[0], np.float32), w.yet.catalog_size)
    ident = synth.Terms(w.terms.occ_ret, w.terms.occ_lim, 0.0, np.inf)
    ylt, oep, _ = oracle.run(yet, w.elts, ident, 42, with_oep=True)
    assert np.all(oep <= ylt) and np.count_nonzero(oep) > 100
    np.testing.assert_array_equal(oep[lens == 1], ylt[lens == 1])
    assert np.all(oep[lens == 0] == 0.0)
    assert np.any(oep[lens > 2] < ylt[lens > 2])
    _, oep2, _ = oracle.run(yet, w.elts, w.terms, 42, with_oep=True)
    np.testing.assert_array_equal(oep, oep2)
