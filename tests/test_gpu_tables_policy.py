"""On-demand quantile tables (rent-or-buy): runs over ELTs whose tables were deferred use
Newton's method, bit for bit as the Newton inversion does, until the ELTs' accumulated Newton work
reaches the cost of building their tables; from then on they use the tables, bit for bit as
tables built at staging do.  Servers build deferred tables when created."""

import numpy as np
import pytest

from paper_1310_2274_b300 import synth

pytestmark = pytest.mark.gpu


def workload(n_trials, n_events):
    # a 10,000-event catalogue: a run of n_trials x n_events meets each record
    # n_trials * n_events / 10,000 times on average
    yet = synth.make_yet(n_trials, n_events, 10_000, seed=1)
    elts = [synth.make_elt(2_000, 10_000, seed=s) for s in (2, 3, 4)]
    return yet, elts, synth.TERMS_TINY


def stage(ara, c, yet_h, elts_h, terms):
    yet = c.create_yet(yet_h.offsets, yet_h.event_ids, yet_h.timestamps, yet_h.catalog_size)
    hs = [c.add_elt(yet, e.event_ids, e.mean, e.sd, e.max_exposure) for e in elts_h]
    layer = c.add_layer(hs, terms.occ_ret, terms.occ_lim, terms.agg_ret, terms.agg_lim)
    return yet, hs, layer


def delta(c, f):
    s0 = c.stats()
    out = f()
    s1 = c.stats()
    return out, {k: s1[k] - s0[k] for k in s0}


def test_rent_then_buy(ara, oracle):
    yet_h, elts_h, terms = workload(20_000, 100)  # 200 expected hits per record per run
    n = yet_h.n_trials
    with ara.Context(seed=42) as eager:
        y_e, hs_e, l_e = stage(ara, eager, yet_h, elts_h, terms)
        ref_table = eager.run(y_e, l_e, 0, n)
        eager.set_option(ara.OPT_INVERSION, ara.INV_NEWTON)
        ref_newton = eager.run(y_e, l_e, 0, n)
    with ara.Context(seed=42) as c:
        c.set_option(ara.OPT_TABLES, ara.TABLES_ON_DEMAND)
        y, hs, layer = stage(ara, c, yet_h, elts_h, terms)
        buy_run = int(np.ceil(ara.TABLE_BUY_HITS / 200.0))  # the first k with 200 k >= threshold
        for r in range(1, buy_run + 2):
            g, d = delta(c, lambda: c.run(y, layer, 0, n))
            if r < buy_run:
                assert d["table_evals"] == 0 and d["inversions"] == d["hits"], r
                np.testing.assert_array_equal(g, ref_newton)
            else:
                assert d["table_evals"] > 0.99 * d["hits"], r
                np.testing.assert_array_equal(g, ref_table)
    o, _ = oracle.run(yet_h, elts_h, terms, 42, elt_handles=[0, 1, 2])
    scale = np.maximum(np.maximum(np.abs(o), terms.agg_ret), 1.0)
    assert np.max(np.abs(ref_newton - o) / scale) <= 1e-5


def test_large_run_buys_at_once_and_partial_ranges_rent(ara):
    yet_h, elts_h, terms = workload(20_000, 1200)  # 2,400 expected hits per record
    with ara.Context(seed=42) as c:
        c.set_option(ara.OPT_TABLES, ara.TABLES_ON_DEMAND)
        y, hs, layer = stage(ara, c, yet_h, elts_h, terms)
        assert 240 < ara.TABLE_BUY_HITS <= 2_400
        # a tenth of the trials: 240 per record, rented
        _, d = delta(c, lambda: c.run(y, layer, 0, 2_000))
        assert d["table_evals"] == 0
        # the rest: 240 + 2,160 reaches the threshold, bought before the run
        _, d = delta(c, lambda: c.run(y, layer, 2_000, 18_000))
        assert d["table_evals"] > 0.99 * d["hits"]
        # a new layer over the same ELTs reuses their tables at once
        l2 = c.add_layer(hs[:2], 0.0, 1e7, 0.0, 1e9)
        _, d = delta(c, lambda: c.run(y, l2, 0, 100))
        assert d["table_evals"] > 0.99 * d["hits"]


def test_server_builds_deferred_tables(ara):
    yet_h, elts_h, terms = workload(5_000, 100)
    req = dict(occ_ret=terms.occ_ret, occ_lim=terms.occ_lim, agg_ret=terms.agg_ret,
               agg_lim=terms.agg_lim, t0=0, n_trials=5_000, rps=(10.0, 100.0))
    with ara.Context(seed=42) as c:
        c.set_option(ara.OPT_TABLES, ara.TABLES_ON_DEMAND)
        y, hs, layer = stage(ara, c, yet_h, elts_h, terms)
        with ara.Server(c, y) as s:
            tk = s.submit(elts=hs, **req)
            assert s.wait(tk, 60.0) == 0
            got = s.result(tk)["ylt"]
        # the ELTs now have tables: a run alone uses them, and equals the served result
        _, d = delta(c, lambda: c.run(y, layer, 0, 5_000))
        assert d["table_evals"] > 0.99 * d["hits"]
        np.testing.assert_array_equal(c.run(y, layer, 0, 5_000), got)


def test_portfolio_mixes_tables_and_newton(ara):
    # one layer over ELTs whose tables exist, one over deferred ELTs: the portfolio groups them
    # by inversion and each row equals its layer run alone
    yet_h, elts_h, terms = workload(3_000, 100)
    with ara.Context(seed=42) as c:
        y = c.create_yet(yet_h.offsets, yet_h.event_ids, yet_h.timestamps, yet_h.catalog_size)
        eager = [c.add_elt(y, e.event_ids, e.mean, e.sd, e.max_exposure) for e in elts_h[:2]]
        c.set_option(ara.OPT_TABLES, ara.TABLES_ON_DEMAND)
        lazy = c.add_elt(y, elts_h[2].event_ids, elts_h[2].mean, elts_h[2].sd,
                         elts_h[2].max_exposure)
        l_table = c.add_layer(eager, terms.occ_ret, terms.occ_lim, terms.agg_ret, terms.agg_lim)
        l_newton = c.add_layer([eager[0], lazy], terms.occ_ret, terms.occ_lim, terms.agg_ret,
                               terms.agg_lim)
        m, d = delta(c, lambda: c.run_portfolio(y, [l_table, l_newton], 0, 3_000))
        assert d["table_evals"] > 0 and d["inversions"] > 0
        np.testing.assert_array_equal(m[0], c.run(y, l_table, 0, 3_000))
        np.testing.assert_array_equal(m[1], c.run(y, l_newton, 0, 3_000))


def test_option_values_are_checked(ara):
    with ara.Context(seed=42) as c:
        for opt, bad in [(ara.OPT_TABLES, 2), (ara.OPT_TABLES, -1), (ara.OPT_STREAM_CHUNK, 1000),
                         (ara.OPT_STREAM_CHUNK, (1 << 30) + 1)]:
            with pytest.raises(ara.AraError) as e:
                c.set_option(opt, bad)
            assert e.value.status == 1
