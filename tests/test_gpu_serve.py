"""Continuous-batching service: a request's results do not depend on what else shares its launches.

Each request's YLT from the server (wide lookup entries, batched launches of several requests,
sliced trial ranges) must equal bit for bit the YLT of ara_run on the same layer and trials run
alone, and its PML/TVaR must equal ara_risk_measures on that YLT.  The admission budget, the
queue bound, argument checks and the latency statistics are checked too.
"""

import threading
import time

import numpy as np
import pytest

from paper_1310_2274_b300 import synth

pytestmark = pytest.mark.gpu

N_TRIALS = 40_000


@pytest.fixture(scope="module")
def staged(ara):
    """A 40,000-trial x 1,000-event YET over the 2,000,000-event catalogue and 8 paper ELTs."""
    c = ara.Context(seed=42)
    yet_h = synth.make_yet(N_TRIALS, 1000, 2_000_000, seed=1)
    elts = synth.paper_elts(8)
    yet = c.create_yet(yet_h.offsets, yet_h.event_ids, yet_h.timestamps, yet_h.catalog_size)
    hs = [c.add_elt(yet, e.event_ids, e.mean, e.sd, e.max_exposure) for e in elts]
    yield c, yet, hs
    c.close()


def request_mix(hs, n, seed=0):
    """n requests: random ELT subsets (random summation order), terms and trial ranges."""
    rng = np.random.default_rng(seed)
    out = []
    for q in range(n):
        k = int(rng.integers(1, len(hs) + 1))
        elts = [hs[i] for i in rng.permutation(len(hs))[:k]]
        occ_ret = float(rng.choice([0.0, 1e5, 1e6]))
        occ_lim = float(rng.choice([1e7, 5e7, 1e12]))
        agg_ret = float(rng.uniform(0, 1.5e8)) * k / len(hs)
        agg_lim = float(rng.choice([2.5e8, 1e9, 1e15]))
        t0 = int(rng.integers(0, N_TRIALS // 2))
        nt = int(rng.integers(1, N_TRIALS - t0 + 1)) if q % 3 else N_TRIALS - t0
        out.append(dict(elts=elts, occ_ret=occ_ret, occ_lim=occ_lim, agg_ret=agg_ret,
                        agg_lim=agg_lim, t0=t0, n_trials=nt, rps=(10.0, 100.0, 250.0)))
    return out


def settled_stats(s, timeout=10.0):
    """Server statistics once the builder thread has freed every finished request's memory."""
    t_end = time.time() + timeout
    st = s.stats()
    while st["hbm_used"] != 0 and time.time() < t_end:
        time.sleep(0.01)
        st = s.stats()
    return st


def alone(c, yet, r):
    layer = c.add_layer(r["elts"], r["occ_ret"], r["occ_lim"], r["agg_ret"], r["agg_lim"])
    y = c.run(yet, layer, r["t0"], r["n_trials"])
    p, t = c.risk_measures(y, r["rps"])
    c.free_layer(layer)
    return y, p, t


def test_batched_requests_equal_requests_run_alone(ara, staged):
    c, yet, hs = staged
    mix = request_mix(hs, 12)
    ref = [alone(c, yet, r) for r in mix]
    # small, ragged slices: each request needs many launches, so requests admitted one after
    # another (the builder thread admits while launches run) share launches
    with ara.Server(c, yet, max_inflight=6, slice_trials=333, max_batch_trials=20_000) as s:
        tickets = [s.submit(**r) for r in mix]
        for tk in tickets:
            assert s.wait(tk, 120.0) == 0
        st = settled_stats(s)
        for tk, r, (y, p, t) in zip(tickets, mix, ref):
            res = s.result(tk)
            assert res["state"] == ara.REQ_DONE
            np.testing.assert_array_equal(res["ylt"], y)
            np.testing.assert_array_equal(res["pml"][:3], p)
            np.testing.assert_array_equal(res["tvar"][:3], t)
            assert res["submit_s"] <= res["admit_s"] <= res["done_s"]
            s.release(tk)
    assert st["completed"] == len(mix) and st["failed"] == 0
    assert st["mean_items_per_launch"] > 1.0  # some launches really were shared
    assert st["hbm_used"] == 0
    assert 0 < st["latency_p50_s"] <= st["latency_p99_s"] <= st["latency_max_s"]


def test_admission_budget_serialises_but_completes(ara, staged):
    c, yet, hs = staged
    mix = request_mix(hs, 5, seed=1)
    ref = [alone(c, yet, r) for r in mix]
    # room for about one request at a time: 16 B x 2M catalogue entries = 32 MB per layer
    with ara.Server(c, yet, max_inflight=8, slice_trials=8192, hbm_budget=48 << 20) as s:
        tickets = [s.submit(**r) for r in mix]
        for tk in tickets:
            assert s.wait(tk, 120.0) == 0
        res = [s.result(tk) for tk in tickets]
        st = settled_stats(s)
    for (y, _, _), r in zip(ref, res):
        np.testing.assert_array_equal(r["ylt"], y)
    # admitted one after another, in arrival order
    admits = [r["admit_s"] for r in res]
    dones = [r["done_s"] for r in res]
    assert admits == sorted(admits)
    for i in range(1, len(res)):
        assert admits[i] >= dones[i - 1] - 1e-6
    assert st["completed"] == 5 and st["hbm_used"] == 0


def test_rejections(ara, staged):
    c, yet, hs = staged
    ok = dict(elts=hs[:2], occ_ret=0.0, occ_lim=1e9, agg_ret=0.0, agg_lim=1e12, t0=0,
              n_trials=10, rps=(10.0,))
    with ara.Server(c, yet, max_queue=0) as s:
        with pytest.raises(ara.AraError) as e:
            s.submit(**ok)
        assert e.value.status == 6  # queue bound
    with ara.Server(c, yet) as s:
        for bad, status in [(dict(ok, t0=N_TRIALS - 5), 1), (dict(ok, n_trials=0), 1),
                            (dict(ok, elts=[hs[0], 999]), 2), (dict(ok, rps=(1.0,)), 1),
                            (dict(ok, elts=[]), 1)]:
            with pytest.raises(ara.AraError) as e:
                s.submit(**bad)
            assert e.value.status == status
        # a duplicated ELT is caught when the layer is built: the request fails, the server goes on
        tk = s.submit(**dict(ok, elts=[hs[0], hs[0]]))
        assert s.wait(tk, 60.0) == 1
        assert s.result(tk)["state"] == ara.REQ_FAILED
        tk = s.submit(**ok)
        assert s.wait(tk, 60.0) == 0
        with pytest.raises(ara.AraError):
            s.release(10_000)
    # the context is usable again once the server is gone
    y, _, _ = alone(c, yet, ok)
    assert y.shape == (10,)


def test_poisson_arrivals_latency(ara, staged):
    c, yet, hs = staged
    mix = request_mix(hs, 40, seed=2)
    ref = {i: alone(c, yet, r)[0] for i, r in enumerate(mix) if i % 8 == 0}
    rng = np.random.default_rng(3)
    gaps = rng.exponential(0.004, size=len(mix))  # about 250 requests/s offered
    with ara.Server(c, yet, max_inflight=16, slice_trials=8192) as s:
        tickets = []

        def producer():
            for r, g in zip(mix, gaps):
                time.sleep(g)
                tickets.append(s.submit(**r))

        th = threading.Thread(target=producer)
        th.start()
        th.join()
        for tk in tickets:
            assert s.wait(tk, 120.0) == 0
        st = s.stats()
        for i, y in ref.items():
            np.testing.assert_array_equal(s.result(tickets[i])["ylt"], y)
    print(f"poisson serving: p50 {st['latency_p50_s'] * 1e3:.2f} ms, "
          f"p99 {st['latency_p99_s'] * 1e3:.2f} ms, {st['requests_per_s']:.1f} req/s, "
          f"{st['mean_items_per_launch']:.2f} requests per launch")
    assert st["completed"] == len(mix)


@pytest.mark.parametrize("mode", ["newton", "kahan"])
def test_trial_major_serving_equals_requests_run_alone(ara, staged, mode):
    # the batched trial-major kernel: Newton inversion, or Kahan FP32 year sums (both keep the
    # trial-major schedule); results again identical to the same requests run alone
    c, yet, hs = staged
    mix = [dict(r, n_trials=min(r["n_trials"], 3000)) for r in request_mix(hs, 4, seed=5)]
    inversion = ara.INV_NEWTON if mode == "newton" else ara.INV_TABLE
    c.set_option(ara.OPT_INVERSION, inversion)
    if mode == "kahan":
        c.set_option(ara.OPT_PRECISION, ara.ACC_KAHAN32)
    try:
        ref = [alone(c, yet, r) for r in mix]
        with ara.Server(c, yet, max_inflight=4, slice_trials=700, inversion=inversion) as s:
            tickets = [s.submit(**r) for r in mix]
            for tk in tickets:
                assert s.wait(tk, 120.0) == 0
            for tk, (y, p, t) in zip(tickets, ref):
                res = s.result(tk)
                np.testing.assert_array_equal(res["ylt"], y)
                np.testing.assert_array_equal(res["pml"][:3], p)
    finally:
        c.set_option(ara.OPT_INVERSION, ara.INV_TABLE)
        c.set_option(ara.OPT_PRECISION, ara.ACC_FP64)


def test_deep_slices_launch_alone_and_match(ara, staged):
    # slices of up to 40,000 trials have grids many waves deep: they run as their own launches
    # beside the batched small ones; every request still equals its run alone
    c, yet, hs = staged
    mix = request_mix(hs, 6, seed=7)
    mix[0] = dict(mix[0], t0=0, n_trials=N_TRIALS)
    ref = [alone(c, yet, r) for r in mix]
    s0 = c.stats()
    with ara.Server(c, yet, max_inflight=6, slice_trials=N_TRIALS) as s:
        tickets = [s.submit(**r) for r in mix]
        for tk in tickets:
            assert s.wait(tk, 120.0) == 0
        for tk, (y, p, t) in zip(tickets, ref):
            res = s.result(tk)
            np.testing.assert_array_equal(res["ylt"], y)
            np.testing.assert_array_equal(res["pml"][:3], p)
            np.testing.assert_array_equal(res["tvar"][:3], t)
    assert c.stats()["launches"] > s0["launches"]
