"""Portfolio runs (Algorithm 1's loops over programs and layers) on the device: every layer's YLT
from one call equals ara_run of that layer alone bit for bit, whatever the mix of schedules and
lookup-entry widths in the call, and matches the FP64 oracle's portfolio run."""

import numpy as np
import pytest

from paper_1310_2274_b300 import synth

pytestmark = pytest.mark.gpu

N = 2000
TOL = 1e-5


@pytest.fixture(scope="module")
def staged(ara):
    # 40 paper-scale ELTs over the 2,000,000-event catalogue; layers of 3..40 ELTs (both lookup
    # widths: up to 32 ELTs one mask word, above two)
    yet_h = synth.make_yet(N, 1000, 2_000_000, seed=1)
    elts_h = synth.paper_elts(40)
    c = ara.Context(seed=42)
    yet = c.create_yet(yet_h.offsets, yet_h.event_ids, yet_h.timestamps, 2_000_000)
    hs = [c.add_elt(yet, e.event_ids, e.mean, e.sd, e.max_exposure) for e in elts_h]
    assert hs == list(range(40))
    yield c, yet_h, elts_h, yet
    c.close()


def portfolio(seed=0):
    """Three programs of layers with 3..40 ELTs and terms scaled to their size."""
    rng = np.random.default_rng(seed)
    pf = []
    for _ in range(3):
        prog = []
        for _ in range(int(rng.integers(2, 5))):
            k = int(rng.choice([3, 5, 16, 30, 33, 40]))
            idx = tuple(int(i) for i in rng.choice(40, size=k, replace=False))
            t = synth.Terms(float(rng.choice([0.0, 1e5])), float(rng.choice([1e7, 5e7])),
                            float(rng.uniform(0.3, 0.9)) * 1.7e7 * k, 2.5e8 * k / 16)
            prog.append((idx, t))
        pf.append(prog)
    return pf


def build_layers(c, pf):
    return [c.add_layer(list(idx), t.occ_ret, t.occ_lim, t.agg_ret, t.agg_lim)
            for prog in pf for idx, t in prog]


@pytest.mark.parametrize("schedule", ["band", "trial"])
def test_portfolio_equals_layers_run_alone(ara, staged, schedule):
    c, yet_h, elts_h, yet = staged
    pf = portfolio()
    layers = build_layers(c, pf)
    c.set_option(ara.OPT_SCHEDULE, ara.SCHED_BAND if schedule == "band" else ara.SCHED_TRIAL)
    try:
        c.run_portfolio(yet, layers, 0, 1)  # makes the layers' band-major YET copies first
        s0 = c.stats()
        m = c.run_portfolio(yet, layers, 0, N)
        s1 = c.stats()
        alone = [c.run(yet, l, 0, N) for l in layers]
        # a sub-range, through device memory
        import torch
        part = torch.zeros((len(layers), 700), dtype=torch.float64, device="cuda")
        c.run_portfolio(yet, layers[::-1], 611, 700, out=part)
    finally:
        c.set_option(ara.OPT_SCHEDULE, ara.SCHED_BAND)
        for l in layers:
            c.free_layer(l)
    for i, y in enumerate(alone):
        np.testing.assert_array_equal(m[i], y)
    np.testing.assert_array_equal(part.cpu().numpy(), m[::-1, 611:1311])
    # at most one batched launch per (schedule, entry width) group, plus band finalisation
    assert s1["launches"] - s0["launches"] <= 6
    assert np.all(np.count_nonzero(m, axis=1) > N // 4)


def test_portfolio_matches_oracle(ara, oracle, staged):
    c, yet_h, elts_h, yet = staged
    pf = portfolio(seed=1)
    layers = build_layers(c, pf)
    try:
        m = c.run_portfolio(yet, layers, 0, N)
    finally:
        for l in layers:
            c.free_layer(l)
    o = oracle.run_portfolio(yet_h, elts_h, pf, 42)
    terms = [t for prog in pf for _, t in prog]
    for i, t in enumerate(terms):
        scale = np.maximum(np.maximum(np.abs(o[i]), t.agg_ret), 1.0)
        assert np.max(np.abs(m[i] - o[i]) / scale) <= TOL, i


def test_portfolio_arguments(ara, staged):
    c, yet_h, elts_h, yet = staged
    layer = c.add_layer([0, 1, 2], 0.0, 1e7, 0.0, 1e9)
    try:
        assert c.run_portfolio(yet, [], 0, N).shape == (0, N)
        same = c.run_portfolio(yet, [layer, layer], 0, 50)
        np.testing.assert_array_equal(same[0], same[1])
        with pytest.raises(ara.AraError):
            c.run_portfolio(yet, [layer, 999], 0, 10)
        with pytest.raises(ara.AraError):
            c.run_portfolio(yet, [layer], N - 5, 10)
    finally:
        c.free_layer(layer)
