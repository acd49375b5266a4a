"""The learned surrogate of InvCDF_beta: tensor-core forward and backward kernels against the FP64
reference network (oracle/mlp.py) and, element by element, against the same network with the
kernels' rounding points (tests/mlp_emulation.py), training on the GPU on 5e7 exact tuples,
certification, and its use inside the run with exact fallback, measured against the FP64 oracle
and against the method without it.
"""

import time

import numpy as np
import pytest

import mlp_emulation as emu
from oracle import mlp as ref
from paper_1310_2274_b300 import synth

pytestmark = pytest.mark.gpu


def rel_l2(a, b):
    return float(np.linalg.norm(a - b) / max(np.linalg.norm(b), 1e-30))


@pytest.fixture(scope="module")
def batch():
    rng = np.random.default_rng(21)
    n = 512
    z = rng.uniform(-1, 1, size=(n, 3))
    x = rng.uniform(0.02, 0.98, size=n)
    t = np.clip(np.log(x / (1 - x)), -30, 30) / ref.OUT_SCALE
    return z, x, t


def test_forward_matches_reference_network(ara, batch):
    z, _, _ = batch
    p = emu.scaled_params(7)
    with ara.Context() as c:
        y = c.mlp_eval(z, params=p).astype(np.float64)
    # element by element against the kernels' arithmetic (BF16 rounding points), within the
    # bound the hardware tanh's error can reach
    want, bound = emu.bounds(p, z)
    assert np.all(np.abs(y - want) <= bound), np.max(np.abs(y - want) / bound)
    assert np.abs(want).max() > 1.0  # outputs of a trained network's size
    # and close to the binary64 network throughout
    yr, _ = ref.forward(p, z)
    assert rel_l2(y, yr) <= 2e-2


def test_gradient_matches_reference_network(ara, batch):
    z, x, t = batch
    p = emu.scaled_params(7)
    with ara.Context() as c:
        loss, g = c.mlp_grad(p, z, x, t)
    (_, want_loss, want), bound = emu.bounds(p, z, x, t)
    assert abs(loss - want_loss) <= 1e-4 * abs(want_loss)
    g = g.astype(np.float64)
    bad = np.abs(g - want) > bound
    names = ["W1", "b1", "W2", "b2", "W3", "b3", "W4", "b4"]
    for name, gb, wb, bb in zip(names, ref.unpack(g), ref.unpack(want), ref.unpack(bound)):
        assert np.all(np.abs(gb - wb) <= bb), (name, float(np.max(np.abs(gb - wb) / bb)))
    assert not bad.any()
    # and near the binary64 network's gradient, parameter block by block: the BF16 rounding of
    # the layer gradients before their sums over the batch (which cancel) moves a block by up to
    # ~8% at this weight scale, as the emulation above, rounding at the same points, shows
    _, gr = ref.loss_grad(p, z, x, t)
    for name, a, b in zip(names, ref.unpack(g), ref.unpack(gr)):
        assert rel_l2(a.reshape(-1), b.reshape(-1)) <= 0.15, name


@pytest.fixture(scope="module")
def trained(ara):
    c = ara.Context(seed=42)
    rep = c.train_surrogate(n_samples=50_000_000, steps=30_000, batch=8192, lr=3e-3,
                            lr_final=3e-5, eps=5e-4, cert_samples=16, seed=3)
    yield c, rep
    c.close()


def test_training_reduces_loss_and_certifies(trained):
    c, rep = trained
    assert rep["bad_targets"] == 0
    assert rep["loss_last"] < 0.1 * rep["loss_first"]
    assert 0.0 < rep["cells_accepted"] <= 1.0
    assert rep["err_median"] < 2e-2
    print("surrogate training:", rep)


def test_save_load_roundtrip(ara, trained, batch):
    c, _ = trained
    blob = c.save_surrogate()
    z, _, _ = batch
    y0 = c.mlp_eval(z)
    with ara.Context() as c2:
        c2.load_surrogate(blob)
        np.testing.assert_array_equal(c2.mlp_eval(z), y0)
        with pytest.raises(ara.AraError):
            c2.load_surrogate(blob[:100])
        bad = bytearray(blob)
        bad[0] ^= 0xFF
        with pytest.raises(ara.AraError):
            c2.load_surrogate(bytes(bad))


def test_surrogate_run_against_oracle_and_gain(ara, oracle, trained):
    c, _ = trained
    w = synth.tiny()
    yet, elts, layer = c.stage_workload(w)
    o, _ = oracle.run(w.yet, w.elts, w.terms, 42, elt_handles=elts)
    op, ot = oracle.risk(o, w.rps)
    c.set_option(ara.OPT_INVERSION, ara.INV_NEWTON)
    exact = c.run(yet, layer, 0, w.yet.n_trials)
    s0 = c.stats()
    c.set_option(ara.OPT_SURROGATE, 1)
    try:
        g = c.run(yet, layer, 0, w.yet.n_trials)
        s1 = c.stats()
    finally:
        c.set_option(ara.OPT_SURROGATE, 0)
        c.set_option(ara.OPT_INVERSION, ara.INV_TABLE)
    net = s1["surrogate_evals"] - s0["surrogate_evals"]
    fallback = s1["inversions"] - s0["inversions"]
    hits = s1["hits"] - s0["hits"]
    assert net > 0 and net + fallback == hits
    gp, gt = c.risk_measures(g, w.rps)
    # the bar for the learned form: PML / TVaR within 1e-3 of the FP64 oracle
    assert np.max(np.abs(gp - op) / op) <= 1e-3
    assert np.max(np.abs(gt - ot) / ot) <= 1e-3
    # year losses stay close to the exact form, hit by hit the network is certified to eps
    scale = np.maximum(np.abs(exact), w.terms.agg_ret)
    assert np.max(np.abs(g - exact) / scale) <= 2e-2
    print(f"surrogate on {w.name}: {net} network evaluations, {fallback} Newton fallbacks "
          f"({fallback / hits:.1%})")


def test_served_losses_within_eps_of_mean_loss(ara, oracle, trained):
    """A hit is served by the network only where its cell's certified error in x is at most
    eps * mu_beta (mu_beta = mean / max exposure of the hit's record), so each served loss is
    within eps of the record's mean loss and a year's sum within eps of its expected value.  The
    cell error is the largest over the cell's sampled points, not a proof: per year the summed
    loss errors must stay within 2 eps of the year's summed mean losses, hit by hit against the
    FP64 oracle's quantiles."""
    c, _ = trained
    w = synth.tiny()
    yet, elts, layer = c.stage_workload(w)
    eps = 5e-4
    c.set_surrogate_eps(eps)
    c.set_option(ara.OPT_INVERSION, ara.INV_NEWTON)
    c.set_option(ara.OPT_SURROGATE, 1)
    try:
        s0 = c.stats()
        gh, _ = c.trace(yet, layer, 0, w.yet.n_trials)
        s1 = c.stats()
    finally:
        c.set_option(ara.OPT_SURROGATE, 0)
        c.set_option(ara.OPT_INVERSION, ara.INV_TABLE)
    oh, _ = oracle.trace(w.yet, w.elts, w.terms, 42, np.arange(w.yet.n_trials), elt_handles=elts)
    np.testing.assert_array_equal(gh["trial"], oh["trial"])
    np.testing.assert_array_equal(gh["rec"], oh["rec"])
    e = w.elts[0]
    rec = oh["rec"]
    mean, mx = e.mean[rec], e.max_exposure[rec]
    err = np.abs(gh["x"].astype(np.float64) - oh["x"]) * mx  # loss error of every hit
    served = err > 1e-5 * mx  # the exact fallback is within 1e-5 in x
    assert s1["surrogate_evals"] - s0["surrogate_evals"] > 0 and served.any()
    per_hit = err / (eps * mean)
    yr_err = np.bincount(oh["trial"], weights=err, minlength=w.yet.n_trials)
    yr_mean = np.bincount(oh["trial"], weights=mean, minlength=w.yet.n_trials)
    has = yr_mean > 0
    yr = yr_err[has] / (eps * yr_mean[has])
    print(f"served {served.mean():.1%} of hits; loss error / (eps x mean): per hit max "
          f"{per_hit.max():.3f}, p99 {np.quantile(per_hit[served], 0.99):.3f}; per year max "
          f"{yr.max():.3f}")
    assert yr.max() <= 2.0


def test_surrogate_cost_against_newton_on_paper_sample(ara, trained):
    """What the network gains over the method without it, on 20,000 trials of the paper-scale
    layer: it replaces the inversions of the hits it serves (a certified share of them, the rest
    falling back to Newton-Halley), at PML within 1e-3 of the exact form; and what it costs.  The
    run cannot be faster than the bookkeeping every form pays (the same layer with every SD zero)
    plus its fallbacks' share of the Newton-Halley inversion time, which is the bound that keeps
    this network (most hits fall back on this law) slower than the plain form."""
    c, _ = trained
    w = synth.paper(n_trials=20_000)
    yet, elts, layer = c.stage_workload(w)
    z_elts = [c.add_elt(yet, e.event_ids, e.mean, np.zeros(e.n), e.max_exposure) for e in w.elts]
    t = w.terms
    z_layer = c.add_layer(z_elts, t.occ_ret, t.occ_lim, t.agg_ret, t.agg_lim)

    def timed(lay, surrogate):
        c.set_option(ara.OPT_INVERSION, ara.INV_NEWTON)
        c.set_option(ara.OPT_SURROGATE, 1 if surrogate else 0)
        c.set_option(ara.OPT_SCHEDULE, ara.SCHED_TRIAL)
        try:
            c.run(yet, lay, 0, w.yet.n_trials)  # warm (and the layer's start tables)
            s0 = c.stats()
            ts = []
            for _ in range(3):
                t0 = time.perf_counter()
                y = c.run(yet, lay, 0, w.yet.n_trials)
                ts.append(time.perf_counter() - t0)
            s1 = c.stats()
        finally:
            c.set_option(ara.OPT_SURROGATE, 0)
            c.set_option(ara.OPT_INVERSION, ara.INV_TABLE)
            c.set_option(ara.OPT_SCHEDULE, ara.SCHED_BAND)
        return sorted(ts)[1], y, {k: (s1[k] - s0[k]) / 3 for k in s0}

    tn, yn, _ = timed(layer, False)
    ts, ys, ds = timed(layer, True)
    t0, _, _ = timed(z_layer, False)
    net, fb = ds["surrogate_evals"], ds["inversions"]
    share = fb / (net + fb)
    pn, _ = c.risk_measures(yn, w.rps)
    ps, _ = c.risk_measures(ys, w.rps)
    print(f"paper-scale 20k trials: Newton-Halley {tn * 1e3:.2f} ms, surrogate {ts * 1e3:.2f} ms "
          f"(speed-up {tn / ts:.2f}), bookkeeping {t0 * 1e3:.2f} ms, network evaluations {net:.0f}, "
          f"fallback share {share:.1%}, PML rel diff {np.max(np.abs(ps - pn) / pn):.2e}")
    assert net > 0 and 0.0 < share < 1.0
    assert np.max(np.abs(ps - pn) / pn) <= 1e-3
    assert ts >= t0 + 0.8 * share * (tn - t0)  # the bound stated above holds on this run
