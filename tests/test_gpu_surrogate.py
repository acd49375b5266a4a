"""The learned surrogate of InvCDF_beta: tensor-core forward and backward kernels against the FP64
reference network (oracle/mlp.py), training on the GPU, certification, and its use inside the run
with exact Newton fallback, measured against the FP64 oracle and against the method without it.
"""

import time

import numpy as np
import pytest

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
    p = ref.init_params(7)
    with ara.Context() as c:
        y = c.mlp_eval(z, params=p)
    yr, _ = ref.forward(p, z)
    # BF16 weights and activations against binary64 throughout
    assert rel_l2(y, yr) <= 2e-2
    assert np.corrcoef(y, yr)[0, 1] >= 0.999


def test_gradient_matches_reference_network(ara, batch):
    z, x, t = batch
    p = ref.init_params(7)
    with ara.Context() as c:
        loss, g = c.mlp_grad(p, z, x, t)
    lr_, gr = ref.loss_grad(p, z, x, t)
    assert abs(loss - lr_) <= 2e-2 * abs(lr_)
    parts_g, parts_r = ref.unpack(g.astype(np.float64)), ref.unpack(gr)
    names = ["W1", "b1", "W2", "b2", "W3", "b3", "W4", "b4"]
    for name, a, b in zip(names, parts_g, parts_r):
        a, b = a.reshape(-1), b.reshape(-1)
        cos = float(a @ b / (np.linalg.norm(a) * np.linalg.norm(b) + 1e-30))
        assert cos >= 0.995, (name, cos)
        assert rel_l2(a, b) <= 8e-2, (name, rel_l2(a, b))


@pytest.fixture(scope="module")
def trained(ara):
    c = ara.Context(seed=42)
    rep = c.train_surrogate(n_samples=8_000_000, steps=30_000, batch=8192, lr=3e-3,
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


def test_surrogate_gain_over_newton_on_paper_sample(ara, trained):
    # what the network gains over the method without it: the same run with Newton everywhere
    # against the surrogate with Newton fallback, on 20,000 trials of the paper-scale layer
    c, _ = trained
    w = synth.paper(n_trials=20_000)
    yet, elts, layer = c.stage_workload(w)
    times = {}
    for mode in ("newton", "surrogate"):
        c.set_option(ara.OPT_INVERSION, ara.INV_NEWTON)
        c.set_option(ara.OPT_SURROGATE, 1 if mode == "surrogate" else 0)
        c.run(yet, layer, 0, w.yet.n_trials)  # warm
        t = time.perf_counter()
        y = c.run(yet, layer, 0, w.yet.n_trials)
        times[mode] = (time.perf_counter() - t, y)
    c.set_option(ara.OPT_SURROGATE, 0)
    c.set_option(ara.OPT_INVERSION, ara.INV_TABLE)
    (tn, yn), (ts, ys) = times["newton"], times["surrogate"]
    pn, _ = c.risk_measures(yn, w.rps)
    ps, _ = c.risk_measures(ys, w.rps)
    print(f"paper-scale 20k trials: Newton {tn * 1e3:.2f} ms, surrogate {ts * 1e3:.2f} ms, "
          f"PML rel diff {np.max(np.abs(ps - pn) / pn):.2e}")
    assert np.max(np.abs(ps - pn) / pn) <= 1e-3
