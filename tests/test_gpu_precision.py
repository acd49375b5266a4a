"""Precision study of the year accumulation (FP64 against Kahan-compensated FP32) on the
precision workload: 800,000 trials x 100 events x 1 ELT, checked on its seeded 10,000-trial
subset against the FP64 oracle, which is also run on the unrounded binary64 ELT values to show
the effect of the single binary32 rounding of the inputs."""

import numpy as np
import pytest

from paper_1310_2274_b300 import synth

pytestmark = pytest.mark.gpu


def test_precision_study(ara, oracle):
    w = synth.precision()
    pick = synth.subset_trials(w.yet.n_trials, 10_000, seed=7)
    o, nc = oracle.run(w.yet, w.elts, w.terms, 42, trials=pick, elt_handles=[0])
    assert nc == 0
    e64 = synth.make_elt(2_000, 10_000, seed=2, round32=False)
    o_unr, _ = oracle.run(w.yet, [e64], w.terms, 42, trials=pick, elt_handles=[0])
    scale = np.maximum(np.maximum(np.abs(o), w.terms.agg_ret), 1.0)
    res = {}
    with ara.Context(seed=42) as c:
        yet, elts, layer = c.stage_workload(w)
        for name, mode in (("fp64", ara.ACC_FP64), ("kahan32", ara.ACC_KAHAN32)):
            c.set_option(ara.OPT_PRECISION, mode)
            g = c.run(yet, layer, 0, w.yet.n_trials)
            p, t = c.risk_measures(g, w.rps)
            res[name] = (g, p, t)
    rows = []
    for name, (g, p, t) in res.items():
        err = np.abs(g[pick] - o) / scale
        rows.append((name, err.max(), np.median(err)))
        assert err.max() <= 1e-5, name
    g64, p64, t64 = res["fp64"]
    gk, pk, tk = res["kahan32"]
    dp = np.max(np.abs(pk - p64) / p64)
    dt = np.max(np.abs(tk - t64) / t64)
    rnd = np.abs(o_unr - o) / scale
    print("\nprecision study (10,000-trial subset of 800,000 x 100 x 1):")
    for name, mx, md in rows:
        print(f"  {name:8s} YLT vs oracle: max {mx:.2e}, median {md:.2e}")
    print(f"  kahan32 vs fp64 (full 800,000 trials): PML {dp:.2e}, TVaR {dt:.2e}")
    print(f"  oracle on unrounded binary64 inputs vs binary32-rounded: max {rnd.max():.2e}")
    # Kahan-compensated binary32 sums of 100 terms stay at the binary64 result's accuracy
    assert dp <= 1e-6 and dt <= 1e-6
    assert np.max(np.abs(gk - g64) / np.maximum(np.abs(g64), w.terms.agg_ret)) <= 1e-6
