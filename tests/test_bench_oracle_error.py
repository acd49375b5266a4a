"""The benchmark's accuracy leg computes the oracle's PML/TVaR from the tail candidates of the
GPU's year-loss table only.  On the CPU: with year losses within the candidate rule (5e-5 of the
oracle's) the oracle's PML/TVaR from the candidates equal those of a full oracle run exactly, and
a table outside the rule is reported as such."""

import types

import numpy as np

import oracle
from paper_1310_2274_b300 import synth


def _bench():
    import bench  # the benchmark module (argument parsing happens in its main() only)

    return bench


def test_candidates_give_the_full_oracle_tail():
    bench = _bench()
    w = synth.tiny(5000)
    o, _ = oracle.run(w.yet, w.elts, w.terms, 42)
    rng = np.random.default_rng(5)
    y = o * (1.0 + rng.uniform(-2e-5, 2e-5, size=o.size))  # inside the rule
    p, t = oracle.risk(y, w.rps)
    a = types.SimpleNamespace(trials=w.yet.n_trials)
    fast = bench.oracle_error(a, w.yet, w.elts, w.terms, w.rps, {"g": (y, p, t, [0])})
    full = bench.oracle_error(a, w.yet, w.elts, w.terms, w.rps, {"g": (y, p, t, [0])}, full=True)
    assert fast["g"]["candidate_rule_holds"]
    assert fast["g"]["trials_checked"] < full["g"]["trials_checked"] == w.yet.n_trials
    assert fast["g"]["oracle_pml"] == full["g"]["oracle_pml"]
    assert fast["g"]["oracle_tvar"] == full["g"]["oracle_tvar"]
    op, ot = oracle.risk(o, w.rps)
    np.testing.assert_array_equal(fast["g"]["oracle_pml"], op)
    np.testing.assert_array_equal(fast["g"]["oracle_tvar"], ot)


def test_table_outside_the_rule_is_flagged():
    bench = _bench()
    w = synth.tiny(600)
    o, _ = oracle.run(w.yet, w.elts, w.terms, 42)
    y = o * (1.0 + 2e-4)
    p, t = oracle.risk(y, w.rps)
    a = types.SimpleNamespace(trials=w.yet.n_trials)
    r = bench.oracle_error(a, w.yet, w.elts, w.terms, w.rps, {"g": (y, p, t, [0])})
    assert not r["g"]["candidate_rule_holds"]
