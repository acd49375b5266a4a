"""Pins for the oracle's YLT order and risk measures (paper §2.4).

PML(RP) is read as the year loss at rank k = N/RP (1-based, largest first) and TVaR(RP) as the
mean of the k largest year losses, ties broken by ascending trial index. Pinned by brute force
over all orderings of tiny YLTs and by invariants.
"""

import itertools
import math

import numpy as np
import pytest


def brute_order(y):
    # The unique permutation whose (loss desc, index asc) pairs are lexicographically sorted.
    n = len(y)
    best = None
    for perm in itertools.permutations(range(n)):
        ok = all((y[perm[r]] > y[perm[r + 1]]) or
                 (y[perm[r]] == y[perm[r + 1]] and perm[r] < perm[r + 1]) for r in range(n - 1))
        if ok:
            assert best is None
            best = perm
    return list(best)


@pytest.mark.parametrize("y", [
    [3.0, 1.0, 2.0],
    [5.0, 5.0, 0.0, 5.0, 1.0],
    [0.0, 0.0, 0.0, 0.0],
    [1e8, 2.5e7, 1e8, 0.0, 3.3, 1e8, 7.0],
])
def test_rank_brute_force(oracle, y):
    assert oracle.rank(np.array(y)).tolist() == brute_order(y)


def test_risk_brute_force_random(oracle):
    rng = np.random.default_rng(11)
    for _ in range(30):
        n = int(rng.integers(1, 8))
        y = rng.choice([0.0, 1.0, 2.5, 7.0, 1e6], size=n).tolist()
        order = brute_order(y)
        rps = [1.5, 2.0, 3.0, 7.0]
        pml, tvar = oracle.risk(np.array(y), rps)
        for q, rp in enumerate(rps):
            k = max(1, min(n, math.ceil(n / rp - 1e-12)))
            assert pml[q] == y[order[k - 1]]
            assert math.isclose(tvar[q], sum(y[o] for o in order[:k]) / k, rel_tol=1e-15)


def test_tail_count(oracle):
    assert oracle.tail_count(1000, 100) == 10
    assert oracle.tail_count(1000, 250) == 4
    assert oracle.tail_count(800_000, 1000) == 800
    assert oracle.tail_count(800_000, 250) == 3200
    assert oracle.tail_count(10_000, 500) == 20
    assert oracle.tail_count(10, 3) == 4  # 3.33 -> 4
    assert oracle.tail_count(5, 100) == 1  # at least one trial
    assert oracle.tail_count(7, 1.0000001) == 7


def test_risk_invariants(oracle):
    rng = np.random.default_rng(2)
    y = np.maximum(rng.lognormal(15, 2, 10_000) - 2e6, 0.0)
    rps = [10.0, 100.0, 250.0, 500.0, 1000.0]
    pml, tvar = oracle.risk(y, rps)
    assert np.all(tvar >= pml)
    assert np.all(np.diff(pml) >= 0) and np.all(np.diff(tvar) >= 0)
    s = np.sort(y)[::-1]
    for q, rp in enumerate(rps):
        k = int(round(10_000 / rp))
        assert pml[q] == s[k - 1]
        assert math.isclose(tvar[q], math.fsum(s[:k]) / k, rel_tol=1e-15)


def test_risk_rejects_bad_return_periods(oracle):
    with pytest.raises(ValueError):
        oracle.risk(np.ones(4), [1.0])
    with pytest.raises(ValueError):
        oracle.risk(np.ones(0), [10.0])
