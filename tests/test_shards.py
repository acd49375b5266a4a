"""Trial shards on CPU ranks: the exchange behind the global PML/TVaR, with world size 2 over
gloo.  The numeric backend is a plain stand-in (the oracle's ordering and tail counts) so that
the orchestration -- candidate counts, padding, gather order, tail counts of the global trial
count -- is checked without a GPU; the device versions of top_k and risk_measures_n are checked
against the oracle in tests/test_gpu_band.py."""

import os
import tempfile

import numpy as np
import pytest
import torch
import torch.distributed as dist
import torch.multiprocessing as mp

import oracle
from paper_1310_2274_b300 import shards


class OracleBackend:
    """top_k and risk_measures_n written out with the oracle's ordering (test stand-in)."""

    def top_k(self, ylt, k):
        y = ylt.numpy() if isinstance(ylt, torch.Tensor) else np.asarray(ylt)
        order = oracle.rank(y)  # (loss desc, index asc)
        pick = np.sort(order[:k])
        return torch.from_numpy(y[pick].copy())

    def risk_measures_n(self, values, n_total, rps):
        v = values.numpy()
        order = oracle.rank(v)
        pml, tvar = [], []
        for rp in rps:
            k = oracle.tail_count(n_total, rp)
            top = v[order[:k]]
            pml.append(top[-1])
            tvar.append(float(np.sum(top)) / k)
        return np.array(pml), np.array(tvar)


N_TOTAL = 10_007
RPS = (10.0, 100.0, 1000.5, 5000.0)


def full_ylt(seed=3):
    rng = np.random.default_rng(seed)
    y = np.round(rng.lognormal(10, 1.2, N_TOTAL), -3)  # rounded: many ties across shards
    y[rng.choice(N_TOTAL, 50, replace=False)] = y.max()  # a block of ties at the top
    return y


def _rank_main(rank, world, init_file, out_file):
    dist.init_process_group("gloo", init_method=f"file://{init_file}", rank=rank,
                            world_size=world)
    try:
        y = full_ylt()
        t0, n = shards.shard_range(N_TOTAL, world, rank)
        pml, tvar = shards.global_risk(OracleBackend(), torch.from_numpy(y[t0:t0 + n].copy()),
                                       N_TOTAL, RPS)
        np.save(f"{out_file}.{rank}.npy", np.concatenate([pml, tvar]))
    finally:
        dist.destroy_process_group()


@pytest.mark.parametrize("world", [2, 3])
def test_global_risk_over_gloo_ranks_equals_single_process(world):
    with tempfile.TemporaryDirectory() as d:
        init_file = os.path.join(d, "init")
        out_file = os.path.join(d, "out")
        mp.spawn(_rank_main, args=(world, init_file, out_file), nprocs=world, join=True)
        results = [np.load(f"{out_file}.{r}.npy") for r in range(world)]
    pml, tvar = oracle.risk(full_ylt(), RPS)
    for res in results:  # every rank receives the same, and it is the single-process answer
        np.testing.assert_array_equal(res[:len(RPS)], pml)
        np.testing.assert_allclose(res[len(RPS):], tvar, rtol=1e-15)


def test_tail_count_matches_oracle():
    for n in (1, 7, 999, 1000, 800_000, 10_007):
        for rp in (1.5, 2.0, 10.0, 100.0, 250.0, 333.3, 1000.5, 1e7):
            assert shards.tail_count(n, rp) == oracle.tail_count(n, rp), (n, rp)


def test_shard_ranges_cover_the_trials_once():
    for n_total, world in ((10, 3), (800_000, 8), (5, 8), (0, 2)):
        seen = []
        for r in range(world):
            t0, n = shards.shard_range(n_total, world, r)
            seen.extend(range(t0, t0 + n))
        assert seen == list(range(n_total))
