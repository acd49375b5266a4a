"""Trial shards across ranks (one process per GPU) and the one exchange they need.

Trials are independent (paper §2.2, §5), so a YET is split into contiguous trial ranges, one per
rank, and each rank computes its YLT alone.  The global PML and TVaR (§2.4) of all N_total trials
need, for each return period RP, the k = N_total/RP largest year losses of all shards.  Each rank
sends the k_max largest of its own (k_max for the smallest return period) in ascending trial
order; gathered in rank order they are in global trial order, so ordering them by (loss
descending, position ascending) is the global ordering restricted to these candidates, which hold
every year loss any tail needs.  The candidate selection and the risk measures run in the
library's kernels; torch.distributed moves k_max values per rank (64 KB at 800,000 trials per
rank and RP 100).

The numeric backend is any object with top_k(ylt, k) and risk_measures_n(values, n_total, rps):
the library context on GPUs.
"""

from __future__ import annotations

import math


def tail_count(n: int, rp: float) -> int:
    """k = n/RP, rounded up when not an integer (within 1e-9 relative), clamped to [1, n]."""
    q = n / rp
    r = round(q)
    k = r if abs(q - r) <= 1e-9 * max(1.0, q) else math.ceil(q)
    return min(max(k, 1), n)


def shard_range(n_total: int, world: int, rank: int) -> tuple:
    """Contiguous trial range (t0, n) of a rank: the first n_total % world ranks take one more."""
    base, extra = divmod(n_total, world)
    t0 = rank * base + min(rank, extra)
    return t0, base + (1 if rank < extra else 0)


def global_risk(backend, ylt_local, n_total: int, rps, group=None):
    """PML and TVaR of all ranks' trials; every rank receives them.

    ylt_local: this rank's year losses, for its trials in order (a torch tensor on the rank's
    device, or on the CPU for the gloo backend)."""
    import torch
    import torch.distributed as dist

    world = dist.get_world_size(group)
    k_max = max(tail_count(n_total, rp) for rp in rps)
    k_loc = min(k_max, int(ylt_local.shape[0]))
    cand = backend.top_k(ylt_local, k_loc)
    if not isinstance(cand, torch.Tensor):
        cand = torch.as_tensor(cand)
    dev = cand.device
    sizes = [torch.zeros(1, dtype=torch.int64, device=dev) for _ in range(world)]
    dist.all_gather(sizes, torch.tensor([k_loc], dtype=torch.int64, device=dev), group=group)
    width = max(int(s.item()) for s in sizes)
    padded = torch.zeros(width, dtype=torch.float64, device=dev)
    padded[:k_loc] = cand
    parts = [torch.zeros(width, dtype=torch.float64, device=dev) for _ in range(world)]
    dist.all_gather(parts, padded, group=group)
    values = torch.cat([p[:int(s.item())] for p, s in zip(parts, sizes)]).contiguous()
    return backend.risk_measures_n(values, n_total, rps)
