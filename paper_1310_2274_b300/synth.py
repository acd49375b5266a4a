"""Seeded synthetic inputs for aggregate risk analysis: Year Event Table, Event Loss Tables, terms.

This module holds random draws only. No step of the method's arithmetic lives here, so both the
CUDA path (tests, bench) and the FP64 oracle (tests, CPU baseline) may take their inputs from it.

The paper's data (an industry YET and XELTs) is proprietary; these generators reproduce the shapes
the paper states and the value laws of the workloads built on it:

* YET (paper §2.1): each trial is a sequence of (event id, timestamp) pairs ordered by ascending
  timestamp; trials hold 800-1500 events in practice. Here every trial has the same number of
  events K (the C-ABI still takes CSR trial offsets). Event ids are uniform with replacement over
  the catalogue; timestamps are sorted uniforms on [0, 365) days, drawn as normalised cumulative
  exponential spacings (the order statistics of K uniforms) so no per-trial sort is needed.
* XELT (paper §2.1, §4.1): a set of distinct catalogue events with non-zero loss. The mean loss is
  LogNormal(12, 1.5) (natural-log parameters), the standard deviation is mean x U(0.3, 1.2) and
  the maximum exposure is mean x U(3, 10). Values are drawn in FP64 and rounded once to FP32, so
  the oracle (FP64) and the device (FP32) see the same numbers.
* Layer terms (paper §2.3): occurrence and aggregate retention/limit.

All generators are deterministic functions of their seed. Large YETs are generated in fixed
blocks of 65,536 trials, each with its own stream keyed by (seed, block), so memory stays bounded
and the result does not depend on how the work is split.
"""

from __future__ import annotations

import dataclasses

import numpy as np

YET_BLOCK = 1 << 16  # trials per generator stream; fixed so output is independent of chunking
DAYS = 365.0


@dataclasses.dataclass
class Yet:
    """Year Event Table in CSR form: trial i owns occurrences offsets[i]..offsets[i+1]-1."""

    offsets: np.ndarray  # int64 [n_trials + 1]
    event_ids: np.ndarray  # int32 [n_occ]
    timestamps: np.ndarray  # float32 [n_occ], nondecreasing within each trial
    catalog_size: int

    @property
    def n_trials(self) -> int:
        return int(self.offsets.shape[0] - 1)


@dataclasses.dataclass
class Elt:
    """Extended event loss table: one record per distinct event with non-zero loss."""

    event_ids: np.ndarray  # int32 [n], distinct
    mean: np.ndarray  # float64 [n], values exactly representable in float32
    sd: np.ndarray  # float64 [n]; the independent SD sigma_I when sd_corr is given
    max_exposure: np.ndarray  # float64 [n]
    sd_corr: np.ndarray = None  # float64 [n], correlated SD sigma_C (paper §3.1); None: zero

    @property
    def n(self) -> int:
        return int(self.event_ids.shape[0])


@dataclasses.dataclass
class Terms:
    """Layer terms (OccR, OccL, AggR, AggL), paper §2.1 and §2.3."""

    occ_ret: float
    occ_lim: float
    agg_ret: float
    agg_lim: float


def _yet_block(seed: int, block: int, n_trials: int, n_events: int, catalog: int):
    rng = np.random.default_rng([seed, block])
    ids = rng.integers(0, catalog, size=(n_trials, n_events), dtype=np.int32)
    spacing = rng.standard_exponential(size=(n_trials, n_events + 1), dtype=np.float32)
    csum = np.cumsum(spacing, axis=1, dtype=np.float32)
    ts = csum[:, :n_events] * (np.float32(DAYS) / csum[:, n_events:])
    # Rounding can only push a value to 365.0 itself; keep the half-open interval.
    np.minimum(ts, np.nextafter(np.float32(DAYS), np.float32(0)), out=ts)
    return ids, ts


def make_yet(n_trials: int, n_events: int, catalog: int, seed: int) -> Yet:
    """Fixed-K YET of n_trials x n_events occurrences over [0, catalog)."""
    n_occ = n_trials * n_events
    ids = np.empty(n_occ, dtype=np.int32)
    ts = np.empty(n_occ, dtype=np.float32)
    for block, t0 in enumerate(range(0, n_trials, YET_BLOCK)):
        nt = min(YET_BLOCK, n_trials - t0)
        b_ids, b_ts = _yet_block(seed, block, nt, n_events, catalog)
        ids[t0 * n_events:(t0 + nt) * n_events] = b_ids.reshape(-1)
        ts[t0 * n_events:(t0 + nt) * n_events] = b_ts.reshape(-1)
    offsets = np.arange(n_trials + 1, dtype=np.int64) * n_events
    return Yet(offsets, ids, ts, catalog)


def make_ragged_yet(n_trials: int, min_events: int, max_events: int, catalog: int,
                    seed: int) -> Yet:
    """YET whose trials hold U{min_events..max_events} events (0 allowed: an empty year)."""
    rng = np.random.default_rng([seed, 0x7A6])
    counts = rng.integers(min_events, max_events + 1, size=n_trials).astype(np.int64)
    offsets = np.zeros(n_trials + 1, dtype=np.int64)
    np.cumsum(counts, out=offsets[1:])
    ids = rng.integers(0, catalog, size=int(offsets[-1]), dtype=np.int32)
    ts = np.empty(int(offsets[-1]), dtype=np.float32)
    for i in range(n_trials):
        a, b = offsets[i], offsets[i + 1]
        ts[a:b] = np.sort(rng.uniform(0.0, DAYS, size=b - a).astype(np.float32))
    return Yet(offsets, ids, ts, catalog)


def _f32(x: np.ndarray) -> np.ndarray:
    return x.astype(np.float32).astype(np.float64)


def make_elt(n: int, catalog: int, seed: int, *, mu: float = 12.0, sigma: float = 1.5,
             sd_range=(0.3, 1.2), max_range=(3.0, 10.0), round32: bool = True) -> Elt:
    """ELT of n distinct events with the lognormal / beta parameterisation above.  Values are
    rounded once to binary32 (both sides then see the same numbers); round32=False keeps the
    binary64 draws of the same stream (the precision study's unrounded inputs)."""
    rnd = _f32 if round32 else (lambda x: x)
    rng = np.random.default_rng(seed)
    ids = rng.choice(catalog, size=n, replace=False).astype(np.int32)
    mean = rnd(rng.lognormal(mu, sigma, size=n))
    sd = rnd(mean * rng.uniform(sd_range[0], sd_range[1], size=n))
    mx = rnd(mean * rng.uniform(max_range[0], max_range[1], size=n))
    return Elt(ids, mean, sd, mx)


def split_sd(elt: Elt, seed: int, lo: float = 0.2, hi: float = 0.8) -> Elt:
    """The same ELT with each record's SD split into independent and correlated parts (paper
    §3.1): sigma_C = f32(sd U(1 - hi, 1 - lo)), sigma_I = f32(sd - sigma_C), so sigma_I + sigma_C
    stays within rounding of the original SD."""
    rng = np.random.default_rng([seed, 0xC0])
    sdc = _f32(elt.sd * (1.0 - rng.uniform(lo, hi, size=elt.n)))
    sdi = _f32(elt.sd - sdc)
    return Elt(elt.event_ids, elt.mean, sdi, elt.max_exposure, sdc)


def elt_size_for_seed(seed: int, lo: int = 20_000, hi: int = 200_000) -> int:
    """Record count of a paper-scale ELT: U{lo..hi} drawn from its own seed."""
    return int(np.random.default_rng([seed, 0x51E]).integers(lo, hi + 1))


# ---------------------------------------------------------------------------------------------
# Named workloads
# ---------------------------------------------------------------------------------------------

SEED_PHILOX = 42

TERMS_TINY = Terms(1e5, 1e7, 5e5, 5e7)
# Paper-scale layer: occurrence terms as in the tiny case; aggregate terms scaled to the ~900 hits
# per trial. On a 2,000-trial oracle sample the year sum S of occurrence losses spans
# 2.46e8..5.0e8 (0.1% / 50% / 99.9% quantiles 2.69e8 / 3.64e8 / 4.81e8), so with AggR = AggL =
# 2.5e8 both terms act, yet well under 1% of the years sit at 0 or at AggL and the 1-in-1000
# tail is not a block of ties.
TERMS_PAPER = Terms(1e5, 1e7, 2.5e8, 2.5e8)
RPS_TINY = (100.0, 250.0)
RPS_PAPER = (100.0, 250.0, 500.0, 1000.0)


@dataclasses.dataclass
class Workload:
    name: str
    yet: Yet
    elts: list
    terms: Terms
    rps: tuple
    seed: int = SEED_PHILOX


def tiny(n_trials: int = 1000) -> Workload:
    """1,000 trials x 100 events over a 10,000-event catalogue; one ELT of 2,000 records."""
    yet = make_yet(n_trials, 100, 10_000, seed=1)
    elt = make_elt(2_000, 10_000, seed=2)
    return Workload("tiny-1000x100x1", yet, [elt], TERMS_TINY, RPS_TINY)


def correlated(n_trials: int = 1000) -> Workload:
    """Paper §3.1-3.2 with both standard deviations: 1,000 trials x 100 events over a 10,000-event
    catalogue, three ELTs of 2,000 records whose SDs are split into independent and correlated
    parts, so that one occurrence's losses in the three ELTs are correlated."""
    yet = make_yet(n_trials, 100, 10_000, seed=1)
    elts = [split_sd(make_elt(2_000, 10_000, seed=s), seed=s) for s in (2, 3, 4)]
    return Workload(f"correlated-{n_trials}x100x3", yet, elts, Terms(1e5, 1e7, 1e6, 1e8), RPS_TINY)


def paper_elts(n_elts: int = 16, catalog: int = 2_000_000, first_seed: int = 2) -> list:
    return [make_elt(elt_size_for_seed(s), catalog, seed=s)
            for s in range(first_seed, first_seed + n_elts)]


def paper(n_trials: int = 800_000, n_events: int = 1000, n_elts: int = 16) -> Workload:
    """Paper-scale layer: 800,000 trials x 1,000 events, 2,000,000-event catalogue, 16 ELTs."""
    yet = make_yet(n_trials, n_events, 2_000_000, seed=1)
    return Workload(f"paper-{n_trials}x{n_events}x{n_elts}", yet, paper_elts(n_elts),
                    TERMS_PAPER, RPS_PAPER)


def precision(n_trials: int = 800_000) -> Workload:
    """Tiny per-trial shape (100 events, 10k catalogue, one ELT) at 800,000 trials."""
    yet = make_yet(n_trials, 100, 10_000, seed=1)
    elt = make_elt(2_000, 10_000, seed=2)
    return Workload(f"precision-{n_trials}x100x1", yet, [elt], TERMS_TINY, RPS_TINY)


def subset_trials(n_total: int, n_pick: int, seed: int = 7) -> np.ndarray:
    """Sorted distinct trial indices for a seeded sample of a YET."""
    rng = np.random.default_rng(seed)
    return np.sort(rng.choice(n_total, size=min(n_pick, n_total), replace=False)).astype(np.int64)
