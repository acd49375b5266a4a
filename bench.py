#!/usr/bin/env python3
"""Benchmark: aggregate risk analysis with secondary uncertainty, paper-scale layer on B300.

A step is one whole analysis of the paper-scale layer (800,000 trials x 1,000 events x 16 ELTs)
from raw inputs already resident in HBM: stage the YET (ara_create_yet), the 16 ELTs
(ara_add_elts: one call, one check) and the layer (ara_add_layer), run Algorithm 1 (ara_run ->
YLT; with ~400 hits per record a single pass buys the records' certified quantile tables, built in
binary32 in one launch, and inverts the beta CDF through them), take PML/TVaR at 1-in-100/250/500/
1000 (ara_risk_measures), and free everything.  The metric is trial-event-ELT evaluations per
second, N * K * J / step time, i.e. the paper's "s per 800k x 1000 run".  Beside it: the same
analysis re-priced with the tables resident (the serving situation), the step through host
buffers (e2e), the error of PML/TVaR against the FP64 oracle, the precision study, the learned
surrogate, serving, and the CPU oracle's rate.  Prints one JSON line (rank 0).

  python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]

--impl reference times the FP64 CPU oracle (the paper's method written plainly) on bounded
trial samples of the same workload, on this machine's host cores.
"""

from __future__ import annotations

import argparse
import json
import os
import statistics
import subprocess
import sys
import tempfile
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

from paper_1310_2274_b300 import synth  # noqa: E402

METRIC = "trial-event-ELT evals/s"
UNIT = "evals/s"
PEAKS = os.path.join(ROOT, "MEASURED_PEAKS.json")
SM_COUNT = 148
FP32_LANES_PER_SM = 128
FALLBACK_SM_MHZ = 2032.0

# Roofline per unit of work: the unit is one beta inversion and its frozen
# algorithmic work W_INV is what the oracle's algorithm (Lentz continued fraction inside a
# safeguarded Newton, the plain method of the paper's §3.3) spends per inversion on the
# paper-scale (alpha, beta, u) mix, counted by the oracle's own counters over 1,076,084
# inversions: 102.09 continued-fraction terms x 17.5 ops + 5.85 evaluations of ln I_x x 23 ops
# + 8 ops per inversion = 1,929 arithmetic ops, plus 88.9 math-library calls (1 op each).
# Against the FP32 issue peak (2 x 148 SMs x 128 lanes x clock) this gives the time the paper's
# method would need; the table path does far less work per inversion, so its fraction can pass 1.
W_INV_OPS = 1929.0
W_INV_CALLS = 88.9
W_INV = W_INV_OPS + W_INV_CALLS

# HBM view of the table path, reported beside it: bytes the method touches per launch = the
# event-word stream (4 B per occurrence) + one 32-byte table piece per table evaluation + the
# YLT (8 B per trial), against the measured copy bandwidth.
BYTES_PER_OCCURRENCE = 4.0
BYTES_PER_TABLE_EVAL = 32.0
BYTES_PER_TRIAL = 8.0

# Device-counted FP32 work of the Newton-Halley inversion (the device algorithm's own trip
# counts): continued-fraction term 14.25 ops; iteration 17 ops + 4 calls for the Newton step and
# 10 for Halley's correction; per inversion 14 + 2.
# inversions the table build performs per record with sd > 0: a knot and a midpoint check per
# piece, plus the analytic start of each of the record's four chains
BUILD_INVERSIONS_PER_RECORD = 2 * 64 + 4
FLOP_PER_CF_TERM = 14.25
FLOP_PER_NEWTON = 17.0 + 4.0 + 10.0
FLOP_PER_INVERSION = 14.0 + 2.0


def parse():
    p = argparse.ArgumentParser()
    p.add_argument("--gpus", type=int, default=1)
    p.add_argument("--steps", type=int, default=40)
    p.add_argument("--warmup", type=int, default=3)
    p.add_argument("--impl", choices=["ours", "reference"], default="ours")
    p.add_argument("--trials", type=int, default=800_000)
    p.add_argument("--events", type=int, default=1000)
    p.add_argument("--elts", type=int, default=16)
    p.add_argument("--no-e2e", action="store_true")
    p.add_argument("--no-cpu", action="store_true")
    p.add_argument("--cpu-seconds", type=float, default=12.0)
    p.add_argument("--no-serve", action="store_true")
    p.add_argument("--no-surrogate", action="store_true")
    p.add_argument("--serve-requests", type=int, default=100)
    p.add_argument("--no-oracle", action="store_true")
    p.add_argument("--oracle-full", action="store_true")
    return p.parse_args()


def dist_env():
    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return rank, world, local


def workload_config(a, world, l2_note=True):
    return {
        "workload": f"paper-scale layer {a.trials}x{a.events}x{a.elts} per GPU",
        "trials": a.trials, "events_per_trial": a.events, "elts": a.elts,
        "catalog": 2_000_000, "elt_records": "U{20000..200000} each",
        "terms": [synth.TERMS_PAPER.occ_ret, synth.TERMS_PAPER.occ_lim,
                  synth.TERMS_PAPER.agg_ret, synth.TERMS_PAPER.agg_lim],
        "return_periods": list(synth.RPS_PAPER), "philox_seed": 42,
        "parallelism": (f"trial batches on {world} GPU(s); global PML/TVaR by one all-gather of "
                        "each rank's k_max largest year losses" if world > 1 else
                        "trial batch on one GPU"),
        "l2": "inputs larger than L2: each step stages 6.4 GB of YET (event ids and "
              "timestamps) and its run streams the 3.2 GB of event ids",
    }


# ---------------------------------------------------------------------------------------------
# clocks
# ---------------------------------------------------------------------------------------------
class ClockSampler:
    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, device_index: int):
        self.idx = device_index
        self.proc = None
        self.path = None

    def start(self):
        fd, self.path = tempfile.mkstemp(suffix=".csv")
        os.close(fd)
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", str(self.idx), f"--query-gpu={self.FIELDS}",
                 "--format=csv,noheader,nounits", "-lms", "100"],
                stdout=open(self.path, "w"), stderr=subprocess.DEVNULL)
        except OSError:
            self.proc = None

    def stop(self):
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except subprocess.TimeoutExpired:
            self.proc.kill()
        sm, smax, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for line in open(self.path):
            f = [x.strip() for x in line.split(",")]
            if len(f) < 9:
                continue
            try:
                sm.append(float(f[1]))
                smax.append(float(f[2]))
            except ValueError:
                continue
            for n, v in zip(names, f[5:9]):
                if v.lower().startswith("active"):
                    reasons.add(n)
        os.unlink(self.path)
        return {"sm_mhz": statistics.median(sm) if sm else None,
                "sm_max_mhz": max(smax) if smax else None,
                "samples": len(sm), "reasons": sorted(reasons)}


# ---------------------------------------------------------------------------------------------
# CPU oracle on a bounded sample (the CPU baseline and the reference arm)
# ---------------------------------------------------------------------------------------------
def oracle_sample_rate(a, seconds: float, elts=None, sample_seed: int = 7):
    """evals/s of the FP64 oracle on a seeded sample of the workload's trials (all host cores)."""
    import oracle

    yet = synth.make_yet(min(a.trials, synth.YET_BLOCK), a.events, 2_000_000, seed=1)
    elts = elts if elts is not None else synth.paper_elts(a.elts)
    cores = oracle.n_threads()
    # grow the sample until one timed run lasts about `seconds` (the first call also pays for
    # building the oracle's search index, so it only sizes the next one)
    n, dt = 64, 0.0
    for _ in range(4):
        pick = synth.subset_trials(yet.n_trials, n, seed=sample_seed)
        t = time.perf_counter()
        oracle.run(yet, elts, synth.TERMS_PAPER, 42, trials=pick, threads=cores)
        dt = time.perf_counter() - t
        if dt >= 0.6 * seconds or n >= yet.n_trials:
            break
        n = int(min(yet.n_trials, max(2 * n, n * 1.1 * seconds / max(dt, 1e-3))))
    evals = n * a.events * a.elts
    return {"value": evals / dt, "unit": UNIT, "cores": cores, "kind": "oracle",
            "sample": f"{n} seeded trials of the first 65,536 of the workload's YET "
                      f"({a.events} events, {a.elts} ELTs), FP64 oracle, {dt:.1f} s wall"}


def run_reference(a):
    rank, world, _ = dist_env()
    if rank != 0:
        return 0
    import oracle  # noqa: F401

    elts = synth.paper_elts(a.elts)
    times, rates = [], []
    per_step = max(2.0, min(10.0, 120.0 / max(1, a.steps + a.warmup)))
    cb = None
    for s in range(a.warmup + a.steps):
        r = oracle_sample_rate(a, per_step, elts=elts, sample_seed=100 + s)
        if s >= a.warmup:
            rates.append(r["value"])
            cb = r
    value = statistics.median(rates)
    ms = a.trials * a.events * a.elts / value * 1e3
    line = {"metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": a.steps,
            "warmup": a.warmup, "ms_per_step": ms, "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": workload_config(a, 1), "impl": "reference",
            "cpu_baseline": cb,
            "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0,
                    "d2h_bytes_per_step": 0},
            "note": "reference arm = the FP64 CPU oracle on host cores; ms_per_step is the "
                    "full workload's time extrapolated linearly from the sampled rate"}
    print(json.dumps(line), flush=True)
    return 0


# ---------------------------------------------------------------------------------------------
# our arm
# ---------------------------------------------------------------------------------------------
PROFILE_FILES = {
    "band": ("band_kernel_table_200000x1000x16.md",
             ("ara_band.cu", "ara_trial_common.cuh", "ara_ibeta.cuh", "ara_philox.cuh")),
    "table_trial": ("trial_kernel_table_200000x1000x16.md",
                    ("ara_trial.cu", "ara_trial_common.cuh", "ara_ibeta.cuh", "ara_philox.cuh")),
    "table_build": ("build_tables_kernel_paper_16_elts.md",
                    ("ara_table.cu", "ara_table.cuh", "ara_ibeta.cuh")),
    "newton_trial": ("trial_kernel_newton_50000x1000x16.md",
                     ("ara_trial.cu", "ara_trial_common.cuh", "ara_ibeta.cuh", "ara_philox.cuh")),
}


def profile_for_current_kernel(schedule):
    """Figures from the committed ncu summary of the dominant kernel (DRAM bytes per 800k-trial
    launch, pipe and memory utilisation), if that capture was taken on the current kernel
    source; else {}."""
    import hashlib

    name, files = PROFILE_FILES[schedule]
    path = os.path.join(ROOT, "profiles", name)
    if not os.path.exists(path):
        return {}
    rec = {}
    for line in open(path):
        if ":" in line and not line.startswith(("|", "#", " ")):
            k, v = line.split(":", 1)
            rec[k.strip()] = v.strip()
    h = hashlib.sha256()
    for f in files:
        h.update(open(os.path.join(ROOT, "paper_1310_2274_b300", "csrc", f), "rb").read())
    if rec.get("source_sha256") != h.hexdigest():
        return {}
    out = {"metrics": {k[len("metric "):]: float(v) for k, v in rec.items()
                       if k.startswith("metric ")}}
    if "dram_bytes_per_launch" in rec:
        out["dram_bytes_per_launch"] = float(rec["dram_bytes_per_launch"])
    return out


def ev_pair():
    import torch

    return torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)


def time_calls(fn, k, stream, dev):
    """Mean device time of fn() over k calls (CUDA events on the library's stream)."""
    import torch

    ev = [ev_pair() for _ in range(k)]
    for e0, e1 in ev:
        e0.record(stream)
        fn()
        e1.record(stream)
    torch.cuda.synchronize(dev)
    return statistics.mean(e0.elapsed_time(e1) for e0, e1 in ev)


def peaks():
    hbm_peak, sm_mhz = 6442.9, FALLBACK_SM_MHZ
    src = "fallback"
    if os.path.exists(PEAKS):
        pk = json.load(open(PEAKS))
        hbm_peak = float(pk.get("hbm_gbs", hbm_peak))
        sm_mhz = float(pk.get("sm_max_mhz", FALLBACK_SM_MHZ))
        src = "measured"
    return hbm_peak, sm_mhz, src


def run_ours(a):
    import torch
    import torch.distributed as dist

    import paper_1310_2274_b300 as ara
    from paper_1310_2274_b300 import shards

    rank, world, local = dist_env()
    if world > 1:
        dist.init_process_group("nccl", init_method="env://")
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)

    # each GPU processes its own batch of trials (independent YET seed): weak scaling
    yet_h = synth.make_yet(a.trials, a.events, 2_000_000, seed=1 + rank)
    elts_h = synth.paper_elts(a.elts)
    terms = synth.TERMS_PAPER
    rps = list(synth.RPS_PAPER)
    n = a.trials
    evals = n * a.events * a.elts

    stream = torch.cuda.current_stream(dev)
    ctx = ara.Context(seed=42, device=local)
    ctx.set_stream(stream)
    hbm_peak, sm_mhz, peak_src = peaks()
    alu_peak = 2.0 * SM_COUNT * FP32_LANES_PER_SM * sm_mhz * 1e6 / 1e12  # TFLOP/s FP32

    # raw inputs resident in HBM (the step's inputs; staging them is part of the step)
    to_dev = lambda x: torch.from_numpy(np.ascontiguousarray(x)).to(dev)  # noqa: E731
    off_d, ids_d, ts_d = (to_dev(yet_h.offsets), to_dev(yet_h.event_ids),
                          to_dev(yet_h.timestamps))
    elts_d = [tuple(to_dev(v) for v in (e.event_ids, e.mean, e.sd, e.max_exposure))
              for e in elts_h]
    ylt = torch.empty(n, dtype=torch.float64, device=dev)
    run_ev = []

    def risk(y):
        # one rank: PML/TVaR of its YLT; several: the global tails of all ranks' trials through
        # the one exchange of the trial-sharded path (each rank's k_max largest, gathered)
        if world > 1:
            return shards.global_risk(ctx, y, world * n, rps)
        return ctx.risk_measures(y, rps)

    cold_handles = []

    def cold_step(timed):
        yet = ctx.create_yet(off_d, ids_d, ts_d, 2_000_000)
        elts = ctx.add_elts(yet, elts_d)
        cold_handles[:] = elts  # the uniforms are keyed by the ELT handles (the oracle needs them)
        layer = ctx.add_layer(elts, terms.occ_ret, terms.occ_lim, terms.agg_ret, terms.agg_lim)
        if timed:
            e0, e1 = ev_pair()
            e0.record(stream)
        ctx.run(yet, layer, 0, n, out=ylt, stream=stream)
        if timed:
            e1.record(stream)
            run_ev.append((e0, e1))
        out = risk(ylt)
        ctx.free_layer(layer)
        for e in elts:
            ctx.free_elt(e)
        ctx.free_yet(yet)
        return out

    # ---- the headline: one whole analysis per step (tables on demand: this single pass of ~400
    # expected hits per record buys them, all 16 ELTs' in one launch, then runs trial-major) ----
    ctx.set_option(ara.OPT_TABLES, ara.TABLES_ON_DEMAND)
    for _ in range(a.warmup):
        cold_step(False)
    torch.cuda.synchronize(dev)
    s0 = ctx.stats()
    clocks = ClockSampler(local)
    clocks.start()
    t_start, t_end = ev_pair()
    if world > 1:
        dist.barrier()
    torch.cuda.synchronize(dev)
    t_start.record(stream)
    for _ in range(a.steps):
        pml, tvar = cold_step(True)
    t_end.record(stream)
    torch.cuda.synchronize(dev)
    if world > 1:
        dist.barrier()
    clk = clocks.stop()
    s1 = ctx.stats()
    step_ms = t_start.elapsed_time(t_end) / a.steps
    if world > 1:
        t = torch.tensor([step_ms], device=dev)
        dist.all_reduce(t, op=dist.ReduceOp.MAX)
        step_ms = float(t.item())
    run_ms = statistics.mean(e0.elapsed_time(e1) for e0, e1 in run_ev)
    value = world * evals / (step_ms * 1e-3)
    d = {k: (s1[k] - s0[k]) / a.steps for k in s0}
    ylt_cold = ylt.cpu().numpy().copy()  # the last timed step's YLT (its ELT handles: cold_handles)
    pml_cold, tvar_cold = [float(v) for v in pml], [float(v) for v in tvar]

    # where a step's time goes, by API call (host clock, each call followed by a synchronise;
    # outside the timed region)
    def phases():
        out = {}

        def tick(name, t0):
            torch.cuda.synchronize(dev)
            out[name] = out.get(name, 0.0) + (time.perf_counter() - t0) * 1e3
            return time.perf_counter()
        torch.cuda.synchronize(dev)
        t = time.perf_counter()
        yet_p = ctx.create_yet(off_d, ids_d, ts_d, 2_000_000)
        t = tick("create_yet", t)
        elts_p = ctx.add_elts(yet_p, elts_d)
        t = tick("add_elts_16", t)
        layer_p = ctx.add_layer(elts_p, terms.occ_ret, terms.occ_lim, terms.agg_ret,
                                terms.agg_lim)
        t = tick("add_layer", t)
        ctx.run(yet_p, layer_p, 0, n, out=ylt, stream=stream)
        t = tick("run", t)
        risk(ylt)
        t = tick("risk_measures", t)
        ctx.free_layer(layer_p)
        for e in elts_p:
            ctx.free_elt(e)
        ctx.free_yet(yet_p)
        tick("frees", t)
        return out
    step_phases = phases()

    # ---- a persistent staging of the same data for the other legs -----------------------------
    yet = ctx.create_yet(off_d, ids_d, ts_d, 2_000_000)
    t_st = time.perf_counter()
    ctx.set_option(ara.OPT_TABLES, ara.TABLES_EAGER)  # certified tables built at staging
    elts = ctx.add_elts(yet, elts_d)
    torch.cuda.synchronize(dev)
    tables_build_s = time.perf_counter() - t_st
    layer = ctx.add_layer(elts, terms.occ_ret, terms.occ_lim, terms.agg_ret, terms.agg_lim)
    nrep = max(3, min(10, a.steps))

    def run_layer(l=None):
        ctx.run(yet, layer if l is None else l, 0, n, out=ylt, stream=stream)

    # the table kernel alone, trial-major as in the headline step (tables resident)
    ctx.set_option(ara.OPT_SCHEDULE, ara.SCHED_TRIAL)
    run_layer()
    table_trial_ms = time_calls(run_layer, nrep, stream, dev)
    # Newton-Halley on both schedules (trial-major first: the band-major copy does not exist yet;
    # the band schedule after the table runs below made it)
    ctx.set_option(ara.OPT_INVERSION, ara.INV_NEWTON)
    run_layer()
    torch.cuda.synchronize(dev)
    sn0 = ctx.stats()
    newton_trial_ms = time_calls(run_layer, nrep, stream, dev)
    sn1 = ctx.stats()
    ylt_newton = ylt.cpu().numpy().copy()
    pml_n, tvar_n = ctx.risk_measures(ylt, rps)
    ctx.set_option(ara.OPT_INVERSION, ara.INV_TABLE)
    dn = {k: (sn1[k] - sn0[k]) / nrep for k in sn0}

    # ---- re-pricing: the same layer with its certified tables resident (band schedule) --------
    ctx.set_option(ara.OPT_SCHEDULE, ara.SCHED_BAND)  # makes the band-major copy at once
    run_layer()
    s2 = ctx.stats()
    rep_ev = [ev_pair() for _ in range(a.steps)]
    r0, r1 = ev_pair()
    r0.record(stream)
    for e0, e1 in rep_ev:
        e0.record(stream)
        run_layer()
        e1.record(stream)
        pml_t, tvar_t = ctx.risk_measures(ylt, rps)
    r1.record(stream)
    torch.cuda.synchronize(dev)
    s3 = ctx.stats()
    rep_step_ms = r0.elapsed_time(r1) / a.steps
    band_ms = statistics.mean(e0.elapsed_time(e1) for e0, e1 in rep_ev)
    dr = {k: (s3[k] - s2[k]) / a.steps for k in s2}
    ylt_table = ylt.cpu().numpy().copy()
    ctx.set_option(ara.OPT_INVERSION, ara.INV_NEWTON)
    run_layer()
    newton_band_ms = time_calls(run_layer, nrep, stream, dev)
    ctx.set_option(ara.OPT_INVERSION, ara.INV_TABLE)

    # roofline of the headline's run call (unit of work: one beta inversion per hit, the
    # per-unit work W_INV frozen from the oracle's algorithm): the binary32 table build (one
    # launch over the 16 ELTs), the layer's table gather and the trial-major table kernel
    n_inv = d["inversions"] + d["table_evals"] + d["surrogate_evals"]
    achieved = n_inv * W_INV / (run_ms * 1e-3) / 1e12
    build_ms = max(run_ms - table_trial_ms, 1e-3)  # the build and the gather
    n_sd = sum(int(np.count_nonzero(e.sd > 0)) for e in elts_h)
    build_inv = n_sd * BUILD_INVERSIONS_PER_RECORD
    prof_t = profile_for_current_kernel("table_trial")
    prof_bt = profile_for_current_kernel("table_build")
    bytes_trial = (BYTES_PER_OCCURRENCE * n * a.events + BYTES_PER_TABLE_EVAL * d["table_evals"]
                   + BYTES_PER_TRIAL * n)
    roofline = {
        "bound": "alu", "achieved": achieved, "peak": alu_peak, "unit": "TFLOP/s",
        "frac": achieved / alu_peak,
        "traffic": (prof_t["dram_bytes_per_launch"] * n / 800_000
                    if prof_t.get("dram_bytes_per_launch") else None),
        "kernel": "the step's ara_run call: build_tables_kernel (the 16 ELTs' certified tables, "
                  "132 binary32 Newton-Halley inversions per record), the layer's table gather, "
                  "trial_kernel with the table inversion (one warp per trial); CUDA events "
                  "inside the timed region; traffic: the table kernel's",
        "kernel_ms": run_ms, "units_per_launch": n_inv,
        "unit_of_work": "one beta inversion per hit (W_inv each, the paper method's work): the "
                        "tables reuse each record's inversions across its ~400 hits, so the run "
                        "does less arithmetic than the units it is credited with",
        "w_inv": {"ops": W_INV_OPS, "library_calls": W_INV_CALLS,
                  "source": "oracle counters, 1,076,084 paper-scale inversions"},
        "peak_source": f"FP32 issue peak 2 x {SM_COUNT} SMs x {FP32_LANES_PER_SM} lanes x "
                       f"{sm_mhz:.0f} MHz (derived; {peak_src} SM clock)",
        "build": {"ms": build_ms, "inversions": build_inv,
                  "achieved": build_inv * W_INV / (build_ms * 1e-3) / 1e12,
                  "frac": build_inv * W_INV / (build_ms * 1e-3) / 1e12 / alu_peak,
                  "note": "run call minus the table kernel timed alone; inversions: 2 x 64 "
                          "knots and midpoints + 4 chain starts per record with sd > 0",
                  "ncu": prof_bt.get("metrics")},
        "table_kernel": {"ms": table_trial_ms, "bytes_per_launch": bytes_trial,
                         "hbm_achieved": bytes_trial / (table_trial_ms * 1e-3) / 1e9,
                         "hbm_peak": hbm_peak,
                         "hbm_frac": bytes_trial / (table_trial_ms * 1e-3) / 1e9 / hbm_peak,
                         "ncu": prof_t.get("metrics")},
    }
    prof = profile_for_current_kernel("newton_trial")
    flops = (FLOP_PER_CF_TERM * dn["cf_terms"] + FLOP_PER_NEWTON * dn["newton"] +
             FLOP_PER_INVERSION * dn["inversions"])
    n_inv_n = dn["inversions"] + dn["table_evals"]
    newton_roofline = {
        "bound": "alu", "achieved": n_inv_n * W_INV / (newton_trial_ms * 1e-3) / 1e12,
        "peak": alu_peak, "unit": "TFLOP/s",
        "frac": n_inv_n * W_INV / (newton_trial_ms * 1e-3) / 1e12 / alu_peak,
        "traffic": (prof["dram_bytes_per_launch"] * n / 800_000
                    if prof.get("dram_bytes_per_launch") else None),
        "kernel": "trial_kernel, Newton-Halley inversion from start tables (one warp per "
                  "trial), tables absent; timed alone",
        "kernel_ms": newton_trial_ms, "inversions_per_launch": n_inv_n,
        "device_counted": {"flops_per_launch": flops,
                           "achieved": flops / (newton_trial_ms * 1e-3) / 1e12,
                           "frac": flops / (newton_trial_ms * 1e-3) / 1e12 / alu_peak,
                           "per_launch": {k: dn[k] for k in ("inversions", "newton",
                                                              "cf_terms")}},
        "ncu": prof.get("metrics"),
    }
    n_inv_t = dr["table_evals"] + dr["inversions"]
    bytes_launch = (BYTES_PER_OCCURRENCE * n * a.events + BYTES_PER_TABLE_EVAL * dr["table_evals"]
                    + BYTES_PER_TRIAL * n)
    prof_b = profile_for_current_kernel("band")
    repricing = {
        "ms_per_step": rep_step_ms, "value": world * evals / (rep_step_ms * 1e-3),
        "kernel": "band_kernel + band_finalize_kernel, certified-table inversion (catalogue "
                  "bands in L2), then ara_risk_measures",
        "kernel_ms": band_ms, "trial_major_ms": table_trial_ms,
        "tables_build_s_16_elts": tables_build_s,
        "roofline": {"bound": "alu", "achieved": n_inv_t * W_INV / (band_ms * 1e-3) / 1e12,
                     "peak": alu_peak, "unit": "TFLOP/s",
                     "frac": n_inv_t * W_INV / (band_ms * 1e-3) / 1e12 / alu_peak,
                     "note": "counts W_inv per evaluation although the certified quintic does "
                             "~60 ops: the inversion work was done when the tables were built "
                             "at staging (tables_build_s), outside this step, so this fraction "
                             "is the step's time against the paper's method at peak, not a "
                             "hardware efficiency",
                     "hbm_view": {"achieved": bytes_launch / (band_ms * 1e-3) / 1e9,
                                  "peak": hbm_peak, "unit": "GB/s",
                                  "frac": bytes_launch / (band_ms * 1e-3) / 1e9 / hbm_peak,
                                  "bytes_per_launch": bytes_launch},
                     "traffic": (prof_b["dram_bytes_per_launch"] * n / 800_000
                                 if prof_b.get("dram_bytes_per_launch") else None),
                     "ncu": prof_b.get("metrics")},
        "per_launch": {k: dr[k] for k in ("hits", "table_evals", "inversions")},
        "risk_measures": {"pml": [float(v) for v in pml_t], "tvar": [float(v) for v in tvar_t]},
    }

    # ---- precision variant: Kahan-compensated FP32 year sums on the same data ------------------
    ctx.set_option(ara.OPT_PRECISION, ara.ACC_KAHAN32)
    run_layer()
    kahan_ms = time_calls(run_layer, nrep, stream, dev)
    kp, kt = ctx.risk_measures(ylt, rps)
    ylt_kahan = ylt.cpu().numpy().copy()
    ctx.set_option(ara.OPT_PRECISION, ara.ACC_FP64)
    precision = {"fp64_exact_band_ms": band_ms, "kahan32_ms": kahan_ms,
                 "kahan32_schedule": "trial-major (order-dependent sums)",
                 "pml_rel_diff_vs_exact": max(abs(float(x) / float(y) - 1.0)
                                              for x, y in zip(kp, pml_t)),
                 "tvar_rel_diff_vs_exact": max(abs(float(x) / float(y) - 1.0)
                                               for x, y in zip(kt, tvar_t))}

    # ---- event-level outputs: OEP year table, per-occurrence losses and net increments --------
    n_occ = int(yet_h.offsets[n] - yet_h.offsets[0])
    ev_out = (torch.empty(n, dtype=torch.float64, device=dev),
              torch.empty(n, dtype=torch.float64, device=dev),
              torch.empty(n_occ, dtype=torch.float32, device=dev),
              torch.empty(n_occ, dtype=torch.float64, device=dev))
    run_events = lambda: ctx.run_events(yet, layer, 0, n, n_occ, out=ev_out, stream=stream)  # noqa: E731
    run_events()
    events_ms = time_calls(run_events, nrep, stream, dev)
    oep_p, _ = ctx.risk_measures(ev_out[1], rps)
    oep_capped = float(torch.count_nonzero(ev_out[1] >= terms.occ_lim).item()) / n
    run_layer()  # the re-pricing YLT again (exact sums)
    ev_y_equal = bool(torch.equal(ev_out[0], ylt))
    del ev_out
    # the OEP tail of a layer whose occurrence limit binds no occurrence (1e10 lies above every
    # event's loss bound here), so the 1-in-N OEP are distinct losses rather than ties at OccL
    u_layer = ctx.add_layer(elts, terms.occ_ret, 1e10, terms.agg_ret, 1e12)
    oep_t = torch.empty(n, dtype=torch.float64, device=dev)
    ctx.run_ep(yet, u_layer, 0, n, out=ylt, oep=oep_t, stream=stream)
    oep_u, oep_ut = ctx.risk_measures(oep_t, rps)
    ctx.free_layer(u_layer)
    del oep_t
    events = {"ms": events_ms, "schedule": "trial-major", "occurrences": n_occ,
              "output_bytes": n_occ * 12 + n * 16,
              "ylt_identical_to_repricing": ev_y_equal,
              "oep_pml_occl_1e7": [float(x) for x in oep_p],
              "oep_years_at_occl_share": oep_capped,
              "oep_uncapped": {"occ_lim": 1e10, "pml": [float(x) for x in oep_u],
                               "tvar": [float(x) for x in oep_ut]}}

    # ---- portfolio: three programs of layers over the same ELTs, one call vs one run per layer -
    rng_pf = np.random.default_rng(5)
    pf_layers, pf_elts = [], 0
    for _prog in range(3):
        for _l in range(3):
            k = int(rng_pf.integers(3, len(elts) + 1))
            pick = [elts[i] for i in rng_pf.choice(len(elts), size=k, replace=False)]
            pf_elts += k
            pf_layers.append(ctx.add_layer(pick, terms.occ_ret, terms.occ_lim,
                                           terms.agg_ret * k / len(elts),
                                           terms.agg_lim * k / len(elts)))
    pf_rows = {}
    for n_pf in (n, min(n, 20_000)):
        pf_out = torch.empty((len(pf_layers), n_pf), dtype=torch.float64, device=dev)
        one = lambda: ctx.run_portfolio(yet, pf_layers, 0, n_pf, out=pf_out, stream=stream)  # noqa: E731

        def each():
            for i, l in enumerate(pf_layers):
                ctx.run(yet, l, 0, n_pf, out=pf_out[i], stream=stream)
        one()
        pf_rows[str(n_pf)] = {"one_call_ms": time_calls(one, 3, stream, dev),
                              "per_layer_runs_ms": time_calls(each, 3, stream, dev)}
        del pf_out
    for l in pf_layers:
        ctx.free_layer(l)
    portfolio = {"programs": 3, "layers": len(pf_layers), "elts_per_layer_mean":
                 pf_elts / len(pf_layers), "by_trials": pf_rows}

    # ---- where the time goes (the paper's split of lookup and secondary uncertainty, §5): the
    # same layer with every SD zero, so each hit is looked up, drawn and loaded but not inverted
    z_elts = [ctx.add_elt(yet, e.event_ids, e.mean, np.zeros(e.n), e.max_exposure)
              for e in elts_h]
    z_layer = ctx.add_layer(z_elts, terms.occ_ret, terms.occ_lim, terms.agg_ret, terms.agg_lim)
    run_layer(z_layer)
    sd0_ms = time_calls(lambda: run_layer(z_layer), nrep, stream, dev)
    ctx.free_layer(z_layer)
    for e in z_elts:
        ctx.free_elt(e)
    time_split = {"sd0_ms": sd0_ms, "table_ms": band_ms, "newton_ms": newton_band_ms,
                  "inversion_share_table": 1.0 - sd0_ms / band_ms,
                  "inversion_share_newton": 1.0 - sd0_ms / newton_band_ms,
                  "note": "sd0: lookups, draws, piece loads, event sums and terms without the "
                          "inversion (band schedule); the rest of each run is its inversion"}

    # ---- correlated standard deviations (paper §3.1-3.2) on the same YET ----------------------
    c_elts = []
    for i, e in enumerate(elts_h):
        es = synth.split_sd(e, seed=100 + i)
        c_elts.append(ctx.add_elt(yet, es.event_ids, es.mean, es.sd, es.max_exposure,
                                  es.sd_corr))
    c_layer = ctx.add_layer(c_elts, terms.occ_ret, terms.occ_lim, terms.agg_ret, terms.agg_lim)
    run_layer(c_layer)
    corr_ms = time_calls(lambda: run_layer(c_layer), nrep, stream, dev)
    cp, _ = ctx.risk_measures(ylt, rps)
    ctx.free_layer(c_layer)
    for e in c_elts:
        ctx.free_elt(e)
    correlated = {"ms": corr_ms, "vs_independent_only": corr_ms / band_ms,
                  "split": "sigma_C = sd x U(0.2, 0.8), sigma_I = sd - sigma_C per record",
                  "pml": [float(x) for x in cp]}

    result = {
        "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": a.steps,
        "warmup": a.warmup, "ms_per_step": step_ms, "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "f32",
        "data": "synthetic (seeded; shapes and value laws of the paper's workload)",
        "config": workload_config(a, world),
        "seconds_per_run": step_ms * 1e-3,
        "gpu_launches": int(s1["launches"] - s0["launches"]),
        "clocks": clk,
        "roofline": roofline,
        "step": {"what": "ara_create_yet (device arrays: copy + validation) + ara_add_elts (16 "
                         "ELTs from device arrays, one check) + ara_add_layer + ara_run + "
                         "ara_risk_measures + frees; tables on demand (this single pass buys "
                         "them: one build launch over the layer's records, then the trial-major "
                         "table kernel)",
                 "run_ms": run_ms, "phases_ms": step_phases,
                 "per_launch": {k: d[k] for k in ("hits", "table_evals", "inversions",
                                                  "newton", "cf_terms")},
                 "risk_measures": {"rps": rps, "pml": pml_cold, "tvar": tvar_cold}},
        "repricing": repricing,
        "newton_path": {"trial_major_ms": newton_trial_ms, "band_ms": newton_band_ms,
                        "band_note": "band schedule once the YET's band-major copy exists",
                        "roofline": newton_roofline,
                        "risk_measures": {"pml": [float(v) for v in pml_n],
                                          "tvar": [float(v) for v in tvar_n]}},
        "schedules_ms": {"table_band": band_ms, "table_trial": table_trial_ms,
                         "newton_trial": newton_trial_ms, "newton_band": newton_band_ms},
        "precision": precision,
        "event_outputs": events,
        "portfolio": portfolio,
        "correlated_sd": correlated,
        "time_split": time_split,
        "uncertified_records": s1["uncertified"],
    }

    # ---- learned surrogate of the inverse (trained here on the GPU) --------------------------
    if not a.no_surrogate:
        result["surrogate"] = surrogate_leg(a, ara, ctx, yet, layer, ylt, stream, dev,
                                            newton_trial_ms)
        ylt_surr = result["surrogate"].pop("_ylt")  # (YLT, PML, TVaR) of the surrogate run
    else:
        ylt_surr = None

    # ---- continuous-batching service on the resident YET (64 ELTs) ---------------------------
    if not a.no_serve and rank == 0:
        result["serving"] = serving(a, ara, ctx, yet, elts, dev)

    ctx.free_layer(layer)
    for e in elts:
        ctx.free_elt(e)
    ctx.free_yet(yet)
    del off_d, ids_d, ts_d, elts_d
    torch.cuda.empty_cache()

    # ---- end to end through the public API with host buffers ---------------------------------
    if not a.no_e2e:
        result["e2e"] = e2e(a, ara, ctx, yet_h, elts_h, terms, rps, dev, stream)

    # ---- accuracy against the FP64 oracle, and the precision study (rank 0, one GPU) ----------
    if rank == 0 and world == 1 and not a.no_oracle:
        result["oracle_error"] = oracle_error(
            a, yet_h, elts_h, terms, rps,
            {"single_pass": (ylt_cold, pml_cold, tvar_cold, list(cold_handles)),
             "newton": (ylt_newton, pml_n, tvar_n, elts),
             "table_repricing": (ylt_table, pml_t, tvar_t, elts),
             "kahan32": (ylt_kahan, kp, kt, elts),
             "surrogate": ylt_surr + (elts,) if ylt_surr is not None else None},
            full=a.oracle_full)
        result["precision_study"] = precision_study(a, ara, ctx, dev, stream)
    ctx.close()

    # ---- CPU baseline (rank 0, one GPU only) --------------------------------------------------
    if rank == 0 and world == 1 and not a.no_cpu:
        cb = oracle_sample_rate(a, a.cpu_seconds, elts=elts_h)
        cb["single_thread"] = oracle_single_thread(a, elts_h, a.cpu_seconds)
        result["cpu_baseline"] = cb
    if world > 1:
        dist.destroy_process_group()
    if rank == 0:
        print(json.dumps(result), flush=True)
    return 0


# accepted error of the surrogate (relative to a record's mean loss), and the other values the
# tiny workload is run at
SURROGATE_EPS = 5e-4
EPS_SWEEP = (2.5e-4, 1e-3, 2e-3)


def surrogate_leg(a, ara, ctx, yet, layer, ylt, stream, dev, newton_ms):
    """Trains the surrogate on 5e7 exact tuples (the GPU's own kernels), then runs the
    paper-scale layer with it (network inside its certified cells, Newton-Halley elsewhere)
    against the Newton-Halley run, and the tiny workload with and without it against the FP64
    oracle."""
    import torch

    import oracle

    t = time.perf_counter()
    rep = ctx.train_surrogate(n_samples=50_000_000, steps=30_000, batch=8192, lr=3e-3,
                              lr_final=3e-5, eps=SURROGATE_EPS, cert_samples=16, seed=3)
    train_s = time.perf_counter() - t
    run = lambda: ctx.run(yet, layer, 0, a.trials, out=ylt, stream=stream)  # noqa: E731
    ctx.set_option(ara.OPT_SURROGATE, 1)
    try:
        run()
        torch.cuda.synchronize(dev)
        s0 = ctx.stats()
        ms = time_calls(run, 2, stream, dev)
        s1 = ctx.stats()
        y_s = ylt.cpu().numpy().copy()
        sp, st = ctx.risk_measures(ylt, list(synth.RPS_PAPER))
        # the tiny workload (one ELT of 2,000 records), surrogate and plain, against the oracle;
        # the surrogate also at other accepted errors eps (the cell table is kept)
        w = synth.tiny()
        ty, te, tl = ctx.stage_workload(w)
        g_s = ctx.run(ty, tl, 0, w.yet.n_trials)
        sweep = {}
        for eps in EPS_SWEEP:
            ctx.set_surrogate_eps(eps)
            e0 = ctx.stats()
            g_e = ctx.run(ty, tl, 0, w.yet.n_trials)
            e1 = ctx.stats()
            sweep[eps] = (g_e, e1["surrogate_evals"] - e0["surrogate_evals"],
                          e1["inversions"] - e0["inversions"])
        ctx.set_surrogate_eps(SURROGATE_EPS)
        ctx.set_option(ara.OPT_SURROGATE, 0)
        ctx.set_option(ara.OPT_INVERSION, ara.INV_NEWTON)
        g_n = ctx.run(ty, tl, 0, w.yet.n_trials)
    finally:
        ctx.set_option(ara.OPT_SURROGATE, 0)
        ctx.set_option(ara.OPT_INVERSION, ara.INV_TABLE)
    o, _ = oracle.run(w.yet, w.elts, w.terms, 42, elt_handles=te)
    op, ot = oracle.risk(o, w.rps)

    def errors(g):
        gp, gt = ctx.risk_measures(g, w.rps)
        scale = np.maximum(np.maximum(np.abs(o), w.terms.agg_ret), 1.0)
        return {"ylt_max_err": float(np.max(np.abs(g - o) / scale)),
                "pml_rel_err": [abs(float(x) / float(y) - 1.0) for x, y in zip(gp, op)],
                "tvar_rel_err": [abs(float(x) / float(y) - 1.0) for x, y in zip(gt, ot)]}

    tiny = {name: errors(g) for name, g in (("surrogate", g_s), ("newton", g_n))}
    tiny["surrogate_eps_sweep"] = [
        dict(eps=eps, fallback_rate=fb / max(1, net + fb), **errors(g))
        for eps, (g, net, fb) in sweep.items()]
    ctx.free_layer(tl)
    for e in te:
        ctx.free_elt(e)
    ctx.free_yet(ty)
    net = (s1["surrogate_evals"] - s0["surrogate_evals"]) / 2
    fb = (s1["inversions"] - s0["inversions"]) / 2
    return {"kernel_ms": ms, "newton_ms": newton_ms, "speedup_vs_newton": newton_ms / ms,
            "network_evals": net, "fallback_rate": fb / max(1, net + fb),
            "cells_accepted": rep["cells_accepted"], "train_s": train_s,
            "eps": SURROGATE_EPS,
            "eps_meaning": "a hit is served where its cell's certified error in x is <= eps x "
                           "mu_beta: each served loss within eps of the record's mean loss",
            "train": {"tuples": 50_000_000, "steps": 30_000, "batch": 8192, "eps": SURROGATE_EPS,
                      "gen_ms": rep["gen_ms"], "train_ms": rep["train_ms"],
                      "cert_ms": rep["cert_ms"], "bad_targets": rep["bad_targets"]},
            "tiny_vs_oracle": tiny, "_ylt": (y_s, sp, st)}


def serving(a, ara, ctx, yet, elts16, dev):
    """Poisson arrivals of layer requests against the resident YET and 64 ELTs (seeds 2..65):
    ELT count U{1..64}, trials U{10,000..N} (prefix ranges), terms log-uniform around the
    paper-scale layer's.  Three legs: the plain form at 20 requests/s (seed 11), the plain form
    at 200 requests/s, which saturates the server and measures its capacity, and the learned
    surrogate form at 20 requests/s.  Reports latency percentiles, capacity and batching."""
    import torch

    more = synth.paper_elts(64 - len(elts16), first_seed=2 + len(elts16))
    elts = list(elts16) + [ctx.add_elt(yet, e.event_ids, e.mean, e.sd, e.max_exposure)
                           for e in more]
    torch.cuda.synchronize(dev)

    def requests(rate, n_req, seed):
        rng = np.random.default_rng(seed)
        gaps = rng.exponential(1.0 / rate, size=n_req)
        reqs = []
        for _ in range(n_req):
            k = int(rng.integers(1, 65))
            pick = [elts[i] for i in np.sort(rng.choice(64, size=k, replace=False))]
            lu = lambda lo, hi: float(np.exp(rng.uniform(np.log(lo), np.log(hi))))  # noqa: E731
            scale = k / 16.0
            reqs.append(dict(elts=pick, occ_ret=lu(3e4, 3e5), occ_lim=lu(3e6, 3e7),
                             agg_ret=scale * lu(1.25e8, 5e8), agg_lim=scale * lu(1.25e8, 5e8),
                             t0=0, n_trials=int(rng.integers(10_000, a.trials + 1)),
                             rps=synth.RPS_PAPER))
        return reqs, gaps

    def leg(rate, n_req, seed, surrogate=False):
        reqs, gaps = requests(rate, n_req, seed)
        evals = sum(r["n_trials"] * a.events * len(r["elts"]) for r in reqs)
        with ara.Server(ctx, yet, max_inflight=16, slice_trials=65536,
                        max_batch_trials=1 << 20, use_surrogate=surrogate) as srv:
            t = time.perf_counter()
            tickets = []
            for r, g in zip(reqs, gaps):
                time.sleep(g)
                tickets.append(srv.submit(**r))
            for tk in tickets:
                if srv.wait(tk, 600.0) != 0:
                    raise RuntimeError(f"serving request {tk} failed")
            wall = time.perf_counter() - t
            st = srv.stats()
        return {"requests": n_req, "arrival_rate_per_s": rate, "wall_s": wall,
                "latency_p50_ms": st["latency_p50_s"] * 1e3,
                "latency_p99_ms": st["latency_p99_s"] * 1e3,
                "latency_max_ms": st["latency_max_s"] * 1e3,
                "requests_per_s": st["requests_per_s"], "evals_per_s": evals / wall,
                "mean_requests_per_launch": st["mean_items_per_launch"],
                "launches": st["launches"], "failed": st["failed"],
                "form": "learned surrogate" if surrogate else "plain (certified tables)"}

    out = {"workload": "resident YET + 64 paper-scale ELTs; Poisson arrivals; ELTs U{1..64}, "
                       "trials U{10000..N} prefixes",
           "plain_20_per_s": leg(20.0, a.serve_requests, 11),
           "saturated": leg(200.0, 2 * a.serve_requests, 12)}
    if not a.no_surrogate:
        out["surrogate_20_per_s"] = leg(20.0, a.serve_requests, 11, surrogate=True)
    for h in elts[len(elts16):]:
        ctx.free_elt(h)
    return out


def oracle_error(a, yet_h, elts_h, terms, rps, ylts, full=False):
    """PML/TVaR (and year losses) of the GPU's paper-scale YLTs against the FP64 oracle.

    ylts: name -> (YLT, the GPU's PML, TVaR from ara_risk_measures, the ELT handles of the run:
    they key the uniforms).  PML/TVaR at RP need only the trials of the tail.  The candidates are
    the trials whose year loss, in any YLT of the same handles, is at least its k_max-th largest
    (k_max = N / min RP) times (1 - 1e-4); the oracle's own k_max largest are among them as long
    as every year loss is within 5e-5 of the oracle's (half that margin; the plain path's parity
    bar is 1e-5), which `candidate_rule_holds` reports from the trials checked (the candidates and
    a seeded sample of 2,000 others).  The oracle computes the candidates' year losses, everything
    else is set below them, and the oracle's PML/TVaR follow exactly.  full=True runs the oracle
    over every trial instead (minutes)."""
    import oracle

    n = a.trials
    k_max = max(oracle.tail_count(n, rp) for rp in rps)
    cores = oracle.n_threads()
    groups = {}  # handles -> names
    for name, v in ylts.items():
        if v is not None:
            groups.setdefault(tuple(int(h) for h in v[3]), []).append(name)
    out = {"method": "full oracle run" if full else
           "oracle on the tail candidates of every YLT plus a seeded sample of 2,000 others",
           "oracle_cores": cores, "rps": list(rps), "oracle_s": 0.0, "candidates": 0}
    rng = np.random.default_rng(23)
    for handles, names in groups.items():
        cand = set()
        for name in names:
            y = ylts[name][0]
            thr = np.partition(y, n - k_max)[n - k_max]
            cand.update(np.nonzero(y >= thr * (1.0 - 1e-4))[0].tolist())
        cand = np.array(sorted(cand), dtype=np.int64)
        others = np.setdiff1d(np.arange(n), cand)
        sample = np.sort(rng.choice(others, size=min(2000, others.size), replace=False))
        pick = np.arange(n) if full else np.union1d(cand, sample)
        t = time.perf_counter()
        o_pick, nc = oracle.run(yet_h, elts_h, terms, 42, trials=pick, elt_handles=list(handles),
                                threads=cores)
        out["oracle_s"] += time.perf_counter() - t
        out["candidates"] += int(cand.size)
        o = np.zeros(n)
        o[pick] = o_pick
        op, ot = oracle.risk(o, rps)
        for name in names:
            y, gp, gt = ylts[name][:3]
            scale = np.maximum(np.maximum(np.abs(o[pick]), terms.agg_ret), 1.0)
            err = np.abs(y[pick] - o[pick]) / scale
            over = o[pick] > terms.agg_ret
            rel = np.abs(y[pick][over] - o[pick][over]) / o[pick][over]
            out[name] = {
                "pml_rel_err": [abs(float(g) / float(r) - 1.0) for g, r in zip(gp, op)],
                "tvar_rel_err": [abs(float(g) / float(r) - 1.0) for g, r in zip(gt, ot)],
                "ylt_err_max": float(err.max()), "ylt_err_median": float(np.median(err)),
                "ylt_pure_rel_err_max_above_aggr": float(rel.max()) if rel.size else None,
                "candidate_rule_holds": bool(full or err.max() <= 5e-5),
                "trials_checked": int(pick.size), "oracle_not_converged": int(nc),
                "pml": [float(v) for v in gp], "oracle_pml": [float(v) for v in op],
                "tvar": [float(v) for v in gt], "oracle_tvar": [float(v) for v in ot]}
    return out


def precision_study(a, ara, ctx, dev, stream):
    """Precision study on the tiny per-trial shape at 800,000 trials (100 events, one ELT of
    2,000 records): exact FP64 year sums and Kahan-compensated FP32 sums (FP32 sampling and
    layer terms, FP64 tail sums in both), each against the FP64 oracle on the same binary32
    inputs and on the unrounded binary64 inputs, over the full run and a seeded 10,000-trial
    subset."""
    import torch

    import oracle

    w = synth.precision(800_000)
    elt64 = synth.make_elt(2_000, 10_000, seed=2, round32=False)
    sub = synth.subset_trials(w.yet.n_trials, 10_000, seed=7)
    yet, elts, layer = ctx.stage_workload(w)
    cores = oracle.n_threads()
    t = time.perf_counter()
    o, _ = oracle.run(w.yet, w.elts, w.terms, 42, elt_handles=elts, threads=cores)
    o64, _ = oracle.run(w.yet, [elt64], w.terms, 42, elt_handles=elts, threads=cores)
    oracle_s = time.perf_counter() - t
    out = {"workload": "800,000 trials x 100 events, catalogue 10,000, one ELT of 2,000 "
                       "records, terms 1e5/1e7/5e5/5e7, RP 100/250; subset: 10,000 trials "
                       "(seed 7)", "oracle_s": oracle_s, "oracle_cores": cores}
    y = torch.empty(w.yet.n_trials, dtype=torch.float64, device=dev)
    for name, prec in (("fp64_exact", ara.ACC_FP64), ("kahan32", ara.ACC_KAHAN32)):
        ctx.set_option(ara.OPT_PRECISION, prec)
        ctx.run(yet, layer, 0, w.yet.n_trials, out=y, stream=stream)
        ms = time_calls(lambda: ctx.run(yet, layer, 0, w.yet.n_trials, out=y, stream=stream), 3,
                        stream, dev)
        g = y.cpu().numpy().copy()
        row = {"ms": ms}
        for ref_name, ref in (("vs_oracle", o), ("vs_oracle_unrounded_inputs", o64)):
            r = {}
            for part, idx in (("full", None), ("subset", sub)):
                gg = g if idx is None else g[idx]
                oo = ref if idx is None else ref[idx]
                scale = np.maximum(np.maximum(np.abs(oo), w.terms.agg_ret), 1.0)
                err = np.abs(gg - oo) / scale
                gp, gt = ctx.risk_measures(gg, w.rps)
                op, ot = oracle.risk(oo, w.rps)
                over = oo > w.terms.agg_ret
                r[part] = {"ylt_err_max": float(err.max()),
                           "ylt_err_median": float(np.median(err)),
                           "ylt_err_p99": float(np.percentile(err, 99)),
                           "ylt_pure_rel_err_max_above_aggr":
                               float((np.abs(gg[over] - oo[over]) / oo[over]).max()),
                           "pml_rel_err": [abs(float(x) / float(z) - 1.0) for x, z in zip(gp, op)],
                           "tvar_rel_err": [abs(float(x) / float(z) - 1.0)
                                            for x, z in zip(gt, ot)]}
            row[ref_name] = r
        out[name] = row
    ctx.set_option(ara.OPT_PRECISION, ara.ACC_FP64)
    ctx.free_layer(layer)
    for e in elts:
        ctx.free_elt(e)
    ctx.free_yet(yet)
    return out


def oracle_single_thread(a, elts, seconds):
    """The oracle on one host core, on a seeded sample sized to about `seconds`, extrapolated
    linearly in trials to the whole workload (the paper finds the run linear in trials, §5)."""
    import oracle

    yet = synth.make_yet(min(a.trials, synth.YET_BLOCK), a.events, 2_000_000, seed=1)
    n, dt = 16, 0.0
    for _ in range(4):
        pick = synth.subset_trials(yet.n_trials, n, seed=31)
        t = time.perf_counter()
        oracle.run(yet, elts, synth.TERMS_PAPER, 42, trials=pick, threads=1)
        dt = time.perf_counter() - t
        if dt >= 0.6 * seconds:
            break
        n = int(min(yet.n_trials, max(2 * n, n * 1.1 * seconds / max(dt, 1e-3))))
    rate = n * a.events * a.elts / dt
    return {"value": rate, "unit": UNIT, "cores": 1, "sample": f"{n} seeded trials, {dt:.1f} s",
            "s_per_run_extrapolated": a.trials * a.events * a.elts / rate}


def e2e(a, ara, ctx, yet_h, elts_h, terms, rps, dev, stream):
    import torch

    def pinned(x):
        t = torch.from_numpy(np.ascontiguousarray(x)).pin_memory()
        return t, t.numpy()

    off_t, off = pinned(yet_h.offsets)
    ids_t, ids = pinned(yet_h.event_ids)
    ts_t, ts = pinned(yet_h.timestamps)
    elt_p = [tuple(pinned(v) for v in (e.event_ids, e.mean, e.sd, e.max_exposure))
             for e in elts_h]
    ylt_t, ylt = pinned(np.zeros(a.trials))
    # the runs never read timestamps: the library checks them on host threads and copies the
    # event ids, offsets and ELT arrays
    h2d = ids.nbytes + off.nbytes + sum(v[1].nbytes for p in elt_p for v in p)
    d2h = ylt.nbytes + 2 * 8 * len(rps)

    def step(host_yet):
        make = ctx.create_yet_host if host_yet else ctx.create_yet
        yet = make(off, ids, ts, 2_000_000)
        elts = ctx.add_elts(yet, [tuple(v[1] for v in p) for p in elt_p])
        layer = ctx.add_layer(elts, terms.occ_ret, terms.occ_lim, terms.agg_ret, terms.agg_lim)
        ctx.run(yet, layer, 0, a.trials, out=ylt)
        pml, tvar = ctx.risk_measures(ylt, rps)
        ctx.free_layer(layer)
        for e in elts:
            ctx.free_elt(e)
        ctx.free_yet(yet)
        return pml

    steps = max(1, min(a.steps, 5))

    def timed(policy, host_yet):
        # tables on demand: one pass of this workload (~400 expected hits per record) is above
        # the break-even of building them, so the run builds them first (one launch over the 16
        # ELTs); eager builds each ELT's at staging.  A host-resident YET is streamed by the run,
        # its copy overlapping the run.
        ctx.set_option(ara.OPT_TABLES, policy)
        try:
            for _ in range(min(a.warmup, 2)):
                step(host_yet)
            torch.cuda.synchronize(dev)
            t = time.perf_counter()
            for _ in range(steps):
                step(host_yet)
            torch.cuda.synchronize(dev)
            return (time.perf_counter() - t) / steps
        finally:
            ctx.set_option(ara.OPT_TABLES, ara.TABLES_EAGER)

    dt = timed(ara.TABLES_ON_DEMAND, True)
    dt_resident = timed(ara.TABLES_ON_DEMAND, False)
    dt_eager = timed(ara.TABLES_EAGER, False)
    _, world = dist_env()[:2]
    evals = a.trials * a.events * a.elts
    return {"value": world * evals / dt, "unit": UNIT, "h2d_bytes_per_step": int(h2d),
            "d2h_bytes_per_step": int(d2h), "ms_per_step": dt * 1e3, "steps": steps,
            "yet": "host-resident, its event ids streamed by the run (copy overlapping compute); "
                   "timestamps checked on host threads meanwhile",
            "tables": "on demand (rent-or-buy): this single pass builds them, then uses them",
            "resident_yet_ms_per_step": dt_resident * 1e3,
            "resident_yet_eager_tables_ms_per_step": dt_eager * 1e3,
            "path": "ara_create_yet_host + ara_add_elts (16 ELTs) + ara_add_layer from pinned host "
                    "memory, ara_run into a host YLT, ara_risk_measures, frees"}


def main():
    a = parse()
    if a.impl == "reference":
        return run_reference(a)
    return run_ours(a)


if __name__ == "__main__":
    sys.exit(main())
