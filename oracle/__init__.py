"""FP64 CPU oracle for aggregate risk analysis with secondary uncertainty.

TEST INFRASTRUCTURE ONLY: imported by tests/, by the package's smoke check and by the
benchmark's CPU-baseline leg, never by the library. The arithmetic lives in ara_oracle.c; this
module only marshals numpy arrays to it with ctypes.
"""

from __future__ import annotations

import ctypes as C
import os

import numpy as np

from . import build as _build

_lib = None


def lib():
    global _lib
    if _lib is None:
        _lib = C.CDLL(_build.build())
        _declare(_lib)
    return _lib


_P = C.c_void_p


def _declare(L):
    L.ora_philox4x32_10.argtypes = [_P, _P, _P]
    L.ora_philox4x32_10.restype = None
    L.ora_uniform.argtypes = [C.c_uint32]
    L.ora_uniform.restype = C.c_double
    L.ora_uniform_n.argtypes = [_P, C.c_int64, _P]
    L.ora_uniform_n.restype = None
    L.ora_su_uniform.argtypes = [C.c_uint64, C.c_int64, C.c_int64, C.c_int32]
    L.ora_su_uniform.restype = C.c_double
    L.ora_betainc.argtypes = [C.c_double, C.c_double, C.c_double]
    L.ora_betainc.restype = C.c_double
    L.ora_betaincinv.argtypes = [C.c_double, C.c_double, C.c_double, C.POINTER(C.c_int)]
    L.ora_betaincinv.restype = C.c_double
    L.ora_beta_moments.argtypes = [C.c_double, C.c_double, C.c_double,
                                   C.POINTER(C.c_double), C.POINTER(C.c_double)]
    L.ora_beta_moments.restype = C.c_int
    L.ora_occ_terms.argtypes = [C.c_double] * 3
    L.ora_occ_terms.restype = C.c_double
    L.ora_agg_terms.argtypes = [C.c_double] * 3
    L.ora_agg_terms.restype = C.c_double
    L.ora_su_loss.argtypes = [C.c_double] * 4 + [C.POINTER(C.c_int)]
    L.ora_su_loss.restype = C.c_double
    L.ora_su_uniform_corr.argtypes = [C.c_uint64, C.c_int64, C.c_int64]
    L.ora_su_uniform_corr.restype = C.c_double
    L.ora_norm_cdf.argtypes = [C.c_double]
    L.ora_norm_cdf.restype = C.c_double
    L.ora_norm_quantile.argtypes = [C.c_double]
    L.ora_norm_quantile.restype = C.c_double
    L.ora_su_combine.argtypes = [C.c_double] * 4
    L.ora_su_combine.restype = C.c_double
    L.ora_run.argtypes = [_P, _P, C.c_int32, _P, _P, _P, _P, _P, _P, _P, _P, C.c_uint64, _P,
                          C.c_int64, _P, _P, C.POINTER(C.c_int64), C.c_int]
    L.ora_run.restype = C.c_int
    L.ora_run_events.argtypes = [_P, _P, C.c_int32, _P, _P, _P, _P, _P, _P, _P, _P, C.c_uint64,
                                 _P, C.c_int64, _P, _P, _P, _P, C.POINTER(C.c_int64), C.c_int]
    L.ora_run_events.restype = C.c_int
    L.ora_trace.argtypes = [_P, _P, C.c_int32, _P, _P, _P, _P, _P, _P, _P, _P, C.c_uint64, _P,
                            C.c_int64, _P, C.c_int64, _P, _P, _P, _P, _P, _P, _P,
                            C.POINTER(C.c_int64)]
    L.ora_trace.restype = C.c_int
    L.ora_rank.argtypes = [_P, C.c_int64, _P]
    L.ora_rank.restype = C.c_int
    L.ora_tail_count.argtypes = [C.c_int64, C.c_double]
    L.ora_tail_count.restype = C.c_int64
    L.ora_risk.argtypes = [_P, C.c_int64, _P, C.c_int32, _P, _P]
    L.ora_risk.restype = C.c_int
    L.ora_counts_enable.argtypes = [C.c_int]
    L.ora_counts_enable.restype = None
    L.ora_counts_reset.argtypes = []
    L.ora_counts_reset.restype = None
    L.ora_counts_get.argtypes = [_P]
    L.ora_counts_get.restype = None


def _ptr(a: np.ndarray):
    return a.ctypes.data_as(_P)


def philox4x32_10(ctr, key) -> np.ndarray:
    c = np.ascontiguousarray(ctr, dtype=np.uint32)
    k = np.ascontiguousarray(key, dtype=np.uint32)
    out = np.zeros(4, dtype=np.uint32)
    lib().ora_philox4x32_10(_ptr(c), _ptr(k), _ptr(out))
    return out


def uniform(w: int) -> float:
    return lib().ora_uniform(int(w) & 0xFFFFFFFF)


def uniform_n(words) -> np.ndarray:
    w = np.ascontiguousarray(words, dtype=np.uint32)
    out = np.zeros(w.shape[0], dtype=np.float64)
    lib().ora_uniform_n(_ptr(w), w.shape[0], _ptr(out))
    return out


def su_uniform(seed: int, trial: int, k: int, elt: int) -> float:
    return lib().ora_su_uniform(seed, trial, k, elt)


def betainc(a: float, b: float, x: float) -> float:
    return lib().ora_betainc(a, b, x)


def betaincinv(a: float, b: float, p: float):
    st = C.c_int(0)
    x = lib().ora_betaincinv(a, b, p, C.byref(st))
    return x, st.value


def beta_moments(mean: float, sd: float, mx: float):
    a, b = C.c_double(0), C.c_double(0)
    rc = lib().ora_beta_moments(mean, sd, mx, C.byref(a), C.byref(b))
    return rc, a.value, b.value


def occ_terms(l, r, lim):
    return lib().ora_occ_terms(l, r, lim)


def agg_terms(s, r, lim):
    return lib().ora_agg_terms(s, r, lim)


def su_uniform_corr(seed: int, trial: int, k: int) -> float:
    return lib().ora_su_uniform_corr(seed, trial, k)


def norm_cdf(x: float) -> float:
    return lib().ora_norm_cdf(x)


def norm_quantile(p: float) -> float:
    return lib().ora_norm_quantile(p)


def su_combine(zp: float, ze: float, sd_i: float, sd_c: float) -> float:
    return lib().ora_su_combine(zp, ze, sd_i, sd_c)


def su_loss(mean, sd, mx, u):
    st = C.c_int(0)
    v = lib().ora_su_loss(mean, sd, mx, u, C.byref(st))
    return v, st.value


def _layer_arrays(elts, elt_handles):
    sizes = [e.n for e in elts]
    off = np.zeros(len(elts) + 1, dtype=np.int64)
    off[1:] = np.cumsum(sizes)
    cat = lambda f: (np.concatenate([np.asarray(f(e)) for e in elts]) if elts else
                     np.zeros(0))
    ids = np.ascontiguousarray(cat(lambda e: e.event_ids), dtype=np.int32)
    mean = np.ascontiguousarray(cat(lambda e: e.mean), dtype=np.float64)
    sd = np.ascontiguousarray(cat(lambda e: e.sd), dtype=np.float64)
    sdc = np.ascontiguousarray(cat(lambda e: e.sd_corr if getattr(e, "sd_corr", None) is not None
                                   else np.zeros(e.n)), dtype=np.float64)
    mx = np.ascontiguousarray(cat(lambda e: e.max_exposure), dtype=np.float64)
    h = np.ascontiguousarray(elt_handles if elt_handles is not None else np.arange(len(elts)),
                             dtype=np.int32)
    return off, ids, mean, sd, sdc, mx, h


def run(yet, elts, terms, seed, trials=None, elt_handles=None, threads: int = 0,
        with_oep: bool = False):
    """Year losses of the selected trials (all by default) -> (ylt float64, not_converged), or
    (ylt, oep, not_converged) with with_oep: oep = each year's largest occurrence loss."""
    off, ids, mean, sd, sdc, mx, h = _layer_arrays(elts, elt_handles)
    t = np.ascontiguousarray(np.arange(yet.n_trials) if trials is None else trials,
                             dtype=np.int64)
    yo = np.ascontiguousarray(yet.offsets, dtype=np.int64)
    yi = np.ascontiguousarray(yet.event_ids, dtype=np.int32)
    tr = np.array([terms.occ_ret, terms.occ_lim, terms.agg_ret, terms.agg_lim], dtype=np.float64)
    ylt = np.zeros(t.shape[0], dtype=np.float64)
    oep = np.zeros(t.shape[0], dtype=np.float64)
    nc = C.c_int64(0)
    rc = lib().ora_run(_ptr(yo), _ptr(yi), len(elts), _ptr(off), _ptr(ids), _ptr(mean),
                       _ptr(sd), _ptr(sdc), _ptr(mx), _ptr(h), _ptr(tr), seed, _ptr(t), t.shape[0],
                       _ptr(ylt), _ptr(oep) if with_oep else None, C.byref(nc), int(threads))
    if rc != 0:
        raise ValueError(f"oracle run failed: {rc}")
    return (ylt, oep, nc.value) if with_oep else (ylt, nc.value)


def run_portfolio(yet, elts, portfolio, seed, trials=None, threads: int = 0):
    """Algorithm 1's outer loops: portfolio = list of programs, each a list of layers
    (ELT indices into elts, Terms).  Every layer's YLT over the selected trials, in program then
    layer order -> float64 array [layers, trials].  An ELT's draws are keyed by its index in elts
    (its handle), so an ELT shared by several layers has the same losses in each."""
    rows = []
    for program in portfolio:
        for idx, terms in program:
            y, nc = run(yet, [elts[i] for i in idx], terms, seed, trials=trials,
                        elt_handles=list(idx), threads=threads)
            if nc:
                raise ValueError(f"{nc} inversions did not converge")
            rows.append(y)
    n = yet.n_trials if trials is None else len(trials)
    return np.array(rows).reshape(len(rows), n)


def run_events(yet, elts, terms, seed, trials=None, elt_handles=None, threads: int = 0):
    """Year losses plus the event-level outputs -> (ylt, oep, olt, inc, not_converged): oep = each
    year's largest occurrence loss; olt / inc per occurrence of the selected trials (concatenated
    in selection order) = occurrence loss after occurrence terms / increment of the year's net
    aggregate loss at that occurrence."""
    off, ids, mean, sd, sdc, mx, h = _layer_arrays(elts, elt_handles)
    t = np.ascontiguousarray(np.arange(yet.n_trials) if trials is None else trials,
                             dtype=np.int64)
    yo = np.ascontiguousarray(yet.offsets, dtype=np.int64)
    yi = np.ascontiguousarray(yet.event_ids, dtype=np.int32)
    tr = np.array([terms.occ_ret, terms.occ_lim, terms.agg_ret, terms.agg_lim], dtype=np.float64)
    n_occ = int(np.sum(yo[t + 1] - yo[t]))
    ylt = np.zeros(t.shape[0])
    oep = np.zeros(t.shape[0])
    olt = np.zeros(n_occ)
    inc = np.zeros(n_occ)
    nc = C.c_int64(0)
    rc = lib().ora_run_events(_ptr(yo), _ptr(yi), len(elts), _ptr(off), _ptr(ids), _ptr(mean),
                              _ptr(sd), _ptr(sdc), _ptr(mx), _ptr(h), _ptr(tr), seed, _ptr(t),
                              t.shape[0], _ptr(ylt), _ptr(oep), _ptr(olt), _ptr(inc),
                              C.byref(nc), int(threads))
    if rc != 0:
        raise ValueError(f"oracle run failed: {rc}")
    return ylt, oep, olt, inc, nc.value


def trace(yet, elts, terms, seed, trials, elt_handles=None, max_hits: int = 1 << 22):
    """Every hit of the selected trials in loop order, plus their year losses."""
    off, ids, mean, sd, sdc, mx, h = _layer_arrays(elts, elt_handles)
    t = np.ascontiguousarray(trials, dtype=np.int64)
    yo = np.ascontiguousarray(yet.offsets, dtype=np.int64)
    yi = np.ascontiguousarray(yet.event_ids, dtype=np.int32)
    tr = np.array([terms.occ_ret, terms.occ_lim, terms.agg_ret, terms.agg_lim], dtype=np.float64)
    ylt = np.zeros(t.shape[0], dtype=np.float64)
    out = dict(trial=np.zeros(max_hits, np.int64), k=np.zeros(max_hits, np.int64),
               j=np.zeros(max_hits, np.int32), rec=np.zeros(max_hits, np.int64),
               u=np.zeros(max_hits, np.float64), x=np.zeros(max_hits, np.float64),
               loss=np.zeros(max_hits, np.float64))
    nh = C.c_int64(0)
    rc = lib().ora_trace(_ptr(yo), _ptr(yi), len(elts), _ptr(off), _ptr(ids), _ptr(mean),
                         _ptr(sd), _ptr(sdc), _ptr(mx), _ptr(h), _ptr(tr), seed, _ptr(t), t.shape[0],
                         _ptr(ylt), max_hits, _ptr(out["trial"]), _ptr(out["k"]),
                         _ptr(out["j"]), _ptr(out["rec"]), _ptr(out["u"]), _ptr(out["x"]),
                         _ptr(out["loss"]), C.byref(nh))
    if rc != 0:
        raise ValueError(f"oracle trace failed: {rc}")
    n = min(nh.value, max_hits)
    return {k: v[:n] for k, v in out.items()}, ylt


def rank(ylt) -> np.ndarray:
    y = np.ascontiguousarray(ylt, dtype=np.float64)
    order = np.zeros(y.shape[0], dtype=np.int64)
    lib().ora_rank(_ptr(y), y.shape[0], _ptr(order))
    return order


def tail_count(n: int, rp: float) -> int:
    return int(lib().ora_tail_count(n, rp))


def risk(ylt, rps):
    y = np.ascontiguousarray(ylt, dtype=np.float64)
    r = np.ascontiguousarray(rps, dtype=np.float64)
    pml = np.zeros(r.shape[0])
    tvar = np.zeros(r.shape[0])
    rc = lib().ora_risk(_ptr(y), y.shape[0], _ptr(r), r.shape[0], _ptr(pml), _ptr(tvar))
    if rc != 0:
        raise ValueError("oracle risk measures: invalid input")
    return pml, tvar


class counting:
    """Context manager: collect the inverse's work counters over the enclosed calls."""

    NAMES = ("inversions", "newton", "bisect", "evals", "cf_terms", "not_conv")

    def __enter__(self):
        lib().ora_counts_reset()
        lib().ora_counts_enable(1)
        self.counts = None
        return self

    def __exit__(self, *exc):
        out = np.zeros(6, dtype=np.int64)
        lib().ora_counts_get(_ptr(out))
        lib().ora_counts_enable(0)
        self.counts = dict(zip(self.NAMES, (int(v) for v in out)))
        return False


def n_threads() -> int:
    return len(os.sched_getaffinity(0)) if hasattr(os, "sched_getaffinity") else os.cpu_count()
