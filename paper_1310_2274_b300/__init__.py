"""B300-native aggregate risk analysis with secondary uncertainty (arXiv 1310.2274).

Thin Python binding of the C-ABI library libara.so (declared in include/ara.h): argument
marshalling only.  Every step of the method runs in the library's CUDA kernels; there is no CPU
fallback, and importing the binding fails loudly when the library has not been built.

Arrays may be numpy arrays (host) or torch tensors (host or CUDA); PyTorch provides device
memory and streams, nothing else.
"""

from __future__ import annotations

import ctypes as C
import os

import numpy as np

__all__ = ["lib", "Context", "Server", "AraError", "ACC_FP64", "ACC_KAHAN32", "LIB_PATH"]

LIB_PATH = os.path.join(os.path.dirname(os.path.abspath(__file__)), "libara.so")
ACC_FP64 = 0
ACC_KAHAN32 = 1
OPT_PRECISION, OPT_SEED, OPT_SURROGATE, OPT_INVERSION = 1, 2, 3, 4
INV_TABLE, INV_NEWTON = 0, 1
OPT_SCHEDULE = 5
OPT_BAND_WIDTH = 6
OPT_TABLES = 7
TABLES_EAGER, TABLES_ON_DEMAND = 0, 1
TABLE_BUY_HITS = 260.0  # expected hits per record at which on-demand tables are built
BAND_BUY_PASSES = 3.0  # YET passes after which ARA_SCHED_AUTO makes the band-major copy
OPT_STREAM_CHUNK = 8
SCHED_BAND, SCHED_TRIAL, SCHED_AUTO = 0, 1, 2
STATUS = {0: "ok", 1: "invalid argument", 2: "bad handle", 3: "out of memory", 4: "CUDA error",
          5: "inversion did not converge", 6: "busy", 7: "no CUDA device"}

_lib = None


class AraError(RuntimeError):
    def __init__(self, status: int, detail: str = ""):
        self.status = status
        super().__init__(f"{STATUS.get(status, status)}: {detail}" if detail else
                         STATUS.get(status, str(status)))


class SurrogateConfig(C.Structure):
    _fields_ = [("n_samples", C.c_int64), ("steps", C.c_int64), ("batch", C.c_int32),
                ("cert_samples", C.c_int32), ("lr", C.c_float), ("lr_final", C.c_float),
                ("eps", C.c_float), ("reserved", C.c_float), ("seed", C.c_uint64)]


class SurrogateReport(C.Structure):
    _fields_ = [("loss_first", C.c_double), ("loss_last", C.c_double), ("gen_ms", C.c_double),
                ("train_ms", C.c_double), ("cert_ms", C.c_double),
                ("cells_accepted", C.c_double), ("err_median", C.c_double),
                ("err_p99", C.c_double), ("bad_targets", C.c_int64)]


MAX_RPS = 16
REQ_PENDING, REQ_RUNNING, REQ_DONE, REQ_FAILED = 0, 1, 2, 3


class ServerConfig(C.Structure):
    _fields_ = [("yet", C.c_int32), ("max_inflight", C.c_int32), ("slice_trials", C.c_int64),
                ("max_batch_trials", C.c_int64), ("max_queue", C.c_int64),
                ("hbm_budget", C.c_int64), ("use_surrogate", C.c_int32),
                ("inversion", C.c_int32)]


class Request(C.Structure):
    _fields_ = [("elts", C.c_int32 * 64), ("n_elts", C.c_int32), ("n_rps", C.c_int32),
                ("occ_ret", C.c_double), ("occ_lim", C.c_double), ("agg_ret", C.c_double),
                ("agg_lim", C.c_double), ("t0", C.c_int64), ("n_trials", C.c_int64),
                ("rps", C.c_double * MAX_RPS)]


class RequestStatus(C.Structure):
    _fields_ = [("state", C.c_int32), ("error", C.c_int32), ("submit_s", C.c_double),
                ("admit_s", C.c_double), ("done_s", C.c_double), ("n_trials", C.c_int64),
                ("pml", C.c_double * MAX_RPS), ("tvar", C.c_double * MAX_RPS)]


class ServerStats(C.Structure):
    _fields_ = [("completed", C.c_int64), ("failed", C.c_int64), ("launches", C.c_int64),
                ("pending", C.c_int64), ("active", C.c_int64),
                ("mean_items_per_launch", C.c_double), ("hbm_budget", C.c_int64),
                ("hbm_used", C.c_int64), ("latency_p50_s", C.c_double),
                ("latency_p99_s", C.c_double), ("latency_max_s", C.c_double),
                ("requests_per_s", C.c_double)]


class _Config(C.Structure):
    _fields_ = [("seed", C.c_uint64), ("precision", C.c_int32), ("use_surrogate", C.c_int32),
                ("device", C.c_int32), ("reserved", C.c_int32)]


_P = C.c_void_p
_I32, _I64, _D = C.c_int32, C.c_int64, C.c_double

_SIGNATURES = {
    "ara_create": ([C.POINTER(_Config), C.POINTER(_P)], C.c_int),
    "ara_destroy": ([_P], None),
    "ara_status_string": ([C.c_int], C.c_char_p),
    "ara_last_error_detail": ([_P, C.c_char_p, C.c_size_t], C.c_int),
    "ara_set_option": ([_P, _I32, _I64], C.c_int),
    "ara_create_yet": ([_P, _I64, _P, _P, _P, _I32, C.POINTER(_I32)], C.c_int),
    "ara_create_yet_host": ([_P, _I64, _P, _P, _P, _I32, C.POINTER(_I32)], C.c_int),
    "ara_free_yet": ([_P, _I32], C.c_int),
    "ara_add_elt": ([_P, _I32, _I64, _P, _P, _P, _P, C.POINTER(_I32)], C.c_int),
    "ara_add_elt_corr": ([_P, _I32, _I64, _P, _P, _P, _P, _P, C.POINTER(_I32)], C.c_int),
    "ara_add_elts": ([_P, _I32, _I32, _P, _P, _P, _P, _P, _P, _P], C.c_int),
    "ara_free_elt": ([_P, _I32], C.c_int),
    "ara_add_layer": ([_P, _P, _I32, _D, _D, _D, _D, C.POINTER(_I32)], C.c_int),
    "ara_free_layer": ([_P, _I32], C.c_int),
    "ara_run": ([_P, _I32, _I32, _I64, _I64, _P, _P], C.c_int),
    "ara_run_ep": ([_P, _I32, _I32, _I64, _I64, _P, _P, _P], C.c_int),
    "ara_run_events": ([_P, _I32, _I32, _I64, _I64, _P, _P, _P, _P, _P], C.c_int),
    "ara_run_portfolio": ([_P, _I32, _P, _I32, _I64, _I64, _P, _P], C.c_int),
    "ara_not_converged": ([_P, C.POINTER(_I64)], C.c_int),
    "ara_risk_measures": ([_P, _P, _I64, _P, _I32, _P, _P], C.c_int),
    "ara_rank_ylt": ([_P, _P, _I64, _P], C.c_int),
    "ara_top_k": ([_P, _P, _I64, _I64, _P], C.c_int),
    "ara_risk_measures_n": ([_P, _P, _I64, _I64, _P, _I32, _P, _P], C.c_int),
    "ara_trace_hits": ([_P, _I32, _I32, _I64, _I64, _I64, _P, _P, _P, _P, _P, _P, _P, _P,
                        C.POINTER(_I64)], C.c_int),
    "ara_synchronize": ([_P], C.c_int),
    "ara_get_stats": ([_P, _P], C.c_int),
    "ara_set_stream": ([_P, _P], C.c_int),
    "ara_train_surrogate": ([_P, C.POINTER(SurrogateConfig), C.POINTER(SurrogateReport)], C.c_int),
    "ara_save_surrogate": ([_P, _P, C.c_size_t, C.POINTER(C.c_size_t)], C.c_int),
    "ara_load_surrogate": ([_P, _P, C.c_size_t], C.c_int),
    "ara_set_surrogate_eps": ([_P, C.c_float], C.c_int),
    "ara_mlp_eval": ([_P, _P, _P, _I64, _P], C.c_int),
    "ara_mlp_grad": ([_P, _P, _P, _P, _P, _I64, _P, C.POINTER(C.c_double)], C.c_int),
    "ara_server_create": ([_P, C.POINTER(ServerConfig), C.POINTER(_P)], C.c_int),
    "ara_server_submit": ([_P, C.POINTER(Request), C.POINTER(_I64)], C.c_int),
    "ara_server_wait": ([_P, _I64, C.c_double], C.c_int),
    "ara_server_result": ([_P, _I64, C.POINTER(RequestStatus), _P, _I64], C.c_int),
    "ara_server_release": ([_P, _I64], C.c_int),
    "ara_server_get_stats": ([_P, C.POINTER(ServerStats)], C.c_int),
    "ara_server_destroy": ([_P], None),
}


def lib():
    """The loaded libara.so.  Raises if it has not been built (no fallback exists)."""
    global _lib
    if _lib is None:
        if not os.path.exists(LIB_PATH):
            raise ImportError(f"libara.so not built at {LIB_PATH}: run "
                              "`python -m paper_1310_2274_b300.build` (nvcc, sm_103a)")
        L = C.CDLL(LIB_PATH)
        for name, (args, res) in _SIGNATURES.items():
            fn = getattr(L, name)
            fn.argtypes = args
            fn.restype = res
        _lib = L
    return _lib


def _ptr(a):
    """Raw address of a numpy array or torch tensor (contiguous)."""
    if a is None:
        return None
    if isinstance(a, np.ndarray):
        assert a.flags.c_contiguous
        return a.ctypes.data
    # torch tensor
    assert a.is_contiguous()
    return a.data_ptr()


def _np(a, dtype):
    if isinstance(a, np.ndarray):
        return np.ascontiguousarray(a, dtype=dtype)
    try:
        import torch

        if isinstance(a, torch.Tensor):
            td = {np.int32: torch.int32, np.int64: torch.int64, np.float32: torch.float32,
                  np.float64: torch.float64}[np.dtype(dtype).type]
            return a.to(td).contiguous()
    except ImportError:
        pass
    return np.ascontiguousarray(a, dtype=dtype)


def _is_cuda(a) -> bool:
    return hasattr(a, "is_cuda") and a.is_cuda


class Context:
    """One ara_ctx: owns the device copies of YETs, ELTs and layers."""

    def __init__(self, seed: int = 42, precision: int = ACC_FP64, device: int = 0,
                 use_surrogate: bool = False):
        cfg = _Config(seed, precision, int(use_surrogate), device, 0)
        h = _P()
        st = lib().ara_create(C.byref(cfg), C.byref(h))
        if st != 0:
            raise AraError(st, "ara_create")
        self._h = h
        self._host_yets = {}  # host-resident YETs: the arrays the library reads, kept alive

    # -- plumbing ------------------------------------------------------------------------------
    @property
    def handle(self):
        return self._h

    def _detail(self) -> str:
        buf = C.create_string_buffer(512)
        lib().ara_last_error_detail(self._h, buf, 512)
        return buf.value.decode(errors="replace")

    def _check(self, st: int, allow_not_converged: bool = False):
        if st == 0 or (allow_not_converged and st == 5):
            return st
        raise AraError(st, self._detail())

    def close(self):
        if getattr(self, "_h", None):
            lib().ara_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.close()

    def set_option(self, option: int, value: int):
        self._check(lib().ara_set_option(self._h, option, int(value)))

    def synchronize(self):
        self._check(lib().ara_synchronize(self._h))

    def stats(self) -> dict:
        """Cumulative work counters of every ara_run on this context."""
        v = np.zeros(9, dtype=np.int64)
        self._check(lib().ara_get_stats(self._h, _ptr(v)))
        return dict(inversions=int(v[0]), newton=int(v[1]), cf_terms=int(v[2]),
                    not_converged=int(v[3]), hits=int(v[4]), launches=int(v[5]),
                    table_evals=int(v[6]), uncertified=int(v[7]), surrogate_evals=int(v[8]))

    def set_stream(self, stream=None):
        """Issue the context's device work on stream (torch.cuda.Stream or cudaStream_t)."""
        s = None if stream is None else getattr(stream, "cuda_stream", stream)
        self._check(lib().ara_set_stream(self._h, s))

    def not_converged(self) -> int:
        v = _I64(0)
        self._check(lib().ara_not_converged(self._h, C.byref(v)))
        return v.value

    # -- staging -------------------------------------------------------------------------------
    def create_yet(self, offsets, event_ids, timestamps, catalog_size: int) -> int:
        off = _np(offsets, np.int64)
        ids = _np(event_ids, np.int32)
        ts = _np(timestamps, np.float32)
        n_trials = int(off.shape[0]) - 1
        out = _I32(-1)
        self._check(lib().ara_create_yet(self._h, n_trials, _ptr(off), _ptr(ids), _ptr(ts),
                                         int(catalog_size), C.byref(out)))
        return out.value

    def add_elt(self, yet: int, event_ids, mean, sd, max_exposure, sd_corr=None) -> int:
        """Stage an ELT; sd is the independent SD sigma_I and sd_corr (optional) the correlated
        SD sigma_C of paper §3.1."""
        ids = _np(event_ids, np.int32)
        mu = _np(mean, np.float64)
        s = _np(sd, np.float64)
        mx = _np(max_exposure, np.float64)
        out = _I32(-1)
        if sd_corr is None:
            self._check(lib().ara_add_elt(self._h, yet, int(ids.shape[0]), _ptr(ids), _ptr(mu),
                                          _ptr(s), _ptr(mx), C.byref(out)))
        else:
            sc = _np(sd_corr, np.float64)
            self._check(lib().ara_add_elt_corr(self._h, yet, int(ids.shape[0]), _ptr(ids),
                                               _ptr(mu), _ptr(s), _ptr(sc), _ptr(mx),
                                               C.byref(out)))
        return out.value

    def add_elts(self, yet: int, elts) -> list:
        """Stage several ELTs at once (one check for all of them; all or none are added).  elts:
        a sequence of (event_ids, mean, sd, max_exposure) or (..., sd_corr) tuples."""
        arrs = []
        for e in elts:
            ids, mu, s, mx = (_np(e[0], np.int32), _np(e[1], np.float64), _np(e[2], np.float64),
                              _np(e[3], np.float64))
            sc = _np(e[4], np.float64) if len(e) > 4 and e[4] is not None else None
            arrs.append((ids, mu, s, mx, sc))
        k = len(arrs)
        n = np.array([int(a[0].shape[0]) for a in arrs], dtype=np.int64)
        col = lambda i: (C.c_void_p * max(k, 1))(*[_ptr(a[i]) for a in arrs])  # noqa: E731
        out = np.full(max(k, 1), -1, dtype=np.int32)
        self._check(lib().ara_add_elts(self._h, yet, k, _ptr(n), col(0), col(1), col(2), col(4),
                                       col(3), _ptr(out)))
        return [int(v) for v in out[:k]]

    def add_layer(self, elts, occ_ret: float, occ_lim: float, agg_ret: float,
                  agg_lim: float) -> int:
        e = np.ascontiguousarray(elts, dtype=np.int32)
        out = _I32(-1)
        self._check(lib().ara_add_layer(self._h, _ptr(e), int(e.shape[0]), occ_ret, occ_lim,
                                        agg_ret, agg_lim, C.byref(out)))
        return out.value

    def create_yet_host(self, offsets, event_ids, timestamps, catalog_size: int) -> int:
        """A YET whose ids and timestamps stay in host memory and are streamed by each run (one
        pass per staging); the arrays (page-locked for copy/compute overlap, e.g. a pinned
        torch tensor's numpy view) are referenced, not copied, until free_yet."""
        off = _np(offsets, np.int64)
        ids = _np(event_ids, np.int32)
        ts = _np(timestamps, np.float32)
        n_trials = int(off.shape[0]) - 1
        out = _I32(-1)
        self._check(lib().ara_create_yet_host(self._h, n_trials, _ptr(off), _ptr(ids), _ptr(ts),
                                              int(catalog_size), C.byref(out)))
        self._host_yets[out.value] = (off, ids, ts)
        return out.value

    def free_yet(self, yet: int):
        self._check(lib().ara_free_yet(self._h, yet))
        self._host_yets.pop(yet, None)

    def free_elt(self, elt: int):
        self._check(lib().ara_free_elt(self._h, elt))

    def free_layer(self, layer: int):
        self._check(lib().ara_free_layer(self._h, layer))

    # -- Algorithm 1 ---------------------------------------------------------------------------
    def run(self, yet: int, layer: int, t0: int, n: int, out=None, stream=None,
            allow_not_converged: bool = False):
        """Year losses of trials [t0, t0+n).  out: float64 numpy array or torch tensor (host or
        CUDA); stream: a torch.cuda.Stream or raw cudaStream_t (asynchronous, CUDA out only)."""
        if out is None:
            out = np.zeros(n, dtype=np.float64)
        s = None
        if stream is not None:
            s = getattr(stream, "cuda_stream", stream)
        st = lib().ara_run(self._h, yet, layer, int(t0), int(n), _ptr(out), s)
        self._check(st, allow_not_converged)
        return out

    def run_ep(self, yet: int, layer: int, t0: int, n: int, out=None, oep=None, stream=None,
               allow_not_converged: bool = False):
        """Year losses (AEP year table) and each year's largest occurrence loss (OEP year table)
        of trials [t0, t0+n) from one pass -> (ylt, oep); out and oep both host or both CUDA."""
        if out is None:
            out = np.zeros(n, dtype=np.float64)
        if oep is None and _is_cuda(out):
            import torch
            oep = torch.zeros(n, dtype=torch.float64, device=out.device)
        elif oep is None:
            oep = np.zeros(n, dtype=np.float64)
        s = None
        if stream is not None:
            s = getattr(stream, "cuda_stream", stream)
        st = lib().ara_run_ep(self._h, yet, layer, int(t0), int(n), _ptr(out), _ptr(oep), s)
        self._check(st, allow_not_converged)
        return out, oep

    def run_portfolio(self, yet: int, layers, t0: int, n: int, out=None, stream=None,
                      allow_not_converged: bool = False):
        """YLTs of several layers (a portfolio's programs' layers, flattened) over trials
        [t0, t0+n) -> float64 [len(layers), n]; out: numpy array or CUDA tensor of that shape."""
        ls = np.ascontiguousarray(layers, dtype=np.int32)
        if out is None:
            out = np.zeros((ls.shape[0], n), dtype=np.float64)
        s = None if stream is None else getattr(stream, "cuda_stream", stream)
        st = lib().ara_run_portfolio(self._h, yet, _ptr(ls), int(ls.shape[0]), int(t0), int(n),
                                     _ptr(out), s)
        self._check(st, allow_not_converged)
        return out

    def run_events(self, yet: int, layer: int, t0: int, n: int, n_occ: int, device=False,
                   increments: bool = True, out=None, stream=None,
                   allow_not_converged: bool = False):
        """Year losses, OEP year table and the per-occurrence outputs of trials [t0, t0+n), whose
        occurrences number n_occ -> (ylt, oep, olt float32, inc float64 or None).  device=True
        returns CUDA tensors, else numpy arrays; out = (ylt, oep, olt, inc) reuses caller buffers
        (inc may be None); stream (CUDA outputs only) makes the call asynchronous."""
        if out is None:
            if device:
                import torch
                mk = lambda m, dt: torch.zeros(m, dtype=dt, device="cuda")  # noqa: E731
                f64, f32 = torch.float64, torch.float32
            else:
                mk = lambda m, dt: np.zeros(m, dtype=dt)  # noqa: E731
                f64, f32 = np.float64, np.float32
            out = (mk(n, f64), mk(n, f64), mk(max(n_occ, 1), f32),
                   mk(max(n_occ, 1), f64) if increments else None)
        ylt, oep, olt, inc = out
        s = None if stream is None else getattr(stream, "cuda_stream", stream)
        st = lib().ara_run_events(self._h, yet, layer, int(t0), int(n), _ptr(ylt), _ptr(oep),
                                  _ptr(olt), _ptr(inc) if inc is not None else None, s)
        self._check(st, allow_not_converged)
        return ylt, oep, olt[:n_occ], (inc[:n_occ] if inc is not None else None)

    # -- risk measures -------------------------------------------------------------------------
    def risk_measures(self, ylt, rps):
        y = ylt if _is_cuda(ylt) else _np(ylt, np.float64)
        r = np.ascontiguousarray(rps, dtype=np.float64)
        pml = np.zeros(r.shape[0])
        tvar = np.zeros(r.shape[0])
        self._check(lib().ara_risk_measures(self._h, _ptr(y), int(y.shape[0]), _ptr(r),
                                            int(r.shape[0]), _ptr(pml), _ptr(tvar)))
        return pml, tvar

    def risk_measures_n(self, values, n_total, rps):
        """PML/TVaR over candidate values with the tail counts of n_total trials."""
        y = values if _is_cuda(values) else _np(values, np.float64)
        r = np.ascontiguousarray(rps, dtype=np.float64)
        pml = np.zeros(r.shape[0])
        tvar = np.zeros(r.shape[0])
        self._check(lib().ara_risk_measures_n(self._h, _ptr(y), int(y.shape[0]), int(n_total),
                                              _ptr(r), int(r.shape[0]), _ptr(pml), _ptr(tvar)))
        return pml, tvar

    def top_k(self, ylt, k, out=None):
        """The k largest year losses (ties: lower index first) in ascending trial order."""
        y = ylt if _is_cuda(ylt) else _np(ylt, np.float64)
        if out is None:
            if _is_cuda(y):
                import torch

                out = torch.empty(int(k), dtype=torch.float64, device=y.device)
            else:
                out = np.zeros(int(k), dtype=np.float64)
        self._check(lib().ara_top_k(self._h, _ptr(y), int(y.shape[0]), int(k), _ptr(out)))
        return out

    def rank(self, ylt, out=None):
        y = ylt if _is_cuda(ylt) else _np(ylt, np.float64)
        if out is None:
            out = np.zeros(int(y.shape[0]), dtype=np.int64)
        self._check(lib().ara_rank_ylt(self._h, _ptr(y), int(y.shape[0]), _ptr(out)))
        return out

    def trace(self, yet: int, layer: int, t0: int, n: int, max_hits: int = 1 << 22):
        bufs = dict(trial=np.zeros(max_hits, np.int32), k=np.zeros(max_hits, np.int32),
                    j=np.zeros(max_hits, np.int32), rec=np.zeros(max_hits, np.int32),
                    u=np.zeros(max_hits, np.float32), x=np.zeros(max_hits, np.float32),
                    loss=np.zeros(max_hits, np.float32))
        ylt = np.zeros(n, dtype=np.float64)
        nh = _I64(0)
        self._check(lib().ara_trace_hits(
            self._h, yet, layer, int(t0), int(n), int(max_hits), _ptr(bufs["trial"]),
            _ptr(bufs["k"]), _ptr(bufs["j"]), _ptr(bufs["rec"]), _ptr(bufs["u"]),
            _ptr(bufs["x"]), _ptr(bufs["loss"]), _ptr(ylt), C.byref(nh)))
        m = min(nh.value, max_hits)
        return {k: v[:m] for k, v in bufs.items()}, ylt

    # -- learned surrogate ---------------------------------------------------------------------
    def train_surrogate(self, n_samples=50_000_000, steps=30_000, batch=8192, lr=3e-3,
                        lr_final=3e-5, eps=5e-4, cert_samples=16, seed=3) -> dict:
        cfg = SurrogateConfig(int(n_samples), int(steps), int(batch), int(cert_samples),
                              float(lr), float(lr_final), float(eps), 0.0, int(seed))
        rep = SurrogateReport()
        self._check(lib().ara_train_surrogate(self._h, C.byref(cfg), C.byref(rep)))
        return {f: getattr(rep, f) for f, _ in SurrogateReport._fields_}

    def save_surrogate(self) -> bytes:
        need = C.c_size_t(0)
        self._check(lib().ara_save_surrogate(self._h, None, 0, C.byref(need)))
        buf = C.create_string_buffer(need.value)
        self._check(lib().ara_save_surrogate(self._h, buf, need.value, C.byref(need)))
        return buf.raw

    def load_surrogate(self, blob: bytes):
        self._check(lib().ara_load_surrogate(self._h, blob, len(blob)))

    def set_surrogate_eps(self, eps: float):
        self._check(lib().ara_set_surrogate_eps(self._h, float(eps)))

    def mlp_eval(self, z, params=None):
        z = np.ascontiguousarray(z, dtype=np.float32)
        p = None if params is None else np.ascontiguousarray(params, dtype=np.float32)
        y = np.zeros(z.shape[0], dtype=np.float32)
        self._check(lib().ara_mlp_eval(self._h, _ptr(p), _ptr(z), z.shape[0], _ptr(y)))
        return y

    def mlp_grad(self, params, z, x, t):
        p = np.ascontiguousarray(params, dtype=np.float32)
        z = np.ascontiguousarray(z, dtype=np.float32)
        x = np.ascontiguousarray(x, dtype=np.float32)
        t = np.ascontiguousarray(t, dtype=np.float32)
        g = np.zeros(p.shape[0], dtype=np.float32)
        loss = C.c_double(0)
        self._check(lib().ara_mlp_grad(self._h, _ptr(p), _ptr(z), _ptr(x), _ptr(t), z.shape[0],
                                       _ptr(g), C.byref(loss)))
        return loss.value, g

    # -- convenience for synthetic workloads ---------------------------------------------------
    def stage_workload(self, w):
        """Stage a synth.Workload: returns (yet, [elt handles], layer)."""
        yet = self.create_yet(w.yet.offsets, w.yet.event_ids, w.yet.timestamps,
                              w.yet.catalog_size)
        elts = [self.add_elt(yet, e.event_ids, e.mean, e.sd, e.max_exposure,
                             getattr(e, "sd_corr", None)) for e in w.elts]
        t = w.terms
        layer = self.add_layer(elts, t.occ_ret, t.occ_lim, t.agg_ret, t.agg_lim)
        return yet, elts, layer


class Server:
    """Continuous-batching service over one context and one staged YET (ara_server_*).

    While a Server exists its context is driven only through it."""

    def __init__(self, ctx: Context, yet: int, max_inflight: int = 32,
                 slice_trials: int = 65536, max_batch_trials: int = 1 << 20,
                 max_queue: int = 1 << 16, hbm_budget: int = 0, use_surrogate: bool = False,
                 inversion: int = INV_TABLE):
        cfg = ServerConfig(yet, max_inflight, slice_trials, max_batch_trials, max_queue,
                           hbm_budget, int(use_surrogate), inversion)
        h = _P()
        st = lib().ara_server_create(ctx.handle, C.byref(cfg), C.byref(h))
        if st != 0:
            raise AraError(st, "ara_server_create")
        self._h = h
        self._ctx = ctx

    def submit(self, elts, occ_ret, occ_lim, agg_ret, agg_lim, t0, n_trials, rps=()) -> int:
        r = Request()
        elts = list(elts)
        rps = list(rps)
        if len(elts) > 64 or len(rps) > MAX_RPS:
            raise AraError(1, "too many ELTs or return periods")
        for i, e in enumerate(elts):
            r.elts[i] = int(e)
        for i, v in enumerate(rps):
            r.rps[i] = float(v)
        r.n_elts, r.n_rps = len(elts), len(rps)
        r.occ_ret, r.occ_lim, r.agg_ret, r.agg_lim = occ_ret, occ_lim, agg_ret, agg_lim
        r.t0, r.n_trials = int(t0), int(n_trials)
        tk = _I64(0)
        st = lib().ara_server_submit(self._h, C.byref(r), C.byref(tk))
        if st != 0:
            raise AraError(st, "ara_server_submit")
        return tk.value

    def wait(self, ticket: int, timeout: float = 60.0) -> int:
        """Status of the wait: 0 done, 6 timed out, else the failed request's status."""
        return lib().ara_server_wait(self._h, ticket, timeout)

    def result(self, ticket: int, ylt: bool = True) -> dict:
        s = RequestStatus()
        st = lib().ara_server_result(self._h, ticket, C.byref(s), None, 0)
        if st != 0:
            raise AraError(st, "ara_server_result")
        out = dict(state=s.state, error=s.error, submit_s=s.submit_s, admit_s=s.admit_s,
                   done_s=s.done_s, n_trials=s.n_trials, pml=np.array(s.pml[:]),
                   tvar=np.array(s.tvar[:]))
        if ylt and s.state == REQ_DONE:
            y = np.empty(s.n_trials, dtype=np.float64)
            st = lib().ara_server_result(self._h, ticket, C.byref(s), _ptr(y), y.shape[0])
            if st != 0:
                raise AraError(st, "ara_server_result")
            out["ylt"] = y
        return out

    def release(self, ticket: int):
        st = lib().ara_server_release(self._h, ticket)
        if st != 0:
            raise AraError(st, "ara_server_release")

    def stats(self) -> dict:
        s = ServerStats()
        st = lib().ara_server_get_stats(self._h, C.byref(s))
        if st != 0:
            raise AraError(st, "ara_server_get_stats")
        return {name: getattr(s, name) for name, _ in ServerStats._fields_}

    def close(self):
        if getattr(self, "_h", None):
            lib().ara_server_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.close()
