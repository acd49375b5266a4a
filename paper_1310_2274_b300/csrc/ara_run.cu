// ara_run.cu -- runs of Algorithm 1 through the C ABI: argument checks, the table policy,
// launch parameters, resident and streamed runs, event-level outputs, portfolios, counters,
// and the verification trace.
#include <cuda_runtime.h>
#include <math.h>
#include <string.h>

#include <algorithm>
#include <cmath>
#include <thread>
#include <vector>

#include "../../include/ara.h"
#include "ara_ctx.h"
#include "ara_host.h"
#include "ara_internal.h"
#include "ara_philox.cuh"

using namespace ara;

// ---- run ------------------------------------------------------------------------------------
static ara_status check_run_args(ara_ctx* ctx, int32_t yet, int32_t layer, int64_t t0, int64_t n) {
  if (yet < 0 || yet >= (int32_t)ctx->yets.size() || !ctx->yets[yet].live)
    return fail(ctx, ARA_ERR_BAD_HANDLE, "bad YET handle %d", yet);
  if (layer < 0 || layer >= (int32_t)ctx->layers.size() || !ctx->layers[layer].live)
    return fail(ctx, ARA_ERR_BAD_HANDLE, "bad layer handle %d", layer);
  const LayerDev& L = ctx->layers[layer];
  if (L.yet != yet) return fail(ctx, ARA_ERR_INVALID_ARG, "layer belongs to another YET");
  for (int j = 0; j < L.n_slots; ++j)
    if (!ctx->elts[L.handles[j]].live)
      return fail(ctx, ARA_ERR_BAD_HANDLE, "layer uses freed ELT %d", L.handles[j]);
  if (t0 < 0 || n < 0 || t0 + n > ctx->yets[yet].n_trials)
    return fail(ctx, ARA_ERR_INVALID_ARG, "trial range [%lld, %lld) outside the YET",
                (long long)t0, (long long)(t0 + n));
  return ARA_OK;
}

bool uses_band_schedule(const ara_ctx* ctx, const LayerDev& L) {
  return layer_inversion(ctx, L) == 0 && ctx->schedule != ARA_SCHED_TRIAL && L.band_log2w > 0 &&
         ctx->cfg.precision == ARA_ACC_FP64;
}

// A single-layer run takes the band schedule for the Newton-Halley inversion too, where the YET's
// band-major copy exists already (made for the table inversion: a Newton pass alone gains ~1 ms
// from it, far less than the copy costs).
static bool run_band_schedule(const ara_ctx* ctx, const LayerDev& L) {
  return layer_inversion(ctx, L) <= 1 && ctx->schedule != ARA_SCHED_TRIAL && L.band_log2w > 0 &&
         ctx->cfg.precision == ARA_ACC_FP64;
}

int layer_inversion(const ara_ctx* ctx, const LayerDev& L) {
  const int m = inversion_mode(ctx);
  return (m == 0 && L.tables == nullptr) ? 1 : m;
}

// A live layer whose in-place tables cover ELT h (its slot in *slot), or null.
static const LayerDev* layer_holding_tables(const ara_ctx* ctx, int32_t h, int* slot) {
  for (const auto& l : ctx->layers) {
    if (!l.live || !l.own_tables || !l.tables) continue;
    for (int j = 0; j < l.n_slots; ++j)
      if (l.handles[j] == h) {
        *slot = j;
        return &l;
      }
  }
  return nullptr;
}

static bool tables_available(const ara_ctx* ctx, int32_t h) {
  int slot;
  return ctx->elts[h].tables != nullptr || layer_holding_tables(ctx, h, &slot) != nullptr;
}

// The certified tables of the ELTs `handles` that lack them, built together (kMaxTableJobs ELTs
// per launch, one synchronisation at the end).
static ara_status ensure_tables(ara_ctx* ctx, const int32_t* handles, int n_handles) {
  std::vector<int32_t> todo;
  for (int j = 0; j < n_handles; ++j) {
    const int32_t h = handles[j];
    if (!ctx->elts[h].tables && std::find(todo.begin(), todo.end(), h) == todo.end())
      todo.push_back(h);
  }
  if (todo.empty()) return ARA_OK;
  // an ELT whose records a live layer holds tables for (built in place) takes a copy of them
  std::vector<int32_t> rest;
  for (int32_t h : todo) {
    int slot = -1;
    const LayerDev* src = layer_holding_tables(ctx, h, &slot);
    if (!src) {
      rest.push_back(h);
      continue;
    }
    EltDev& e = ctx->elts[h];
    unsigned long long uncert = 0;
    cudaError_t err = obj_alloc(ctx, &e.tables, e.n * kTablePieces);
    if (err == cudaSuccess) err = ensure_scratch(ctx, scratch_bytes<unsigned long long>(1));
    unsigned long long* d_uncert = reinterpret_cast<unsigned long long*>(ctx->d_scratch);
    if (err == cudaSuccess) err = cudaMemsetAsync(d_uncert, 0, sizeof uncert, ctx->stream);
    if (err == cudaSuccess)
      err = launch_unpack_tables(e.n, e.ids, slot, src->mask_words, src->evt, src->tables,
                                 e.tables, d_uncert, ctx->stream);
    if (err == cudaSuccess)
      err = cudaMemcpyAsync(&uncert, d_uncert, sizeof uncert, cudaMemcpyDeviceToHost,
                            ctx->stream);
    if (err == cudaSuccess) err = cudaStreamSynchronize(ctx->stream);
    if (err != cudaSuccess) {
      cudaGetLastError();
      cudaStreamSynchronize(ctx->stream);
      obj_free(ctx, e.tables);
      e.tables = nullptr;
      return fail(ctx, err == cudaErrorMemoryAllocation ? ARA_ERR_OOM : ARA_ERR_CUDA,
                  "tables from a layer: %s", cudaGetErrorString(err));
    }
    e.n_uncertified = (int64_t)uncert;
  }
  todo.swap(rest);
  if (todo.empty()) return ARA_OK;
  const int n = (int)todo.size();
  std::vector<unsigned long long> uncert(n, 0ull);
  cudaError_t err = ensure_scratch(ctx, scratch_bytes<unsigned long long>(n));
  for (int j = 0; j < n && err == cudaSuccess; ++j) {
    EltDev& e = ctx->elts[todo[j]];
    err = obj_alloc(ctx, &e.tables, e.n * kTablePieces);
  }
  auto undo = [&]() {
    cudaGetLastError();
    cudaStreamSynchronize(ctx->stream);
    for (int32_t h : todo) {
      obj_free(ctx, ctx->elts[h].tables);
      ctx->elts[h].tables = nullptr;
    }
  };
  if (err != cudaSuccess) {
    undo();
    return fail(ctx, ARA_ERR_OOM, "tables of %d ELTs: %s", n, cudaGetErrorString(err));
  }
  unsigned long long* d_uncert = reinterpret_cast<unsigned long long*>(ctx->d_scratch);
  err = cudaMemsetAsync(d_uncert, 0, sizeof(unsigned long long) * (size_t)n, ctx->stream);
  for (int b = 0; b < n && err == cudaSuccess; b += kMaxTableJobs) {
    TableJobs jobs{};
    jobs.n = std::min(kMaxTableJobs, n - b);
    for (int j = 0; j < jobs.n; ++j) {
      const EltDev& e = ctx->elts[todo[b + j]];
      jobs.recs[j] = e.recs;
      jobs.tables[j] = e.tables;
      jobs.first[j + 1] = jobs.first[j] + e.n;
    }
    err = launch_build_tables(jobs, d_uncert + b, ctx->stream);
  }
  if (err == cudaSuccess)
    err = cudaMemcpyAsync(uncert.data(), d_uncert, sizeof(unsigned long long) * (size_t)n,
                          cudaMemcpyDeviceToHost, ctx->stream);
  if (err == cudaSuccess) err = cudaStreamSynchronize(ctx->stream);
  if (err != cudaSuccess) {
    undo();
    return fail(ctx, ARA_ERR_CUDA, "building tables: %s", cudaGetErrorString(err));
  }
  for (int j = 0; j < n; ++j) ctx->elts[todo[j]].n_uncertified = (int64_t)uncert[j];
  return ARA_OK;
}

// The start tables of the ELTs `handles` that lack them (stream-ordered on the context's stream).
static ara_status ensure_starts(ara_ctx* ctx, const int32_t* handles, int n_handles) {
  for (int j = 0; j < n_handles; ++j) {
    EltDev& e = ctx->elts[handles[j]];
    if (e.starts) continue;
    cudaError_t err = obj_alloc(ctx, &e.starts, e.n * kStartFloats);
    if (err == cudaSuccess) err = launch_build_starts(e.n, e.recs, e.starts, ctx->stream);
    if (err != cudaSuccess) {
      cudaGetLastError();
      cudaStreamSynchronize(ctx->stream);
      obj_free(ctx, e.starts);
      e.starts = nullptr;
      return fail(ctx, err == cudaErrorMemoryAllocation ? ARA_ERR_OOM : ARA_ERR_CUDA,
                  "start tables: %s", cudaGetErrorString(err));
    }
  }
  return ARA_OK;
}

// A layer's tables built straight into its packed order from its packed records (none of its
// ELTs has tables yet): the ELTs' own copies and the gather are skipped; their rent-or-buy goes
// on for other layers.
static ara_status build_layer_tables(ara_ctx* ctx, LayerDev& L) {
  unsigned long long uncert = 0;
  cudaError_t err = obj_alloc(ctx, &L.tables, L.n_packed * kTablePieces);
  if (err == cudaSuccess) err = ensure_scratch(ctx, scratch_bytes<unsigned long long>(1));
  if (err != cudaSuccess) {
    cudaGetLastError();
    obj_free(ctx, L.tables);
    L.tables = nullptr;
    return fail(ctx, ARA_ERR_OOM, "layer tables: %s", cudaGetErrorString(err));
  }
  unsigned long long* d_uncert = reinterpret_cast<unsigned long long*>(ctx->d_scratch);
  TableJobs jobs{};
  jobs.n = 1;
  jobs.recs[0] = L.packed;
  jobs.tables[0] = L.tables;
  jobs.first[1] = L.n_packed;
  err = cudaMemsetAsync(d_uncert, 0, sizeof uncert, ctx->stream);
  if (err == cudaSuccess) err = launch_build_tables(jobs, d_uncert, ctx->stream);
  if (err == cudaSuccess)
    err = cudaMemcpyAsync(&uncert, d_uncert, sizeof uncert, cudaMemcpyDeviceToHost, ctx->stream);
  if (err == cudaSuccess) err = cudaStreamSynchronize(ctx->stream);
  if (err != cudaSuccess) {
    cudaGetLastError();
    cudaStreamSynchronize(ctx->stream);
    obj_free(ctx, L.tables);
    L.tables = nullptr;
    return fail(ctx, ARA_ERR_CUDA, "building layer tables: %s", cudaGetErrorString(err));
  }
  L.n_uncertified = (int64_t)uncert;
  L.own_tables = true;
  return ARA_OK;
}

// The layer's packed table copy: built in place when none of its ELTs has tables, else gathered
// from theirs (those missing built first).
static ara_status ensure_layer_tables(ara_ctx* ctx, LayerDev& L) {
  if (L.tables) return ARA_OK;
  bool none = true;
  for (int j = 0; j < L.n_slots; ++j) none = none && !tables_available(ctx, L.handles[j]);
  if (none) return build_layer_tables(ctx, L);
  const ara_status s = ensure_tables(ctx, L.handles, L.n_slots);
  if (s != ARA_OK) return s;
  const TablePiece** d_src = nullptr;  // staging scratch
  cudaError_t err;
  if ((err = obj_alloc(ctx, &L.tables, L.n_packed * kTablePieces)) != cudaSuccess ||
      (err = ensure_scratch(ctx, scratch_bytes<const TablePiece*>(L.n_packed))) != cudaSuccess) {
    cudaGetLastError();
    obj_free(ctx, L.tables);
    L.tables = nullptr;
    return fail(ctx, ARA_ERR_OOM, "layer tables: %s", cudaGetErrorString(err));
  }
  d_src = reinterpret_cast<const TablePiece**>(ctx->d_scratch);
  // the scatter rewrites the packed records as they are and fills the table source pointers
  err = cudaSuccess;
  for (int j = 0; j < L.n_slots && err == cudaSuccess; ++j)
    err = launch_layer_scatter(ctx->elts[L.handles[j]], j, L.mask_words, L.evt, L.packed, d_src,
                               L.packed_rec, L.corr, nullptr, ctx->stream);
  if (err == cudaSuccess) err = launch_gather_tables(L.n_packed, d_src, L.tables, ctx->stream);
  if (err == cudaSuccess) err = cudaStreamSynchronize(ctx->stream);
  if (err != cudaSuccess) {
    cudaGetLastError();
    cudaStreamSynchronize(ctx->stream);
    obj_free(ctx, L.tables);
    L.tables = nullptr;
    return fail(ctx, ARA_ERR_CUDA, "layer tables: %s", cudaGetErrorString(err));
  }
  return ARA_OK;
}

// The layer's packed start tables (its ELTs' own, built first if missing), for runs that invert
// by Newton-Halley steps.
static ara_status ensure_layer_starts(ara_ctx* ctx, LayerDev& L) {
  if (L.starts) return ARA_OK;
  const ara_status s = ensure_starts(ctx, L.handles, L.n_slots);
  if (s != ARA_OK) return s;
  cudaError_t err;
  if ((err = obj_alloc(ctx, &L.starts, L.n_packed * kStartFloats)) != cudaSuccess ||
      (err = ensure_scratch(ctx, scratch_bytes<const TablePiece*>(L.n_packed) +
                                     scratch_bytes<const float*>(L.n_packed))) != cudaSuccess) {
    cudaGetLastError();
    obj_free(ctx, L.starts);
    L.starts = nullptr;
    return fail(ctx, ARA_ERR_OOM, "layer start tables: %s", cudaGetErrorString(err));
  }
  // staging scratch: the table and start-table source of each packed record
  ScratchCarver sc{ctx->d_scratch};
  const TablePiece** d_src = sc.take<const TablePiece*>(L.n_packed);
  const float** d_ssrc = sc.take<const float*>(L.n_packed);
  err = cudaSuccess;
  for (int j = 0; j < L.n_slots && err == cudaSuccess; ++j)
    err = launch_layer_scatter(ctx->elts[L.handles[j]], j, L.mask_words, L.evt, L.packed, d_src,
                               L.packed_rec, L.corr, d_ssrc, ctx->stream);
  if (err == cudaSuccess) err = launch_gather_starts(L.n_packed, d_ssrc, L.starts, ctx->stream);
  if (err == cudaSuccess) err = cudaStreamSynchronize(ctx->stream);
  if (err != cudaSuccess) {
    cudaGetLastError();
    cudaStreamSynchronize(ctx->stream);
    obj_free(ctx, L.starts);
    L.starts = nullptr;
    return fail(ctx, ARA_ERR_CUDA, "layer start tables: %s", cudaGetErrorString(err));
  }
  return ARA_OK;
}

static ara_status rent_or_buy(ara_ctx* ctx, LayerDev& L, int64_t n);

ara_status prepare_layer_for_run(ara_ctx* ctx, LayerDev& L, int64_t n, bool band_ok) {
  ara_status s = rent_or_buy(ctx, L, n);
  if (s != ARA_OK) return s;
  if (band_ok && L.band_want > 0 && L.band_log2w == 0 && layer_inversion(ctx, L) == 0 &&
      ctx->schedule != ARA_SCHED_TRIAL && ctx->cfg.precision == ARA_ACC_FP64) {
    // under ARA_SCHED_AUTO the copy is bought once the YET's trial-major table runs plus this
    // one cover ARA_BAND_BUY_PASSES times its occurrences; until then this run rents
    YetDev& Y = ctx->yets[L.yet];
    const double occ =
        Y.n_trials > 0 ? (double)Y.n_occ * ((double)n / (double)Y.n_trials) : 0.0;
    if (ctx->schedule == ARA_SCHED_AUTO &&
        Y.band_rent_occ + occ < ARA_BAND_BUY_PASSES * (double)Y.n_occ) {
      Y.band_rent_occ += occ;
    } else {
      bool banded = false;
      s = ensure_band_variant(ctx, L.yet, L.band_want, &banded);
      if (s != ARA_OK) return s;
      if (banded) L.band_log2w = L.band_want;
      L.band_want = 0;
    }
  }
  // Newton-Halley runs and the surrogate's fallbacks start from the layer's start tables
  return layer_inversion(ctx, L) >= 1 ? ensure_layer_starts(ctx, L) : ARA_OK;
}

static ara_status rent_or_buy(ara_ctx* ctx, LayerDev& L, int64_t n) {
  if (L.tables || inversion_mode(ctx) != 0) return ARA_OK;
  if (ctx->table_policy == ARA_TABLES_EAGER) return ensure_layer_tables(ctx, L);
  const YetDev& Y = ctx->yets[L.yet];
  // expected hits per record of this run: each occurrence meets a given record with
  // probability 1 / catalogue
  const double per_rec = Y.n_trials > 0 && Y.catalog > 0
                             ? (double)Y.n_occ * ((double)n / (double)Y.n_trials) / Y.catalog
                             : 0.0;
  bool buy = true;
  for (int j = 0; j < L.n_slots; ++j) {
    const EltDev& e = ctx->elts[L.handles[j]];
    if (!tables_available(ctx, L.handles[j]) && e.rent_hits + per_rec < ARA_TABLE_BUY_HITS)
      buy = false;
  }
  if (buy) return ensure_layer_tables(ctx, L);
  for (int j = 0; j < L.n_slots; ++j) {
    EltDev& e = ctx->elts[L.handles[j]];
    if (!e.tables) e.rent_hits += per_rec;
  }
  return ARA_OK;
}

static std::vector<int32_t> live_elts_of(const ara_ctx* ctx, int32_t yet) {
  std::vector<int32_t> hs;
  for (int32_t h = 0; h < (int32_t)ctx->elts.size(); ++h)
    if (ctx->elts[h].live && ctx->elts[h].yet == yet) hs.push_back(h);
  return hs;
}

ara_status ensure_yet_tables(ara_ctx* ctx, int32_t yet) {
  const std::vector<int32_t> hs = live_elts_of(ctx, yet);
  return ensure_tables(ctx, hs.data(), (int)hs.size());
}

ara_status ensure_yet_starts(ara_ctx* ctx, int32_t yet) {
  const std::vector<int32_t> hs = live_elts_of(ctx, yet);
  const ara_status s = ensure_starts(ctx, hs.data(), (int)hs.size());
  if (s != ARA_OK) return s;
  CUDA_TRY(ctx, cudaStreamSynchronize(ctx->stream));
  return ARA_OK;
}

ara_status ensure_band_variant(ara_ctx* ctx, int32_t yet, int log2w, bool* available) {
  *available = false;
  YetDev& Y = ctx->yets[yet];
  if (Y.host) return ARA_OK;  // a streamed YET runs trial-major
  if (!band_layout_fits(Y, log2w)) return ARA_OK;
  for (int v = 0; v < kMaxBandVariants; ++v)
    if (Y.bands[v].log2w == log2w) {
      *available = true;
      return ARA_OK;
    }
  for (int v = 0; v < kMaxBandVariants; ++v)
    if (Y.bands[v].log2w == 0) {
      const cudaError_t err = build_band_variant(Y, log2w, Y.bands[v], ctx->stream);
      if (err != cudaSuccess) {
        cudaGetLastError();
        return fail(ctx, err == cudaErrorMemoryAllocation ? ARA_ERR_OOM : ARA_ERR_CUDA,
                    "band-major YET copy: %s", cudaGetErrorString(err));
      }
      *available = true;
      return ARA_OK;
    }
  return ARA_OK;  // every slot taken: the layer runs trial-major
}

int inversion_mode(const ara_ctx* ctx) {
  if (ctx->cfg.use_surrogate && ctx->mlp_ready) return 2;
  return ctx->inversion;
}

// The end of a run call: nothing more for an asynchronous call; else the YLT back to a host
// buffer, and ARA_ERR_NOT_CONVERGED if the convergence counter moved during the call.
static ara_status finish_run(ara_ctx* ctx, void* stream, bool dev_out, double* ylt,
                             const double* d_ylt, int64_t total, unsigned long long nc_before,
                             cudaStream_t st) {
  if (stream) return ARA_OK;
  if (!dev_out)
    CUDA_TRY(ctx, cudaMemcpyAsync(ylt, d_ylt, sizeof(double) * (size_t)total,
                                  cudaMemcpyDeviceToHost, st));
  unsigned long long nc_after = 0;
  CUDA_TRY(ctx, cudaMemcpyAsync(&nc_after, ctx->d_not_conv, sizeof nc_after,
                                cudaMemcpyDeviceToHost, st));
  CUDA_TRY(ctx, cudaStreamSynchronize(st));
  if (nc_after != nc_before)
    return fail(ctx, ARA_ERR_NOT_CONVERGED, "%llu inversions hit the iteration cap",
                nc_after - nc_before);
  return ARA_OK;
}

// Where the net aggregate loss A(s) = min(max(s*unit - AggR, 0), AggL) (binary64, s grid units,
// s*unit exact) is constant: A = 0 for s <= *zero_max, A = AggL for s >= *full_min.  Both by
// bisection on the same binary64 expression the kernels evaluate, which is monotone in s.
static void agg_bounds(double unit, double agg_ret, double agg_lim, unsigned long long* zero_max,
                       unsigned long long* full_min) {
  const unsigned long long top = 1ull << 63;  // year sums stay below 2^62 + max_len / 2 units
  auto net = [&](unsigned long long s) { return (double)s * unit - agg_ret; };
  // largest s in [0, top] with net(s) <= 0 (net(0) <= 0 always)
  unsigned long long lo = 0, hi = top;
  if (net(top) <= 0.0) {
    lo = top;
  } else {
    while (hi - lo > 1) {
      const unsigned long long mid = lo + (hi - lo) / 2;
      if (net(mid) <= 0.0) lo = mid; else hi = mid;
    }
  }
  *zero_max = lo;
  // smallest s in [0, top] with net(s) >= AggL, or never
  if (!(net(top) >= agg_lim)) {
    *full_min = ~0ull;
    return;
  }
  lo = 0;
  hi = top;
  if (net(0) >= agg_lim) {
    *full_min = 0;
    return;
  }
  while (hi - lo > 1) {
    const unsigned long long mid = lo + (hi - lo) / 2;
    if (net(mid) >= agg_lim) hi = mid; else lo = mid;
  }
  *full_min = hi;
}

TrialParams make_params(ara_ctx* ctx, const YetDev& Y, const LayerDev& L, int64_t t0,
                        int64_t n, double* d_ylt) {
  TrialParams p;
  memset(&p, 0, sizeof p);
  p.ids = Y.ids;
  p.offsets = Y.offsets;
  p.evt = L.evt;
  p.recs = L.packed;
  p.tables = L.tables;
  p.corr = L.corr;
  p.starts = L.starts;
  p.rec_idx = L.packed_rec;
  for (int j = 0; j < kMaxLayerElts; ++j) p.handles[j] = L.handles[j];
  p.n_slots = L.n_slots;
  p.occ_ret = (float)L.occ_ret;
  p.occ_lim = (float)L.occ_lim;
  p.agg_ret = L.agg_ret;
  p.agg_lim = L.agg_lim;
  p.seed = ctx->cfg.seed;
  ara::philox_round_keys(p.seed, p.rk0, p.rk1);
  p.t0 = t0;
  p.n = n;
  p.ylt = d_ylt;
  p.not_conv = ctx->d_not_conv;
  p.stats = ctx->d_stats;
  p.yet_n = Y.n_trials;
  const int qe = year_grid_exponent(occurrence_bound(L.ev_bound, L.occ_ret, L.occ_lim), Y.max_len);
  p.q_scale = std::ldexp(1.0f, -qe);
  p.q_unit = std::ldexp(1.0, qe);
  agg_bounds(p.q_unit, L.agg_ret, L.agg_lim, &p.agg_zero_max, &p.agg_full_min);
  if (L.band_log2w > 0) {
    for (const auto& v : Y.bands)
      if (v.log2w == L.band_log2w) {
        p.bocc = v.occ;
        p.boff = v.off;
        p.log2w = v.log2w;
        p.kbits = v.kbits;
        p.n_bands = v.n_bands;
      }
  }
  if (ctx->cfg.use_surrogate && ctx->mlp_ready) {
    p.mlp = &ctx->mlp_W->fwd;
    p.mlp_bound = ctx->mlp_bound;
    p.mlp_eps = ctx->mlp_eps;
  }
  return p;
}

ara_status ensure_stream_ring(ara_ctx* ctx, int64_t cap) {
  if (cap > ctx->stream_cap) {
    ctx->pf_yet = -1;
    if (ctx->copy_stream) CUDA_TRY(ctx, cudaStreamSynchronize(ctx->copy_stream));
    for (int b = 0; b < kStreamBufs; ++b) {
      dev_free(ctx->d_sids[b]);
      ctx->d_sids[b] = nullptr;
    }
    ctx->stream_cap = 0;
    for (int b = 0; b < kStreamBufs; ++b)
      CUDA_TRY(ctx, dev_alloc(&ctx->d_sids[b], cap));
    ctx->stream_cap = cap;
  }
  if (!ctx->copy_stream)
    CUDA_TRY(ctx, cudaStreamCreateWithFlags(&ctx->copy_stream, cudaStreamNonBlocking));
  for (int b = 0; b < kStreamBufs; ++b) {
    if (!ctx->ev_ready[b])
      CUDA_TRY(ctx, cudaEventCreateWithFlags(&ctx->ev_ready[b], cudaEventDisableTiming));
    if (!ctx->ev_free[b])
      CUDA_TRY(ctx, cudaEventCreateWithFlags(&ctx->ev_free[b], cudaEventDisableTiming));
  }
  return ARA_OK;
}

int64_t stream_chunk_end(const YetDev& Y, int64_t tb, int64_t end, int64_t cap) {
  int64_t te = tb + 1;
  while (te < end && Y.h_off[(size_t)te + 1] - Y.h_off[(size_t)tb] <= cap) ++te;
  return te;
}

void prefetch_stream(ara_ctx* ctx, int32_t yet) {
  const YetDev& Y = ctx->yets[yet];
  ctx->pf_yet = -1;
  ctx->pf_count = 0;
  if (Y.n_occ == 0) return;
  const std::string detail = ctx->detail;  // a failure here is not the caller's error
  const int64_t cap = std::max<int64_t>(ctx->stream_chunk, Y.max_len);
  if (ensure_stream_ring(ctx, cap) != ARA_OK) {
    cudaGetLastError();
    ctx->detail = detail;
    return;
  }
  // copies of at most 2^21 ids (8 MB, ~0.15 ms of PCIe): the caller's staging copies, issued
  // meanwhile on the compute stream, wait behind one piece at most
  constexpr int64_t kPiece = (int64_t)1 << 21;
  int k = 0;
  for (int64_t tb = 0; tb < Y.n_trials && k < kStreamBufs; ++k) {
    const int64_t te = stream_chunk_end(Y, tb, Y.n_trials, cap);
    const int64_t ob = Y.h_off[(size_t)tb], len = Y.h_off[(size_t)te] - ob;
    bool ok = cudaStreamWaitEvent(ctx->copy_stream, ctx->ev_free[k], 0) == cudaSuccess;
    for (int64_t q = 0; ok && q < len; q += kPiece)
      ok = cudaMemcpyAsync(ctx->d_sids[k] + q, Y.h_ids + ob + q,
                           sizeof(int32_t) * (size_t)std::min(kPiece, len - q),
                           cudaMemcpyHostToDevice, ctx->copy_stream) == cudaSuccess;
    if (!ok || cudaEventRecord(ctx->ev_ready[k], ctx->copy_stream) != cudaSuccess) {
      cudaGetLastError();
      cudaStreamSynchronize(ctx->copy_stream);
      return;
    }
    ctx->pf_tb[k] = tb;
    ctx->pf_te[k] = te;
    tb = te;
  }
  ctx->pf_count = k;
  ctx->pf_cap = cap;
  ctx->pf_yet = yet;
}

extern "C" {

// A run over a host-resident YET: trials in chunks of whole trials (up to ctx->stream_chunk
// occurrences), each chunk's ids copied on the copy stream into the next buffer of the ring while
// earlier chunks are checked and run on st; the run of a chunk skips its work if any chunk so far
// failed the check.  Chunks that ara_create_yet_host copied ahead are used as they are when this
// run starts at trial 0 (the ring then holds chunk k in buffer k).  (Timestamps never cross: the
// caller checks them on host threads.)  Outputs are device pointers for trials [t0, t0 + n).
static ara_status run_streamed(ara_ctx* ctx, int32_t yet, const LayerDev& L, int64_t t0,
                               int64_t n, double* d_ylt, double* d_oep, float* d_olt,
                               double* d_inc, cudaStream_t st) {
  const YetDev& Y = ctx->yets[yet];
  const int64_t cap = std::max<int64_t>(ctx->stream_chunk, Y.max_len);
  const int n_ahead = (ctx->pf_yet == yet && ctx->pf_cap == cap && t0 == 0) ? ctx->pf_count : 0;
  ctx->pf_yet = -1;  // the ring is this run's from here on
  ara_status s = ensure_stream_ring(ctx, cap);
  if (s != ARA_OK) return s;
  for (int b = 0; b < kStreamBufs; ++b)
    CUDA_TRY(ctx, cudaEventRecord(ctx->ev_free[b], st));  // every buffer free once st gets here
  CUDA_TRY(ctx, cudaMemsetAsync(ctx->d_flags, 0, sizeof(unsigned int), st));
  const int64_t q_first = Y.h_off[(size_t)t0];
  int k = 0;
  for (int64_t tb = t0; tb < t0 + n; ++k) {
    const int64_t te = stream_chunk_end(Y, tb, t0 + n, cap);
    const int64_t ob = Y.h_off[(size_t)tb], len = Y.h_off[(size_t)te] - ob;
    const int b = k % kStreamBufs;
    if (!(k < n_ahead && ctx->pf_tb[k] == tb && ctx->pf_te[k] == te)) {
      CUDA_TRY(ctx, cudaStreamWaitEvent(ctx->copy_stream, ctx->ev_free[b], 0));
      if (len > 0)
        CUDA_TRY(ctx, cudaMemcpyAsync(ctx->d_sids[b], Y.h_ids + ob, sizeof(int32_t) * (size_t)len,
                                      cudaMemcpyHostToDevice, ctx->copy_stream));
      CUDA_TRY(ctx, cudaEventRecord(ctx->ev_ready[b], ctx->copy_stream));
    }
    CUDA_TRY(ctx, cudaStreamWaitEvent(st, ctx->ev_ready[b], 0));
    CUDA_TRY(ctx, launch_validate_yet_range(ctx->d_sids[b], nullptr, ob, Y.offsets, tb, te - tb,
                                            Y.catalog, ctx->d_flags, st));
    TrialParams p = make_params(ctx, Y, L, tb, te - tb, d_ylt + (tb - t0));
    p.ids = ctx->d_sids[b];
    p.occ_base = ob;
    p.abort_flag = ctx->d_flags;
    p.oep = d_oep ? d_oep + (tb - t0) : nullptr;
    p.olt = d_olt ? d_olt + (ob - q_first) : nullptr;
    p.inc = d_inc ? d_inc + (ob - q_first) : nullptr;
    CUDA_TRY(ctx, launch_trial(p, L.mask_words, ctx->cfg.precision, layer_inversion(ctx, L),
                               false, st));
    CUDA_TRY(ctx, cudaEventRecord(ctx->ev_free[b], st));
    tb = te;
  }
  return ARA_OK;
}

ara_status ara_run_events(ara_ctx* ctx, int32_t yet, int32_t layer, int64_t t0, int64_t n,
                          double* ylt, double* oep, float* olt, double* inc, void* stream) {
  if (!ctx) return ARA_ERR_INVALID_ARG;
  ara_status s = check_run_args(ctx, yet, layer, t0, n);
  if (s != ARA_OK) return s;
  if (n > 0 && !ylt) return fail(ctx, ARA_ERR_INVALID_ARG, "ylt is NULL");
  if (n == 0) return ARA_OK;
  CUDA_TRY(ctx, cudaSetDevice(ctx->device));
  const bool dev_out = is_device_ptr(ylt);
  if ((oep && is_device_ptr(oep) != dev_out) || (olt && is_device_ptr(olt) != dev_out) ||
      (inc && is_device_ptr(inc) != dev_out))
    return fail(ctx, ARA_ERR_INVALID_ARG, "outputs must all be host or all device memory");
  const bool per_occ = olt != nullptr || inc != nullptr;
  if (ctx->yets[yet].host && stream)
    return fail(ctx, ARA_ERR_INVALID_ARG, "runs over a host-resident YET are blocking");
  if (inc && ctx->cfg.precision != ARA_ACC_FP64)
    return fail(ctx, ARA_ERR_INVALID_ARG, "occurrence increments need ARA_ACC_FP64 year sums");
  cudaStream_t st = stream ? (cudaStream_t)stream : ctx->stream;
  if (stream && !dev_out)
    return fail(ctx, ARA_ERR_INVALID_ARG, "asynchronous runs need device outputs");
  const YetDev& Y = ctx->yets[yet];
  double* d_ylt = ylt;
  double* d_oep = oep;
  float* d_olt = olt;
  double* d_inc = inc;
  int64_t n_occ = 0;
  OrderedTemp tmp_olt{nullptr, st}, tmp_inc{nullptr, st};  // staged outputs' device memory
  // host outputs are staged on the device; so are all outputs of a streamed run, which are
  // handed over only once every chunk has passed validation
  const bool staged = !dev_out || Y.host;
  if (staged) {
    s = ensure_ylt_tmp(ctx, oep ? 2 * n : n);
    if (s != ARA_OK) return s;
    d_ylt = ctx->d_ylt_tmp;
    d_oep = oep ? ctx->d_ylt_tmp + n : nullptr;
    if (per_occ) {
      int64_t ends[2];
      CUDA_TRY(ctx, cudaMemcpyAsync(&ends[0], Y.offsets + t0, sizeof(int64_t),
                                    cudaMemcpyDeviceToHost, st));
      CUDA_TRY(ctx, cudaMemcpyAsync(&ends[1], Y.offsets + t0 + n, sizeof(int64_t),
                                    cudaMemcpyDeviceToHost, st));
      CUDA_TRY(ctx, cudaStreamSynchronize(st));
      n_occ = ends[1] - ends[0];
      if (olt) {
        CUDA_TRY(ctx, mem_alloc(ctx, &d_olt, n_occ, true, st));
        tmp_olt.p = d_olt;
      }
      if (inc) {
        CUDA_TRY(ctx, mem_alloc(ctx, &d_inc, n_occ, true, st));
        tmp_inc.p = d_inc;
      }
    }
  }
  unsigned long long nc_before = 0;
  if (!stream)
    CUDA_TRY(ctx, cudaMemcpyAsync(&nc_before, ctx->d_not_conv, sizeof nc_before,
                                  cudaMemcpyDeviceToHost, st));
  s = prepare_layer_for_run(ctx, ctx->layers[layer], n, !per_occ);
  if (s != ARA_OK) return s;
  TrialParams p = make_params(ctx, Y, ctx->layers[layer], t0, n, d_ylt);
  p.oep = d_oep;
  p.olt = d_olt;
  p.inc = d_inc;
  // per-occurrence outputs are written in trial order, so they keep the trial-major schedule
  // a host YET's timestamps are checked once, on host threads, while its first run streams;
  // the check starts once every copy and launch of the run is queued (its threads would
  // otherwise hold the cores the queueing thread needs)
  unsigned int ts_flags = 0;
  std::thread ts_check;
  struct Joiner {
    std::thread& t;
    ~Joiner() {
      if (t.joinable()) t.join();
    }
  } joiner{ts_check};
  if (Y.host) {
    s = run_streamed(ctx, yet, ctx->layers[layer], t0, n, d_ylt, d_oep, d_olt, d_inc, st);
    if (s != ARA_OK) return s;
    if (!Y.ts_checked && Y.n_occ > 0)
      ts_check = std::thread(
          [&]() { ts_flags = validate_timestamps_host(Y.h_off.data(), Y.h_ts, Y.n_trials); });
  } else if (!per_occ && run_band_schedule(ctx, ctx->layers[layer])) {
    // year sums (8 B per trial), then the OEP maxima (4 B per trial) in the same scratch
    s = ensure_ysum(ctx, oep ? n + (n + 1) / 2 : n);
    if (s != ARA_OK) return s;
    p.ysum = ctx->d_ysum;
    p.omax = oep ? reinterpret_cast<unsigned int*>(ctx->d_ysum + n) : nullptr;
    CUDA_TRY(ctx, launch_band(p, ctx->layers[layer].mask_words, ctx->cfg.precision,
                              layer_inversion(ctx, ctx->layers[layer]), st));
  } else {
    CUDA_TRY(ctx, launch_trial(p, ctx->layers[layer].mask_words, ctx->cfg.precision,
                               layer_inversion(ctx, ctx->layers[layer]), false, st));
  }
  if (stream) return ARA_OK;
  unsigned long long nc_after = 0;
  unsigned int yet_flags = 0;
  CUDA_TRY(ctx, cudaMemcpyAsync(&nc_after, ctx->d_not_conv, sizeof nc_after,
                                cudaMemcpyDeviceToHost, st));
  if (Y.host) {
    CUDA_TRY(ctx, cudaMemcpyAsync(&yet_flags, ctx->d_flags, sizeof yet_flags,
                                  cudaMemcpyDeviceToHost, st));
    CUDA_TRY(ctx, cudaStreamSynchronize(st));
    if (ts_check.joinable()) {
      ts_check.join();
      yet_flags |= ts_flags;
      if (ts_flags == 0) ctx->yets[yet].ts_checked = true;
    }
    if (yet_flags)  // nothing is written to the caller's outputs
      return fail(ctx, ARA_ERR_INVALID_ARG, "YET rejected:%s%s%s",
                  (yet_flags & 1) ? " event id outside [0, catalog_size)" : "",
                  (yet_flags & 2) ? " timestamps decrease within a trial" : "",
                  (yet_flags & 4) ? " NaN timestamp" : "");
  }
  if (staged) {  // to host or device outputs alike
    CUDA_TRY(ctx, cudaMemcpyAsync(ylt, d_ylt, sizeof(double) * (size_t)n, cudaMemcpyDefault, st));
    if (oep)
      CUDA_TRY(ctx, cudaMemcpyAsync(oep, d_oep, sizeof(double) * (size_t)n, cudaMemcpyDefault,
                                    st));
    if (olt && n_occ > 0)
      CUDA_TRY(ctx, cudaMemcpyAsync(olt, d_olt, sizeof(float) * (size_t)n_occ, cudaMemcpyDefault,
                                    st));
    if (inc && n_occ > 0)
      CUDA_TRY(ctx, cudaMemcpyAsync(inc, d_inc, sizeof(double) * (size_t)n_occ,
                                    cudaMemcpyDefault, st));
  }
  CUDA_TRY(ctx, cudaStreamSynchronize(st));
  if (nc_after != nc_before)
    return fail(ctx, ARA_ERR_NOT_CONVERGED, "%llu inversions hit the iteration cap",
                nc_after - nc_before);
  return ARA_OK;
}

ara_status ara_run_ep(ara_ctx* ctx, int32_t yet, int32_t layer, int64_t t0, int64_t n,
                      double* ylt, double* oep, void* stream) {
  return ara_run_events(ctx, yet, layer, t0, n, ylt, oep, nullptr, nullptr, stream);
}

ara_status ara_run(ara_ctx* ctx, int32_t yet, int32_t layer, int64_t t0, int64_t n, double* ylt,
                   void* stream) {
  return ara_run_events(ctx, yet, layer, t0, n, ylt, nullptr, nullptr, nullptr, stream);
}

ara_status ara_run_portfolio(ara_ctx* ctx, int32_t yet, const int32_t* layers, int32_t n_layers,
                             int64_t t0, int64_t n, double* ylt, void* stream) {
  if (!ctx) return ARA_ERR_INVALID_ARG;
  if (n_layers < 0 || (n_layers > 0 && !layers))
    return fail(ctx, ARA_ERR_INVALID_ARG, "bad layer list");
  for (int32_t i = 0; i < n_layers; ++i) {
    const ara_status s = check_run_args(ctx, yet, layers[i], t0, n);
    if (s != ARA_OK) return s;
  }
  if (n == 0 || n_layers == 0) return ARA_OK;
  if (!ylt) return fail(ctx, ARA_ERR_INVALID_ARG, "ylt is NULL");
  CUDA_TRY(ctx, cudaSetDevice(ctx->device));
  const bool dev_out = is_device_ptr(ylt);
  cudaStream_t st = stream ? (cudaStream_t)stream : ctx->stream;
  if (stream && !dev_out)
    return fail(ctx, ARA_ERR_INVALID_ARG, "asynchronous runs need a device ylt");
  const int64_t total = (int64_t)n_layers * n;
  double* d_ylt = ylt;
  if (!dev_out) {
    ara_status s = ensure_ylt_tmp(ctx, total);
    if (s != ARA_OK) return s;
    d_ylt = ctx->d_ylt_tmp;
  }
  if (ctx->yets[yet].host)
    return fail(ctx, ARA_ERR_INVALID_ARG, "a host-resident YET runs one layer per call");
  for (int32_t i = 0; i < n_layers; ++i) {
    ara_status s = prepare_layer_for_run(ctx, ctx->layers[layers[i]], n, true);
    if (s != ARA_OK) return s;
  }
  // one launch item per layer, grouped by schedule, inversion and lookup-entry width (one
  // batched launch per group): band-major items first, each with its own year-sum rows
  const YetDev& Y = ctx->yets[yet];
  std::vector<int32_t> order(n_layers);
  for (int32_t i = 0; i < n_layers; ++i) order[i] = i;
  auto group = [&](int32_t i) {  // 0, 1 band-major; 2 + 2 inversion + (width - 1) trial-major
    const LayerDev& L = ctx->layers[layers[i]];
    const int w = L.mask_words == 1 ? 0 : 1;
    return uses_band_schedule(ctx, L) ? w : 2 + 2 * layer_inversion(ctx, L) + w;
  };
  std::stable_sort(order.begin(), order.end(),
                   [&](int32_t a, int32_t b) { return group(a) < group(b); });
  int32_t n_band = 0;
  for (int32_t i = 0; i < n_layers; ++i) n_band += group(i) < 2 ? 1 : 0;
  if (n_band > 0) {
    ara_status s = ensure_ysum(ctx, (int64_t)n_band * n);
    if (s != ARA_OK) return s;
    CUDA_TRY(ctx, cudaMemsetAsync(ctx->d_ysum, 0,
                                  sizeof(unsigned long long) * (size_t)n_band * (size_t)n, st));
  }
  std::vector<TrialParams> items(n_layers);
  std::vector<int64_t> begin(3 * (size_t)n_layers, 0);  // warp / block / trial firsts per item
  struct Group {
    int32_t first = 0, count = 0;
    int64_t units = 0, trials = 0;
    bool corr = false;  // some item carries correlated weights
  };
  Group g[8];
  int32_t band_row = 0;
  unsigned long long nc_before = 0;
  if (!stream)
    CUDA_TRY(ctx, cudaMemcpyAsync(&nc_before, ctx->d_not_conv, sizeof nc_before,
                                  cudaMemcpyDeviceToHost, st));
  // a layer whose own grid is many waves deep runs as its own launch (launch parameters in the
  // constant bank, as ara_run); only small layers share a batched launch, where filling the GPU
  // matters more than the items' parameters being read from global memory
  const int64_t big_warps = 12ll * ctx->sm_count * 32;  // 12 waves of 32 resident warps per SM
  int32_t n_items = 0;
  for (int32_t k = 0; k < n_layers; ++k) {
    const int32_t i = order[k];
    const LayerDev& L = ctx->layers[layers[i]];
    TrialParams p = make_params(ctx, Y, L, t0, n, d_ylt + (int64_t)i * n);
    const bool band = group(i) < 2;
    // band-major: a warp per 32 trials per band; trial-major: a warp per trial
    const int64_t own_warps = band ? (int64_t)p.n_bands * ((n + 31) / 32) : n;
    if (own_warps >= big_warps) {
      if (band) {
        p.ysum = ctx->d_ysum + (int64_t)band_row++ * n;
        CUDA_TRY(ctx, launch_band(p, L.mask_words, ctx->cfg.precision, 0, st));
      } else {
        CUDA_TRY(ctx, launch_trial(p, L.mask_words, ctx->cfg.precision,
                                   layer_inversion(ctx, L), false, st));
      }
      continue;
    }
    const int32_t kk = n_items++;
    Group& G = g[group(i)];
    if (G.count == 0) G.first = kk;
    if (band) {
      p.tiles = (int32_t)band_tiles(n);
      p.ysum = ctx->d_ysum + (int64_t)band_row++ * n;
      begin[n_layers + kk] = G.units;
      begin[2 * (size_t)n_layers + kk] = G.trials;
      G.units += (int64_t)p.n_bands * p.tiles;
      G.trials += n;
    } else {
      begin[kk] = G.units;
      G.units += n;
    }
    G.count++;
    G.corr = G.corr || p.corr != nullptr;
    items[kk] = p;
  }
  if (n_items == 0) return finish_run(ctx, stream, dev_out, ylt, d_ylt, total, nc_before, st);
  TrialParams* d_items = nullptr;
  int64_t* d_begin = nullptr;
  CUDA_TRY(ctx, mem_alloc(ctx, &d_items, n_layers, true, st));
  OrderedTemp tmp_items{d_items, st};
  CUDA_TRY(ctx, mem_alloc(ctx, &d_begin, 3 * (int64_t)n_layers, true, st));
  OrderedTemp tmp_begin{d_begin, st};
  // pageable sources: each copy has read its source when the call returns
  CUDA_TRY(ctx, cudaMemcpyAsync(d_items, items.data(), sizeof(TrialParams) * (size_t)n_layers,
                                cudaMemcpyHostToDevice, st));
  CUDA_TRY(ctx, cudaMemcpyAsync(d_begin, begin.data(), sizeof(int64_t) * begin.size(),
                                cudaMemcpyHostToDevice, st));
  for (int gi = 0; gi < 8; ++gi) {
    const Group& G = g[gi];
    if (G.count == 0) continue;
    const int mw = (gi & 1) ? 2 : 1;
    const int inv = gi < 2 ? 0 : (gi - 2) / 2;
    if (gi < 2)
      CUDA_TRY(ctx, launch_band_batch(d_items + G.first, d_begin + n_layers + G.first,
                                      d_begin + 2 * (int64_t)n_layers + G.first, G.count,
                                      G.units, G.trials, mw, G.corr, ctx->cfg.precision,
                                      st));
    else
      CUDA_TRY(ctx, launch_trial_batch(d_items + G.first, d_begin + G.first, G.count, G.units,
                                       mw, ctx->cfg.precision, inv, st));
  }
  return finish_run(ctx, stream, dev_out, ylt, d_ylt, total, nc_before, st);
}

ara_status ara_get_stats(ara_ctx* ctx, int64_t out[9]) {
  if (!ctx || !out) return ARA_ERR_INVALID_ARG;
  CUDA_TRY(ctx, cudaSetDevice(ctx->device));
  CUDA_TRY(ctx, cudaDeviceSynchronize());
  unsigned long long raw[kStatCounters * kStatStripes], v[kStatCounters] = {}, nc = 0;
  CUDA_TRY(ctx, cudaMemcpy(raw, ctx->d_stats, sizeof raw, cudaMemcpyDeviceToHost));
  for (int c = 0; c < kStatCounters; ++c)
    for (int s = 0; s < kStatStripes; ++s) v[c] += raw[c * kStatStripes + s];
  CUDA_TRY(ctx, cudaMemcpy(&nc, ctx->d_not_conv, sizeof nc, cudaMemcpyDeviceToHost));
  out[0] = (int64_t)v[0];
  out[1] = (int64_t)v[1];
  out[2] = (int64_t)v[2];
  out[3] = (int64_t)nc;
  out[4] = (int64_t)v[3];
  out[5] = launches_so_far();
  out[6] = (int64_t)v[4];
  int64_t unc = 0;
  for (const auto& e : ctx->elts)
    if (e.live) unc += e.n_uncertified;
  for (const auto& l : ctx->layers)
    if (l.live) unc += l.n_uncertified;
  out[7] = unc;
  out[8] = (int64_t)v[5];
  return ARA_OK;
}

ara_status ara_set_stream(ara_ctx* ctx, void* stream) {
  if (!ctx) return ARA_ERR_INVALID_ARG;
  CUDA_TRY(ctx, cudaSetDevice(ctx->device));
  CUDA_TRY(ctx, cudaStreamSynchronize(ctx->stream));
  ctx->stream = stream ? (cudaStream_t)stream : ctx->own_stream;
  return ARA_OK;
}

ara_status ara_not_converged(ara_ctx* ctx, int64_t* count) {
  if (!ctx || !count) return ARA_ERR_INVALID_ARG;
  CUDA_TRY(ctx, cudaSetDevice(ctx->device));
  CUDA_TRY(ctx, cudaDeviceSynchronize());
  unsigned long long v = 0;
  CUDA_TRY(ctx, cudaMemcpy(&v, ctx->d_not_conv, sizeof v, cudaMemcpyDeviceToHost));
  *count = (int64_t)v;
  return ARA_OK;
}

ara_status ara_trace_hits(ara_ctx* ctx, int32_t yet, int32_t layer, int64_t t0, int64_t n,
                          int64_t max_hits, int32_t* hit_trial, int32_t* hit_k, int32_t* hit_j,
                          int32_t* hit_rec, float* hit_u, float* hit_x, float* hit_loss,
                          double* ylt, int64_t* n_hits) {
  if (!ctx) return ARA_ERR_INVALID_ARG;
  ara_status s = check_run_args(ctx, yet, layer, t0, n);
  if (s != ARA_OK) return s;
  if (!n_hits || max_hits < 0 || (max_hits > 0 && (!hit_trial || !hit_k || !hit_j || !hit_rec ||
                                                     !hit_u || !hit_x || !hit_loss)) || !ylt)
    return fail(ctx, ARA_ERR_INVALID_ARG, "NULL trace buffer");
  if (ctx->yets[yet].host)
    return fail(ctx, ARA_ERR_INVALID_ARG, "tracing needs a device-resident YET");
  CUDA_TRY(ctx, cudaSetDevice(ctx->device));
  const YetDev& Y = ctx->yets[yet];
  LayerDev& L = ctx->layers[layer];
  const int64_t cap = std::max<int64_t>(1, Y.max_len * L.n_slots);
  const int64_t total = n * cap;
  if (total > ((int64_t)1 << 27)) return fail(ctx, ARA_ERR_INVALID_ARG, "trace too large");
  if (n == 0) {
    *n_hits = 0;
    return ARA_OK;
  }
  // the layer as a run of these trials would see it (tables or start tables), so that the trace
  // reproduces the run's year losses bit for bit
  s = prepare_layer_for_run(ctx, L, n, false);
  if (s != ARA_OK) return s;
  int32_t *d_k = nullptr, *d_j = nullptr, *d_rec = nullptr, *d_cnt = nullptr;
  float *d_u = nullptr, *d_x = nullptr, *d_loss = nullptr;
  double* d_ylt = nullptr;
  auto cleanup = [&]() {
    cudaStreamSynchronize(ctx->stream);
    dev_free(d_k); dev_free(d_j); dev_free(d_rec); dev_free(d_cnt);
    dev_free(d_u); dev_free(d_x); dev_free(d_loss); dev_free(d_ylt);
  };
  cudaError_t e;
  if ((e = dev_alloc(&d_k, total)) != cudaSuccess || (e = dev_alloc(&d_j, total)) != cudaSuccess ||
      (e = dev_alloc(&d_rec, total)) != cudaSuccess || (e = dev_alloc(&d_cnt, n)) != cudaSuccess ||
      (e = dev_alloc(&d_u, total)) != cudaSuccess || (e = dev_alloc(&d_x, total)) != cudaSuccess ||
      (e = dev_alloc(&d_loss, total)) != cudaSuccess || (e = dev_alloc(&d_ylt, n)) != cudaSuccess) {
    cudaGetLastError();
    cleanup();
    return fail(ctx, ARA_ERR_OOM, "trace buffers: %s", cudaGetErrorString(e));
  }
  TrialParams p = make_params(ctx, Y, L, t0, n, d_ylt);
  p.trace_cap = cap;
  p.tr_k = d_k; p.tr_j = d_j; p.tr_rec = d_rec; p.tr_u = d_u; p.tr_x = d_x; p.tr_loss = d_loss;
  p.tr_count = d_cnt;
  std::vector<int32_t> cnt(n), k(total), j(total), rec(total);
  std::vector<float> u(total), x(total), loss(total);
  e = launch_trial(p, L.mask_words, ARA_ACC_FP64, layer_inversion(ctx, L), true, ctx->stream);
  if (e == cudaSuccess) e = cudaMemcpyAsync(cnt.data(), d_cnt, sizeof(int32_t) * n, cudaMemcpyDeviceToHost, ctx->stream);
  if (e == cudaSuccess) e = cudaMemcpyAsync(k.data(), d_k, sizeof(int32_t) * total, cudaMemcpyDeviceToHost, ctx->stream);
  if (e == cudaSuccess) e = cudaMemcpyAsync(j.data(), d_j, sizeof(int32_t) * total, cudaMemcpyDeviceToHost, ctx->stream);
  if (e == cudaSuccess) e = cudaMemcpyAsync(rec.data(), d_rec, sizeof(int32_t) * total, cudaMemcpyDeviceToHost, ctx->stream);
  if (e == cudaSuccess) e = cudaMemcpyAsync(u.data(), d_u, sizeof(float) * total, cudaMemcpyDeviceToHost, ctx->stream);
  if (e == cudaSuccess) e = cudaMemcpyAsync(x.data(), d_x, sizeof(float) * total, cudaMemcpyDeviceToHost, ctx->stream);
  if (e == cudaSuccess) e = cudaMemcpyAsync(loss.data(), d_loss, sizeof(float) * total, cudaMemcpyDeviceToHost, ctx->stream);
  if (e == cudaSuccess) e = cudaMemcpyAsync(ylt, d_ylt, sizeof(double) * n, cudaMemcpyDeviceToHost, ctx->stream);
  if (e == cudaSuccess) e = cudaStreamSynchronize(ctx->stream);
  cleanup();
  if (e != cudaSuccess) {
    cudaGetLastError();
    return fail(ctx, ARA_ERR_CUDA, "trace: %s", cudaGetErrorString(e));
  }
  int64_t h = 0;
  for (int64_t t = 0; t < n; ++t) {
    for (int32_t q = 0; q < cnt[t] && q < cap; ++q) {
      if (h < max_hits) {
        const int64_t o = t * cap + q;
        hit_trial[h] = (int32_t)t;
        hit_k[h] = k[o];
        hit_j[h] = j[o];
        hit_rec[h] = rec[o];
        hit_u[h] = u[o];
        hit_x[h] = x[o];
        hit_loss[h] = loss[o];
      }
      ++h;
    }
  }
  *n_hits = h;
  return ARA_OK;
}

}  // extern "C"
