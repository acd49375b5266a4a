// ara_api.cu -- the C ABI of libara (include/ara.h): contexts, handles, validation, launches.
#include <cuda_runtime.h>
#include <math.h>
#include <stdarg.h>
#include <stdio.h>
#include <string.h>

#include <algorithm>
#include <cmath>
#include <new>
#include <random>
#include <string>
#include <vector>

#include "../../include/ara.h"
#include "ara_internal.h"
#include "ara_ctx.h"
#include "ara_philox.cuh"

using namespace ara;


namespace {

ara_status fail(ara_ctx* c, ara_status s, const char* fmt, ...) {
  if (c) {
    char buf[512];
    va_list ap;
    va_start(ap, fmt);
    vsnprintf(buf, sizeof buf, fmt, ap);
    va_end(ap);
    c->detail = buf;
  }
  return s;
}

#define CUDA_TRY(ctx, call)                                                                   \
  do {                                                                                        \
    cudaError_t _e = (call);                                                                  \
    if (_e != cudaSuccess) {                                                                  \
      cudaGetLastError();                                                                     \
      return fail(ctx, _e == cudaErrorMemoryAllocation ? ARA_ERR_OOM : ARA_ERR_CUDA, "%s: %s", \
                  #call, cudaGetErrorString(_e));                                             \
    }                                                                                         \
  } while (0)

bool is_device_ptr(const void* p) {
  if (!p) return false;
  cudaPointerAttributes a;
  if (cudaPointerGetAttributes(&a, p) != cudaSuccess) {
    cudaGetLastError();
    return false;
  }
  return a.type == cudaMemoryTypeDevice || a.type == cudaMemoryTypeManaged;
}

template <class T>
cudaError_t dev_alloc(T** p, int64_t n) {
  *p = nullptr;
  if (n <= 0) n = 1;
  return cudaMalloc(reinterpret_cast<void**>(p), sizeof(T) * (size_t)n);
}

void dev_free(void* p) {
  if (p) cudaFree(p);
}

// Allocation either plain (cudaMalloc/cudaFree, which waits for the device) or stream-ordered
// on st (cudaMallocAsync/cudaFreeAsync from the device's memory pool, which never blocks the host:
// the serving loop builds and frees layers while launches run).
template <class T>
cudaError_t mem_alloc(T** p, int64_t n, bool ordered, cudaStream_t st) {
  *p = nullptr;
  if (n <= 0) n = 1;
  const size_t bytes = sizeof(T) * (size_t)n;
  return ordered ? cudaMallocAsync(reinterpret_cast<void**>(p), bytes, st)
                 : cudaMalloc(reinterpret_cast<void**>(p), bytes);
}

void mem_free(const void* p, bool ordered, cudaStream_t st) {
  if (!p) return;
  if (ordered) cudaFreeAsync(const_cast<void*>(p), st);
  else cudaFree(const_cast<void*>(p));
}

// A stream-ordered temporary freed when the call returns, on whichever path.
struct OrderedTemp {
  void* p;
  cudaStream_t st;
  ~OrderedTemp() { mem_free(p, true, st); }
};

// Copies n elements from a host or device pointer into device memory on the stream.
template <class T>
cudaError_t copy_in(T* dst, const T* src, int64_t n, cudaStream_t st) {
  if (n <= 0) return cudaSuccess;
  return cudaMemcpyAsync(dst, src, sizeof(T) * (size_t)n, cudaMemcpyDefault, st);
}

void free_yet(YetDev& y) {
  for (auto& v : y.bands) free_band_variant(v);
  dev_free(y.ids);
  dev_free(y.ts);
  dev_free(y.offsets);
  y = YetDev();
}
void free_elt(EltDev& e) {
  dev_free(e.ids);
  dev_free(e.recs);
  dev_free(e.tables);
  dev_free(e.corr);
  dev_free(e.ab64);
  e = EltDev();
}

ara_status set_device(ara_ctx* c) {
  CUDA_TRY(c, cudaSetDevice(c->device));
  return ARA_OK;
}

ara_status ensure_ylt_tmp(ara_ctx* c, int64_t n) {
  if (n <= c->ylt_tmp_cap) return ARA_OK;
  dev_free(c->d_ylt_tmp);
  c->d_ylt_tmp = nullptr;
  c->ylt_tmp_cap = 0;
  CUDA_TRY(c, dev_alloc(&c->d_ylt_tmp, n));
  c->ylt_tmp_cap = n;
  return ARA_OK;
}

ara_status ensure_ysum(ara_ctx* c, int64_t n) {
  if (n <= c->ysum_cap) return ARA_OK;
  dev_free(c->d_ysum);
  c->d_ysum = nullptr;
  c->ysum_cap = 0;
  CUDA_TRY(c, dev_alloc(&c->d_ysum, n));
  c->ysum_cap = n;
  return ARA_OK;
}

ara_status ensure_sort(ara_ctx* c, int64_t n) {
  SortScratch& s = c->sort;
  const int64_t tiles = sort_tiles(n);
  const int64_t hist_n = 256 * tiles;
  if (n > s.cap) {
    for (int b = 0; b < 2; ++b) {
      dev_free(s.keys[b]);
      dev_free(s.vals[b]);
      s.keys[b] = nullptr;
      s.vals[b] = nullptr;
    }
    s.cap = 0;
    for (int b = 0; b < 2; ++b) {
      CUDA_TRY(c, dev_alloc(&s.keys[b], n));
      CUDA_TRY(c, dev_alloc(&s.vals[b], n));
    }
    s.cap = n;
  }
  if (hist_n > s.hist_cap) {
    dev_free(s.hist);
    dev_free(s.scan_tmp);
    s.hist = nullptr;
    s.scan_tmp = nullptr;
    s.hist_cap = 0;
    CUDA_TRY(c, dev_alloc(&s.hist, hist_n));
    s.scan_cap = scan_tmp_words(hist_n);
    CUDA_TRY(c, dev_alloc(&s.scan_tmp, s.scan_cap));
    s.hist_cap = hist_n;
  }
  if (!s.digit_flags) CUDA_TRY(c, dev_alloc(&s.digit_flags, 4));
  return ARA_OK;
}

int64_t tail_count(int64_t n, double rp) {
  const double q = (double)n / rp;
  const double r = nearbyint(q);
  int64_t k = (fabs(q - r) <= 1e-9 * fmax(1.0, q)) ? (int64_t)r : (int64_t)ceil(q);
  if (k < 1) k = 1;
  if (k > n) k = n;
  return k;
}

}  // namespace

void free_layer_on(LayerDev& l, bool ordered, cudaStream_t st) {
  mem_free(l.evt, ordered, st);
  mem_free(l.tables, ordered, st);
  mem_free(l.packed, ordered, st);
  mem_free(l.packed_rec, ordered, st);
  mem_free(l.corr, ordered, st);
  l = LayerDev();
}

void free_layer(LayerDev& l) { free_layer_on(l, false, nullptr); }

extern "C" {

const char* ara_status_string(ara_status s) {
  switch (s) {
    case ARA_OK: return "ok";
    case ARA_ERR_INVALID_ARG: return "invalid argument";
    case ARA_ERR_BAD_HANDLE: return "bad handle";
    case ARA_ERR_OOM: return "out of memory";
    case ARA_ERR_CUDA: return "CUDA error";
    case ARA_ERR_NOT_CONVERGED: return "inversion did not converge";
    case ARA_ERR_BUSY: return "busy";
    case ARA_ERR_NO_DEVICE: return "no CUDA device";
  }
  return "unknown status";
}

ara_status ara_create(const ara_config* cfg, ara_ctx** out) {
  if (!out) return ARA_ERR_INVALID_ARG;
  *out = nullptr;
  ara_config c{};
  c.seed = 42;
  if (cfg) c = *cfg;
  if (c.precision != ARA_ACC_FP64 && c.precision != ARA_ACC_KAHAN32) return ARA_ERR_INVALID_ARG;
  int ndev = 0;
  if (cudaGetDeviceCount(&ndev) != cudaSuccess || ndev <= 0) {
    cudaGetLastError();
    return ARA_ERR_NO_DEVICE;
  }
  if (c.device < 0 || c.device >= ndev) return ARA_ERR_INVALID_ARG;
  ara_ctx* ctx = new (std::nothrow) ara_ctx();
  if (!ctx) return ARA_ERR_OOM;
  ctx->cfg = c;
  ctx->device = c.device;
  if (cudaSetDevice(ctx->device) != cudaSuccess ||
      cudaStreamCreateWithFlags(&ctx->own_stream, cudaStreamNonBlocking) != cudaSuccess ||
      (ctx->stream = ctx->own_stream, false) ||
      dev_alloc(&ctx->d_not_conv, 1) != cudaSuccess || dev_alloc(&ctx->d_flags, 4) != cudaSuccess ||
      dev_alloc(&ctx->d_stats, kStatCounters * kStatStripes) != cudaSuccess ||
      cudaMemsetAsync(ctx->d_stats, 0, sizeof(unsigned long long) * kStatCounters * kStatStripes,
                      ctx->stream) != cudaSuccess ||
      cudaMalloc(&ctx->d_misc, 4096) != cudaSuccess ||
      cudaMemsetAsync(ctx->d_not_conv, 0, sizeof(unsigned long long), ctx->stream) != cudaSuccess ||
      cudaDeviceGetAttribute(&ctx->sm_count, cudaDevAttrMultiProcessorCount, ctx->device) !=
          cudaSuccess ||
      cudaStreamSynchronize(ctx->stream) != cudaSuccess) {
    cudaGetLastError();
    ara_destroy(ctx);
    return ARA_ERR_CUDA;
  }
  *out = ctx;
  return ARA_OK;
}

void ara_destroy(ara_ctx* ctx) {
  if (!ctx) return;
  cudaSetDevice(ctx->device);
  if (ctx->stream) cudaStreamSynchronize(ctx->stream);
  for (auto& y : ctx->yets) free_yet(y);
  for (auto& e : ctx->elts) free_elt(e);
  for (auto& l : ctx->layers) free_layer(l);
  for (int b = 0; b < 2; ++b) {
    dev_free(ctx->sort.keys[b]);
    dev_free(ctx->sort.vals[b]);
  }
  dev_free(ctx->sort.hist);
  dev_free(ctx->sort.scan_tmp);
  dev_free(ctx->sort.digit_flags);
  dev_free(ctx->d_ylt_tmp);
  dev_free(ctx->d_ysum);
  dev_free(ctx->d_sel);
  dev_free(ctx->d_not_conv);
  dev_free(ctx->d_stats);
  dev_free(ctx->d_flags);
  dev_free(ctx->d_misc);
  dev_free(ctx->mlp_P);
  dev_free(ctx->mlp_M);
  dev_free(ctx->mlp_V);
  dev_free(ctx->mlp_G);
  dev_free(ctx->mlp_W);
  dev_free(ctx->mlp_bound);
  for (int b = 0; b < 2; ++b) {
    dev_free(ctx->d_sids[b]);
    dev_free(ctx->d_sts[b]);
    if (ctx->ev_ready[b]) cudaEventDestroy(ctx->ev_ready[b]);
    if (ctx->ev_free[b]) cudaEventDestroy(ctx->ev_free[b]);
  }
  if (ctx->copy_stream) {
    cudaStreamSynchronize(ctx->copy_stream);
    cudaStreamDestroy(ctx->copy_stream);
  }
  if (ctx->own_stream) cudaStreamDestroy(ctx->own_stream);
  cudaGetLastError();
  delete ctx;
}

ara_status ara_last_error_detail(const ara_ctx* ctx, char* buf, size_t n) {
  if (!ctx || !buf || n == 0) return ARA_ERR_INVALID_ARG;
  snprintf(buf, n, "%s", ctx->detail.c_str());
  return ARA_OK;
}

ara_status ara_set_option(ara_ctx* ctx, int32_t option, int64_t value) {
  if (!ctx) return ARA_ERR_INVALID_ARG;
  switch (option) {
    case ARA_OPT_PRECISION:
      if (value != ARA_ACC_FP64 && value != ARA_ACC_KAHAN32)
        return fail(ctx, ARA_ERR_INVALID_ARG, "precision must be ARA_ACC_FP64 or ARA_ACC_KAHAN32");
      ctx->cfg.precision = (int32_t)value;
      return ARA_OK;
    case ARA_OPT_SEED:
      ctx->cfg.seed = (uint64_t)value;
      return ARA_OK;
    case ARA_OPT_INVERSION:
      if (value != ARA_INV_TABLE && value != ARA_INV_NEWTON)
        return fail(ctx, ARA_ERR_INVALID_ARG, "inversion must be ARA_INV_TABLE or ARA_INV_NEWTON");
      ctx->inversion = (int32_t)value;
      return ARA_OK;
    case ARA_OPT_SURROGATE:
      if (value != 0 && value != 1) return fail(ctx, ARA_ERR_INVALID_ARG, "surrogate is 0 or 1");
      if (value == 1 && !ctx->mlp_ready)
        return fail(ctx, ARA_ERR_INVALID_ARG, "no surrogate trained or loaded");
      ctx->cfg.use_surrogate = (int32_t)value;
      return ARA_OK;
    case ARA_OPT_BAND_WIDTH:
      if (value != 0 && (value < 10 || value > 20))
        return fail(ctx, ARA_ERR_INVALID_ARG, "band width exponent must be 0 or 10..20");
      ctx->band_log2w = (int32_t)value;
      return ARA_OK;
    case ARA_OPT_STREAM_CHUNK:
      if (value < 1024 || value > ((int64_t)1 << 30))
        return fail(ctx, ARA_ERR_INVALID_ARG, "stream chunk must be 1024 .. 2^30 occurrences");
      ctx->stream_chunk = value;
      return ARA_OK;
    case ARA_OPT_TABLES:
      if (value != ARA_TABLES_EAGER && value != ARA_TABLES_ON_DEMAND)
        return fail(ctx, ARA_ERR_INVALID_ARG, "tables must be ARA_TABLES_EAGER or _ON_DEMAND");
      ctx->table_policy = (int32_t)value;
      return ARA_OK;
    case ARA_OPT_SCHEDULE:
      if (value != ARA_SCHED_BAND && value != ARA_SCHED_TRIAL)
        return fail(ctx, ARA_ERR_INVALID_ARG, "schedule must be ARA_SCHED_BAND or ARA_SCHED_TRIAL");
      ctx->schedule = (int32_t)value;
      return ARA_OK;
  }
  return fail(ctx, ARA_ERR_INVALID_ARG, "unknown option %d", option);
}

ara_status ara_synchronize(ara_ctx* ctx) {
  if (!ctx) return ARA_ERR_INVALID_ARG;
  CUDA_TRY(ctx, cudaSetDevice(ctx->device));
  CUDA_TRY(ctx, cudaStreamSynchronize(ctx->stream));
  return ARA_OK;
}

// ---- YET ------------------------------------------------------------------------------------
ara_status ara_create_yet(ara_ctx* ctx, int64_t n_trials, const int64_t* trial_offsets,
                          const int32_t* event_ids, const float* timestamps,
                          int32_t catalog_size, int32_t* yet_out) {
  if (!ctx) return ARA_ERR_INVALID_ARG;
  if (!yet_out) return fail(ctx, ARA_ERR_INVALID_ARG, "yet_out is NULL");
  if (n_trials < 0) return fail(ctx, ARA_ERR_INVALID_ARG, "n_trials < 0");
  if (catalog_size <= 0) return fail(ctx, ARA_ERR_INVALID_ARG, "catalog_size <= 0");
  if (!trial_offsets) return fail(ctx, ARA_ERR_INVALID_ARG, "trial_offsets is NULL");
  ara_status s = set_device(ctx);
  if (s != ARA_OK) return s;
  // offsets are validated on the host (n_trials + 1 values)
  std::vector<int64_t> off((size_t)n_trials + 1);
  CUDA_TRY(ctx, cudaMemcpy(off.data(), trial_offsets, sizeof(int64_t) * off.size(),
                           cudaMemcpyDefault));
  if (off[0] != 0) return fail(ctx, ARA_ERR_INVALID_ARG, "trial_offsets[0] != 0");
  int64_t max_len = 0;
  for (int64_t i = 0; i < n_trials; ++i) {
    const int64_t len = off[(size_t)i + 1] - off[(size_t)i];
    if (len < 0) return fail(ctx, ARA_ERR_INVALID_ARG, "trial_offsets decrease at trial %lld",
                             (long long)i);
    if (len > max_len) max_len = len;
  }
  const int64_t n_occ = off[(size_t)n_trials];
  if (n_occ > 0 && (!event_ids || !timestamps))
    return fail(ctx, ARA_ERR_INVALID_ARG, "event_ids or timestamps is NULL");
  if (n_occ >= ((int64_t)1 << 40)) return fail(ctx, ARA_ERR_INVALID_ARG, "YET too large");
  YetDev y;
  y.n_trials = n_trials;
  y.n_occ = n_occ;
  y.catalog = catalog_size;
  y.max_len = max_len;
  cudaError_t e;
  if ((e = dev_alloc(&y.ids, n_occ)) != cudaSuccess || (e = dev_alloc(&y.ts, n_occ)) != cudaSuccess ||
      (e = dev_alloc(&y.offsets, n_trials + 1)) != cudaSuccess) {
    cudaGetLastError();
    free_yet(y);
    return fail(ctx, ARA_ERR_OOM, "YET of %lld occurrences: %s", (long long)n_occ,
                cudaGetErrorString(e));
  }
  if ((e = copy_in(y.ids, event_ids, n_occ, ctx->stream)) != cudaSuccess ||
      (e = copy_in(y.ts, timestamps, n_occ, ctx->stream)) != cudaSuccess ||
      (e = copy_in(y.offsets, off.data(), n_trials + 1, ctx->stream)) != cudaSuccess ||
      (e = cudaMemsetAsync(ctx->d_flags, 0, sizeof(unsigned int), ctx->stream)) != cudaSuccess ||
      (e = launch_validate_yet(y, ctx->d_flags, ctx->stream)) != cudaSuccess) {
    cudaGetLastError();
    free_yet(y);
    return fail(ctx, ARA_ERR_CUDA, "staging YET: %s", cudaGetErrorString(e));
  }
  unsigned int flags = 0;
  if ((e = cudaMemcpyAsync(&flags, ctx->d_flags, sizeof flags, cudaMemcpyDeviceToHost,
                           ctx->stream)) != cudaSuccess ||
      (e = cudaStreamSynchronize(ctx->stream)) != cudaSuccess) {
    cudaGetLastError();
    free_yet(y);
    return fail(ctx, ARA_ERR_CUDA, "staging YET: %s", cudaGetErrorString(e));
  }
  if (flags) {
    free_yet(y);
    return fail(ctx, ARA_ERR_INVALID_ARG, "YET rejected:%s%s%s",
                (flags & 1) ? " event id outside [0, catalog_size)" : "",
                (flags & 2) ? " timestamps decrease within a trial" : "",
                (flags & 4) ? " NaN timestamp" : "");
  }
  y.live = true;
  ctx->yets.push_back(y);
  *yet_out = (int32_t)ctx->yets.size() - 1;
  return ARA_OK;
}

ara_status ara_create_yet_host(ara_ctx* ctx, int64_t n_trials, const int64_t* trial_offsets,
                               const int32_t* event_ids, const float* timestamps,
                               int32_t catalog_size, int32_t* yet_out) {
  if (!ctx) return ARA_ERR_INVALID_ARG;
  if (!yet_out) return fail(ctx, ARA_ERR_INVALID_ARG, "yet_out is NULL");
  if (n_trials < 0) return fail(ctx, ARA_ERR_INVALID_ARG, "n_trials < 0");
  if (catalog_size <= 0) return fail(ctx, ARA_ERR_INVALID_ARG, "catalog_size <= 0");
  if (!trial_offsets) return fail(ctx, ARA_ERR_INVALID_ARG, "trial_offsets is NULL");
  if (is_device_ptr(trial_offsets) || (event_ids && is_device_ptr(event_ids)) ||
      (timestamps && is_device_ptr(timestamps)))
    return fail(ctx, ARA_ERR_INVALID_ARG, "a host-resident YET takes host arrays");
  ara_status s = set_device(ctx);
  if (s != ARA_OK) return s;
  YetDev y;
  y.host = true;
  y.h_off.assign(trial_offsets, trial_offsets + n_trials + 1);
  if (y.h_off[0] != 0) return fail(ctx, ARA_ERR_INVALID_ARG, "trial_offsets[0] != 0");
  int64_t max_len = 0;
  for (int64_t i = 0; i < n_trials; ++i) {
    const int64_t len = y.h_off[(size_t)i + 1] - y.h_off[(size_t)i];
    if (len < 0)
      return fail(ctx, ARA_ERR_INVALID_ARG, "trial_offsets decrease at trial %lld", (long long)i);
    max_len = std::max(max_len, len);
  }
  const int64_t n_occ = y.h_off[(size_t)n_trials];
  if (n_occ > 0 && (!event_ids || !timestamps))
    return fail(ctx, ARA_ERR_INVALID_ARG, "event_ids or timestamps is NULL");
  if (n_occ >= ((int64_t)1 << 40)) return fail(ctx, ARA_ERR_INVALID_ARG, "YET too large");
  y.n_trials = n_trials;
  y.n_occ = n_occ;
  y.catalog = catalog_size;
  y.max_len = max_len;
  y.h_ids = event_ids;
  y.h_ts = timestamps;
  cudaError_t e;
  if ((e = dev_alloc(&y.offsets, n_trials + 1)) != cudaSuccess ||
      (e = copy_in(y.offsets, y.h_off.data(), n_trials + 1, ctx->stream)) != cudaSuccess ||
      (e = cudaStreamSynchronize(ctx->stream)) != cudaSuccess) {
    cudaGetLastError();
    free_yet(y);
    return fail(ctx, ARA_ERR_CUDA, "staging YET offsets: %s", cudaGetErrorString(e));
  }
  y.live = true;
  ctx->yets.push_back(std::move(y));
  *yet_out = (int32_t)ctx->yets.size() - 1;
  return ARA_OK;
}

ara_status ara_free_yet(ara_ctx* ctx, int32_t yet) {
  if (!ctx) return ARA_ERR_INVALID_ARG;
  if (yet < 0 || yet >= (int32_t)ctx->yets.size() || !ctx->yets[yet].live)
    return fail(ctx, ARA_ERR_BAD_HANDLE, "bad YET handle %d", yet);
  for (auto& e : ctx->elts)
    if (e.live && e.yet == yet) return fail(ctx, ARA_ERR_INVALID_ARG, "YET still has ELTs");
  CUDA_TRY(ctx, cudaSetDevice(ctx->device));
  CUDA_TRY(ctx, cudaStreamSynchronize(ctx->stream));
  free_yet(ctx->yets[yet]);
  return ARA_OK;
}

// ---- ELT ------------------------------------------------------------------------------------
ara_status ara_add_elt_corr(ara_ctx* ctx, int32_t yet, int64_t n, const int32_t* event_ids,
                            const double* mean, const double* sd_indep, const double* sd_corr,
                            const double* max_exposure, int32_t* elt_out) {
  const double* sd = sd_indep;
  if (!ctx) return ARA_ERR_INVALID_ARG;
  if (!elt_out) return fail(ctx, ARA_ERR_INVALID_ARG, "elt_out is NULL");
  if (yet < 0 || yet >= (int32_t)ctx->yets.size() || !ctx->yets[yet].live)
    return fail(ctx, ARA_ERR_BAD_HANDLE, "bad YET handle %d", yet);
  if (n < 0 || n >= ((int64_t)1 << 31)) return fail(ctx, ARA_ERR_INVALID_ARG, "bad record count");
  if (n > 0 && (!event_ids || !mean || !sd || !max_exposure))
    return fail(ctx, ARA_ERR_INVALID_ARG, "NULL ELT array");
  ara_status s = set_device(ctx);
  if (s != ARA_OK) return s;
  const YetDev& y = ctx->yets[yet];
  const bool defer = ctx->table_policy == ARA_TABLES_ON_DEMAND;
  EltDev e;
  e.yet = yet;
  e.n = n;
  double *d_mean = nullptr, *d_sd = nullptr, *d_sdc = nullptr, *d_mx = nullptr;
  unsigned int* d_dup = nullptr;
  unsigned long long* d_uncert = nullptr;
  double2* d_ab64 = nullptr;
  unsigned long long uncert = 0;
  cudaError_t err;
  auto cleanup = [&]() {
    cudaStreamSynchronize(ctx->stream);
    dev_free(d_mean);
    dev_free(d_sd);
    dev_free(d_sdc);
    dev_free(d_mx);
    dev_free(d_dup);
    dev_free(d_uncert);
    if (!defer) dev_free(d_ab64);  // deferred tables keep (alpha, beta) in e.ab64
  };
  if ((err = dev_alloc(&e.ids, n)) != cudaSuccess || (err = dev_alloc(&e.recs, n)) != cudaSuccess ||
      (!defer && (err = dev_alloc(&e.tables, n * kTablePieces)) != cudaSuccess) ||
      (err = dev_alloc(&d_mean, n)) != cudaSuccess || (err = dev_alloc(&d_sd, n)) != cudaSuccess ||
      (err = dev_alloc(&d_mx, n)) != cudaSuccess || (err = dev_alloc(&d_dup, y.catalog)) != cudaSuccess ||
      (err = dev_alloc(&d_uncert, 1)) != cudaSuccess || (err = dev_alloc(&d_ab64, n)) != cudaSuccess ||
      (sd_corr && ((err = dev_alloc(&d_sdc, n)) != cudaSuccess ||
                   (err = dev_alloc(&e.corr, n)) != cudaSuccess))) {
    cudaGetLastError();
    if (defer) e.ab64 = d_ab64;
    cleanup();
    free_elt(e);
    return fail(ctx, ARA_ERR_OOM, "ELT of %lld records: %s", (long long)n, cudaGetErrorString(err));
  }
  if (defer) e.ab64 = d_ab64;
  unsigned int flags = 0;
  if ((err = copy_in(e.ids, event_ids, n, ctx->stream)) != cudaSuccess ||
      (err = copy_in(d_mean, mean, n, ctx->stream)) != cudaSuccess ||
      (err = copy_in(d_sd, sd, n, ctx->stream)) != cudaSuccess ||
      (sd_corr && (err = copy_in(d_sdc, sd_corr, n, ctx->stream)) != cudaSuccess) ||
      (err = copy_in(d_mx, max_exposure, n, ctx->stream)) != cudaSuccess ||
      (err = cudaMemsetAsync(d_dup, 0, sizeof(unsigned int) * (size_t)y.catalog, ctx->stream)) != cudaSuccess ||
      (err = cudaMemsetAsync(ctx->d_flags, 0, sizeof(unsigned int), ctx->stream)) != cudaSuccess ||
      (err = launch_prepare_elt(n, e.ids, d_mean, d_sd, d_sdc, d_mx, y.catalog, e.recs, d_ab64,
                                e.corr, d_dup, ctx->d_flags, ctx->stream)) != cudaSuccess ||
      (err = cudaMemsetAsync(d_uncert, 0, sizeof(unsigned long long), ctx->stream)) != cudaSuccess ||
      (!defer &&
       (err = launch_build_tables(n, e.recs, d_ab64, e.tables, d_uncert, ctx->stream)) != cudaSuccess) ||
      (err = cudaMemcpyAsync(&uncert, d_uncert, sizeof uncert, cudaMemcpyDeviceToHost,
                             ctx->stream)) != cudaSuccess ||
      (err = cudaMemcpyAsync(&flags, ctx->d_flags, sizeof flags, cudaMemcpyDeviceToHost,
                             ctx->stream)) != cudaSuccess ||
      (err = cudaStreamSynchronize(ctx->stream)) != cudaSuccess) {
    cudaGetLastError();
    cleanup();
    free_elt(e);
    return fail(ctx, ARA_ERR_CUDA, "staging ELT: %s", cudaGetErrorString(err));
  }
  cleanup();
  if (flags) {
    free_elt(e);
    return fail(ctx, ARA_ERR_INVALID_ARG, "ELT rejected:%s%s%s%s",
                (flags & 8) ? " event id outside the catalogue" : "",
                (flags & 16) ? " mean <= 0, an sd < 0 or non-finite value" : "",
                (flags & 32) ? " max_exposure <= mean with sd > 0" : "",
                (flags & 64) ? " duplicate event id" : "");
  }
  e.n_uncertified = (int64_t)uncert;
  e.live = true;
  ctx->elts.push_back(e);
  *elt_out = (int32_t)ctx->elts.size() - 1;
  return ARA_OK;
}

ara_status ara_add_elt(ara_ctx* ctx, int32_t yet, int64_t n, const int32_t* event_ids,
                       const double* mean, const double* sd, const double* max_exposure,
                       int32_t* elt_out) {
  return ara_add_elt_corr(ctx, yet, n, event_ids, mean, sd, nullptr, max_exposure, elt_out);
}

ara_status ara_free_elt(ara_ctx* ctx, int32_t elt) {
  if (!ctx) return ARA_ERR_INVALID_ARG;
  if (elt < 0 || elt >= (int32_t)ctx->elts.size() || !ctx->elts[elt].live)
    return fail(ctx, ARA_ERR_BAD_HANDLE, "bad ELT handle %d", elt);
  CUDA_TRY(ctx, cudaSetDevice(ctx->device));
  CUDA_TRY(ctx, cudaStreamSynchronize(ctx->stream));
  free_elt(ctx->elts[elt]);
  return ARA_OK;
}

// ---- layer ------------------------------------------------------------------------------------
}  // extern "C"

// Builds a layer; wide = true forces 16-byte index entries (two mask words) whatever the ELT
// count, the form the batched serving kernel takes.
ara_status ara_build_layer(ara_ctx* ctx, const int32_t* elts, int32_t n_elts, double occ_ret,
                           double occ_lim, double agg_ret, double agg_lim, bool wide,
                           cudaStream_t st, bool may_build_band, bool ordered,
                           LayerDev* out) {
  if (!ctx) return ARA_ERR_INVALID_ARG;
  if (!out || !elts) return fail(ctx, ARA_ERR_INVALID_ARG, "NULL argument");
  if (n_elts < 1 || n_elts > kMaxLayerElts)
    return fail(ctx, ARA_ERR_INVALID_ARG, "a layer covers 1..%d ELTs", kMaxLayerElts);
  const double terms[4] = {occ_ret, occ_lim, agg_ret, agg_lim};
  for (double t : terms)
    if (!(t >= 0.0) || !isfinite(t))
      return fail(ctx, ARA_ERR_INVALID_ARG, "layer terms must be finite and >= 0");
  int32_t yet = -1;
  for (int j = 0; j < n_elts; ++j) {
    const int32_t h = elts[j];
    if (h < 0 || h >= (int32_t)ctx->elts.size() || !ctx->elts[h].live)
      return fail(ctx, ARA_ERR_BAD_HANDLE, "bad ELT handle %d", h);
    for (int j2 = 0; j2 < j; ++j2)
      if (elts[j2] == h) return fail(ctx, ARA_ERR_INVALID_ARG, "ELT %d listed twice", h);
    if (yet < 0) yet = ctx->elts[h].yet;
    if (ctx->elts[h].yet != yet)
      return fail(ctx, ARA_ERR_INVALID_ARG, "ELTs of a layer must share one YET");
  }
  ara_status s = set_device(ctx);
  if (s != ARA_OK) return s;
  const int64_t C = ctx->yets[yet].catalog;
  LayerDev L;
  L.yet = yet;
  L.n_slots = n_elts;
  L.mask_words = (n_elts <= 32 && !wide) ? 1 : 2;
  for (int j = 0; j < kMaxLayerElts; ++j) L.handles[j] = j < n_elts ? elts[j] : 0;
  L.occ_ret = occ_ret;
  L.occ_lim = occ_lim;
  L.agg_ret = agg_ret;
  L.agg_lim = agg_lim;
  const int MW = L.mask_words;
  uint32_t *d_mask = nullptr, *d_cnt = nullptr, *d_base = nullptr, *d_tmp = nullptr;
  const int64_t tmp_words = scan_tmp_words(C);
  cudaError_t err;
  auto cleanup = [&]() {
    if (!ordered) cudaStreamSynchronize(st);
    mem_free(d_mask, ordered, st);
    mem_free(d_cnt, ordered, st);
    mem_free(d_base, ordered, st);
    mem_free(d_tmp, ordered, st);
  };
  const int64_t evt_words = C * (MW == 1 ? 2 : 4);
  if ((err = mem_alloc(&d_mask, C * MW, ordered, st)) != cudaSuccess || (err = mem_alloc(&d_cnt, C, ordered, st)) != cudaSuccess ||
      (err = mem_alloc(&d_base, C, ordered, st)) != cudaSuccess || (err = mem_alloc(&d_tmp, tmp_words, ordered, st)) != cudaSuccess ||
      (err = mem_alloc(&L.evt, evt_words, ordered, st)) != cudaSuccess) {
    cudaGetLastError();
    cleanup();
    free_layer_on(L, ordered, st);
    return fail(ctx, ARA_ERR_OOM, "layer index: %s", cudaGetErrorString(err));
  }
  uint32_t last[2] = {0, 0};
  err = cudaMemsetAsync(d_mask, 0, sizeof(uint32_t) * (size_t)(C * MW), st);
  for (int j = 0; j < n_elts && err == cudaSuccess; ++j)
    err = launch_layer_mask(ctx->elts[elts[j]], j, MW, d_mask, st);
  if (err == cudaSuccess) err = launch_layer_counts(d_mask, MW, C, d_cnt, st);
  if (err == cudaSuccess) err = launch_exclusive_scan_u32(d_cnt, d_base, C, d_tmp, tmp_words, st);
  if (err == cudaSuccess)
    err = cudaMemcpyAsync(&last[0], d_base + (C - 1), sizeof(uint32_t), cudaMemcpyDeviceToHost, st);
  if (err == cudaSuccess)
    err = cudaMemcpyAsync(&last[1], d_cnt + (C - 1), sizeof(uint32_t), cudaMemcpyDeviceToHost, st);
  if (err == cudaSuccess) err = launch_layer_index(d_mask, d_base, MW, C, L.evt, st);
  if (err == cudaSuccess) err = cudaStreamSynchronize(st);
  if (err != cudaSuccess) {
    cudaGetLastError();
    cleanup();
    free_layer_on(L, ordered, st);
    return fail(ctx, ARA_ERR_CUDA, "layer index: %s", cudaGetErrorString(err));
  }
  L.n_packed = (int64_t)last[0] + (int64_t)last[1];
  // packed records, then the records' tables copied into packed order (one gather per hit);
  // correlated weights only when some ELT of the layer has a correlated SD
  const TablePiece** d_src = nullptr;
  bool has_corr = false, all_tables = true;
  for (int j = 0; j < n_elts; ++j) {
    has_corr = has_corr || ctx->elts[elts[j]].corr != nullptr;
    all_tables = all_tables && ctx->elts[elts[j]].tables != nullptr;
  }
  if ((err = mem_alloc(&L.packed, L.n_packed, ordered, st)) != cudaSuccess ||
      (err = mem_alloc(&L.packed_rec, L.n_packed, ordered, st)) != cudaSuccess ||
      (all_tables && (err = mem_alloc(&L.tables, L.n_packed * kTablePieces, ordered, st)) !=
                         cudaSuccess) ||
      (err = mem_alloc(&d_src, L.n_packed, ordered, st)) != cudaSuccess ||
      (has_corr && (err = mem_alloc(&L.corr, L.n_packed, ordered, st)) != cudaSuccess)) {
    cudaGetLastError();
    cleanup();
    mem_free(d_src, ordered, st);
    free_layer_on(L, ordered, st);
    return fail(ctx, ARA_ERR_OOM, "layer records and tables: %s", cudaGetErrorString(err));
  }
  for (int j = 0; j < n_elts && err == cudaSuccess; ++j)
    err = launch_layer_scatter(ctx->elts[elts[j]], j, MW, L.evt, L.packed, d_src, L.packed_rec,
                               L.corr, st);
  if (err == cudaSuccess && all_tables) err = launch_gather_tables(L.n_packed, d_src, L.tables, st);
  if (err == cudaSuccess) err = cudaStreamSynchronize(st);
  cleanup();
  mem_free(d_src, ordered, st);
  if (err != cudaSuccess) {
    cudaGetLastError();
    free_layer_on(L, ordered, st);
    return fail(ctx, ARA_ERR_CUDA, "layer records: %s", cudaGetErrorString(err));
  }
  // band-major copy of the YET at this layer's band width (built once per width)
  const int log2w = ctx->band_log2w > 0 ? ctx->band_log2w : choose_band_log2w(C, L.n_packed);
  bool banded = false;
  if (may_build_band) {
    const ara_status bs = ensure_band_variant(ctx, yet, log2w, &banded);
    if (bs != ARA_OK) {
      free_layer_on(L, ordered, st);
      return bs;
    }
  } else {
    for (const auto& v : ctx->yets[yet].bands) banded = banded || v.log2w == log2w;
  }
  if (banded) L.band_log2w = log2w;
  L.live = true;
  *out = L;
  return ARA_OK;
}

ara_status ara_add_layer_impl(ara_ctx* ctx, const int32_t* elts, int32_t n_elts, double occ_ret,
                              double occ_lim, double agg_ret, double agg_lim, bool wide,
                              int32_t* layer_out) {
  if (!ctx) return ARA_ERR_INVALID_ARG;
  if (!layer_out) return fail(ctx, ARA_ERR_INVALID_ARG, "NULL argument");
  LayerDev L;
  const ara_status s = ara_build_layer(ctx, elts, n_elts, occ_ret, occ_lim, agg_ret, agg_lim,
                                       wide, ctx->stream, true, false, &L);
  if (s != ARA_OK) return s;
  ctx->layers.push_back(L);
  *layer_out = (int32_t)ctx->layers.size() - 1;
  return ARA_OK;
}

extern "C" {

ara_status ara_add_layer(ara_ctx* ctx, const int32_t* elts, int32_t n_elts, double occ_ret,
                         double occ_lim, double agg_ret, double agg_lim, int32_t* layer_out) {
  return ara_add_layer_impl(ctx, elts, n_elts, occ_ret, occ_lim, agg_ret, agg_lim, false,
                            layer_out);
}

ara_status ara_free_layer(ara_ctx* ctx, int32_t layer) {
  if (!ctx) return ARA_ERR_INVALID_ARG;
  if (layer < 0 || layer >= (int32_t)ctx->layers.size() || !ctx->layers[layer].live)
    return fail(ctx, ARA_ERR_BAD_HANDLE, "bad layer handle %d", layer);
  CUDA_TRY(ctx, cudaSetDevice(ctx->device));
  CUDA_TRY(ctx, cudaStreamSynchronize(ctx->stream));
  free_layer(ctx->layers[layer]);
  return ARA_OK;
}

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

}  // extern "C"

bool uses_band_schedule(const ara_ctx* ctx, const LayerDev& L) {
  return layer_inversion(ctx, L) == 0 && ctx->schedule == ARA_SCHED_BAND && L.band_log2w > 0 &&
         ctx->cfg.precision == ARA_ACC_FP64;
}

int layer_inversion(const ara_ctx* ctx, const LayerDev& L) {
  const int m = inversion_mode(ctx);
  return (m == 0 && L.tables == nullptr) ? 1 : m;
}

// The certified tables of one ELT, from the (alpha, beta) kept at staging.
static ara_status ensure_elt_tables(ara_ctx* ctx, EltDev& e) {
  if (e.tables) return ARA_OK;
  if (!e.ab64) return fail(ctx, ARA_ERR_INVALID_ARG, "ELT has neither tables nor parameters");
  unsigned long long* d_uncert = nullptr;
  unsigned long long uncert = 0;
  cudaError_t err;
  if ((err = dev_alloc(&e.tables, e.n * kTablePieces)) != cudaSuccess ||
      (err = dev_alloc(&d_uncert, 1)) != cudaSuccess) {
    cudaGetLastError();
    dev_free(e.tables);
    e.tables = nullptr;
    dev_free(d_uncert);
    return fail(ctx, ARA_ERR_OOM, "tables of %lld records", (long long)e.n);
  }
  if ((err = cudaMemsetAsync(d_uncert, 0, sizeof uncert, ctx->stream)) != cudaSuccess ||
      (err = launch_build_tables(e.n, e.recs, e.ab64, e.tables, d_uncert, ctx->stream)) !=
          cudaSuccess ||
      (err = cudaMemcpyAsync(&uncert, d_uncert, sizeof uncert, cudaMemcpyDeviceToHost,
                             ctx->stream)) != cudaSuccess ||
      (err = cudaStreamSynchronize(ctx->stream)) != cudaSuccess) {
    cudaGetLastError();
    cudaStreamSynchronize(ctx->stream);
    dev_free(e.tables);
    e.tables = nullptr;
    dev_free(d_uncert);
    return fail(ctx, ARA_ERR_CUDA, "building tables: %s", cudaGetErrorString(err));
  }
  dev_free(d_uncert);
  dev_free(e.ab64);
  e.ab64 = nullptr;
  e.n_uncertified = (int64_t)uncert;
  return ARA_OK;
}

// The layer's packed table copy (its ELTs' tables first).
static ara_status ensure_layer_tables(ara_ctx* ctx, LayerDev& L) {
  if (L.tables) return ARA_OK;
  for (int j = 0; j < L.n_slots; ++j) {
    const ara_status s = ensure_elt_tables(ctx, ctx->elts[L.handles[j]]);
    if (s != ARA_OK) return s;
  }
  const TablePiece** d_src = nullptr;
  cudaError_t err;
  if ((err = dev_alloc(&L.tables, L.n_packed * kTablePieces)) != cudaSuccess ||
      (err = dev_alloc(&d_src, L.n_packed)) != cudaSuccess) {
    cudaGetLastError();
    dev_free(L.tables);
    L.tables = nullptr;
    dev_free(d_src);
    return fail(ctx, ARA_ERR_OOM, "layer tables: %s", cudaGetErrorString(err));
  }
  // the scatter rewrites the packed records as they are and fills the table source pointers
  err = cudaSuccess;
  for (int j = 0; j < L.n_slots && err == cudaSuccess; ++j)
    err = launch_layer_scatter(ctx->elts[L.handles[j]], j, L.mask_words, L.evt, L.packed, d_src,
                               L.packed_rec, L.corr, ctx->stream);
  if (err == cudaSuccess) err = launch_gather_tables(L.n_packed, d_src, L.tables, ctx->stream);
  if (err == cudaSuccess) err = cudaStreamSynchronize(ctx->stream);
  dev_free(d_src);
  if (err != cudaSuccess) {
    cudaGetLastError();
    dev_free(L.tables);
    L.tables = nullptr;
    return fail(ctx, ARA_ERR_CUDA, "layer tables: %s", cudaGetErrorString(err));
  }
  return ARA_OK;
}

ara_status prepare_layer_for_run(ara_ctx* ctx, LayerDev& L, int64_t n) {
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
    if (!e.tables && e.rent_hits + per_rec < ARA_TABLE_BUY_HITS) buy = false;
  }
  if (buy) return ensure_layer_tables(ctx, L);
  for (int j = 0; j < L.n_slots; ++j) {
    EltDev& e = ctx->elts[L.handles[j]];
    if (!e.tables) e.rent_hits += per_rec;
  }
  return ARA_OK;
}

ara_status ensure_yet_tables(ara_ctx* ctx, int32_t yet) {
  for (auto& e : ctx->elts)
    if (e.live && e.yet == yet) {
      const ara_status s = ensure_elt_tables(ctx, e);
      if (s != ARA_OK) return s;
    }
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
  const unsigned long long top = 1ull << 53;  // year sums stay below 2^52 units
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
  const int qe = year_grid_exponent((float)L.occ_lim, Y.max_len);
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

extern "C" {

// A run over a host-resident YET: trials in chunks of whole trials (up to ctx->stream_chunk
// occurrences), each chunk's ids and timestamps copied on the copy stream into one of two device
// buffers while the previous chunk is validated and run on st; the run of a chunk skips its work
// if any chunk so far failed validation.  Outputs are device pointers for trials [t0, t0 + n).
static ara_status run_streamed(ara_ctx* ctx, const YetDev& Y, const LayerDev& L, int64_t t0,
                               int64_t n, double* d_ylt, double* d_oep, float* d_olt,
                               double* d_inc, cudaStream_t st) {
  const int64_t cap = std::max<int64_t>(ctx->stream_chunk, Y.max_len);
  if (cap > ctx->stream_cap) {
    for (int b = 0; b < 2; ++b) {
      dev_free(ctx->d_sids[b]);
      dev_free(ctx->d_sts[b]);
      ctx->d_sids[b] = nullptr;
      ctx->d_sts[b] = nullptr;
    }
    ctx->stream_cap = 0;
    for (int b = 0; b < 2; ++b)
      CUDA_TRY(ctx, dev_alloc(&ctx->d_sids[b], cap));
    for (int b = 0; b < 2; ++b)
      CUDA_TRY(ctx, dev_alloc(&ctx->d_sts[b], cap));
    ctx->stream_cap = cap;
  }
  if (!ctx->copy_stream)
    CUDA_TRY(ctx, cudaStreamCreateWithFlags(&ctx->copy_stream, cudaStreamNonBlocking));
  for (int b = 0; b < 2; ++b) {
    if (!ctx->ev_ready[b])
      CUDA_TRY(ctx, cudaEventCreateWithFlags(&ctx->ev_ready[b], cudaEventDisableTiming));
    if (!ctx->ev_free[b])
      CUDA_TRY(ctx, cudaEventCreateWithFlags(&ctx->ev_free[b], cudaEventDisableTiming));
    CUDA_TRY(ctx, cudaEventRecord(ctx->ev_free[b], st));  // both buffers free once st gets here
  }
  CUDA_TRY(ctx, cudaMemsetAsync(ctx->d_flags, 0, sizeof(unsigned int), st));
  const int64_t q_first = Y.h_off[(size_t)t0];
  int k = 0;
  for (int64_t tb = t0; tb < t0 + n; ++k) {
    int64_t te = tb + 1;  // whole trials up to cap occurrences (a trial never exceeds cap)
    while (te < t0 + n && Y.h_off[(size_t)te + 1] - Y.h_off[(size_t)tb] <= cap) ++te;
    const int64_t ob = Y.h_off[(size_t)tb], len = Y.h_off[(size_t)te] - ob;
    const int b = k & 1;
    CUDA_TRY(ctx, cudaStreamWaitEvent(ctx->copy_stream, ctx->ev_free[b], 0));
    if (len > 0) {
      CUDA_TRY(ctx, cudaMemcpyAsync(ctx->d_sids[b], Y.h_ids + ob, sizeof(int32_t) * (size_t)len,
                                    cudaMemcpyHostToDevice, ctx->copy_stream));
      CUDA_TRY(ctx, cudaMemcpyAsync(ctx->d_sts[b], Y.h_ts + ob, sizeof(float) * (size_t)len,
                                    cudaMemcpyHostToDevice, ctx->copy_stream));
    }
    CUDA_TRY(ctx, cudaEventRecord(ctx->ev_ready[b], ctx->copy_stream));
    CUDA_TRY(ctx, cudaStreamWaitEvent(st, ctx->ev_ready[b], 0));
    CUDA_TRY(ctx, launch_validate_yet_range(ctx->d_sids[b], ctx->d_sts[b], ob, Y.offsets, tb,
                                            te - tb, Y.catalog, ctx->d_flags, st));
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
  OrderedTemp tmp_olt{nullptr, st}, tmp_inc{nullptr, st};  // host outputs' device staging
  if (!dev_out) {
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
        CUDA_TRY(ctx, mem_alloc(&d_olt, n_occ, true, st));
        tmp_olt.p = d_olt;
      }
      if (inc) {
        CUDA_TRY(ctx, mem_alloc(&d_inc, n_occ, true, st));
        tmp_inc.p = d_inc;
      }
    }
  }
  unsigned long long nc_before = 0;
  if (!stream)
    CUDA_TRY(ctx, cudaMemcpyAsync(&nc_before, ctx->d_not_conv, sizeof nc_before,
                                  cudaMemcpyDeviceToHost, st));
  s = prepare_layer_for_run(ctx, ctx->layers[layer], n);
  if (s != ARA_OK) return s;
  TrialParams p = make_params(ctx, Y, ctx->layers[layer], t0, n, d_ylt);
  p.oep = d_oep;
  p.olt = d_olt;
  p.inc = d_inc;
  // per-occurrence outputs are written in trial order, so they keep the trial-major schedule
  if (Y.host) {
    s = run_streamed(ctx, Y, ctx->layers[layer], t0, n, d_ylt, d_oep, d_olt, d_inc, st);
    if (s != ARA_OK) return s;
  } else if (!per_occ && uses_band_schedule(ctx, ctx->layers[layer])) {
    // year sums (8 B per trial), then the OEP maxima (4 B per trial) in the same scratch
    s = ensure_ysum(ctx, oep ? n + (n + 1) / 2 : n);
    if (s != ARA_OK) return s;
    p.ysum = ctx->d_ysum;
    p.omax = oep ? reinterpret_cast<unsigned int*>(ctx->d_ysum + n) : nullptr;
    CUDA_TRY(ctx, launch_band(p, ctx->layers[layer].mask_words, ctx->cfg.precision, st));
  } else {
    CUDA_TRY(ctx, launch_trial(p, ctx->layers[layer].mask_words, ctx->cfg.precision,
                               layer_inversion(ctx, ctx->layers[layer]), false, st));
  }
  if (stream) return ARA_OK;
  if (!dev_out) {
    CUDA_TRY(ctx, cudaMemcpyAsync(ylt, d_ylt, sizeof(double) * (size_t)n, cudaMemcpyDeviceToHost,
                                  st));
    if (oep)
      CUDA_TRY(ctx, cudaMemcpyAsync(oep, d_oep, sizeof(double) * (size_t)n,
                                    cudaMemcpyDeviceToHost, st));
    if (olt && n_occ > 0)
      CUDA_TRY(ctx, cudaMemcpyAsync(olt, d_olt, sizeof(float) * (size_t)n_occ,
                                    cudaMemcpyDeviceToHost, st));
    if (inc && n_occ > 0)
      CUDA_TRY(ctx, cudaMemcpyAsync(inc, d_inc, sizeof(double) * (size_t)n_occ,
                                    cudaMemcpyDeviceToHost, st));
  }
  unsigned long long nc_after = 0;
  unsigned int yet_flags = 0;
  CUDA_TRY(ctx, cudaMemcpyAsync(&nc_after, ctx->d_not_conv, sizeof nc_after,
                                cudaMemcpyDeviceToHost, st));
  if (Y.host)
    CUDA_TRY(ctx, cudaMemcpyAsync(&yet_flags, ctx->d_flags, sizeof yet_flags,
                                  cudaMemcpyDeviceToHost, st));
  CUDA_TRY(ctx, cudaStreamSynchronize(st));
  if (yet_flags)
    return fail(ctx, ARA_ERR_INVALID_ARG, "YET rejected:%s%s%s",
                (yet_flags & 1) ? " event id outside [0, catalog_size)" : "",
                (yet_flags & 2) ? " timestamps decrease within a trial" : "",
                (yet_flags & 4) ? " NaN timestamp" : "");
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
    ara_status s = prepare_layer_for_run(ctx, ctx->layers[layers[i]], n);
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
  const int64_t big_blocks = 12ll * ctx->sm_count * 4;
  int32_t n_items = 0;
  for (int32_t k = 0; k < n_layers; ++k) {
    const int32_t i = order[k];
    const LayerDev& L = ctx->layers[layers[i]];
    TrialParams p = make_params(ctx, Y, L, t0, n, d_ylt + (int64_t)i * n);
    const bool band = group(i) < 2;
    const int64_t own_blocks = band ? (int64_t)p.n_bands * band_tiles(n) : (n + 7) / 8;
    if (own_blocks >= big_blocks) {
      if (band) {
        p.ysum = ctx->d_ysum + (int64_t)band_row++ * n;
        CUDA_TRY(ctx, launch_band(p, L.mask_words, ctx->cfg.precision, st));
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
  CUDA_TRY(ctx, mem_alloc(&d_items, n_layers, true, st));
  OrderedTemp tmp_items{d_items, st};
  CUDA_TRY(ctx, mem_alloc(&d_begin, 3 * (int64_t)n_layers, true, st));
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

// ---- ordering and risk measures -------------------------------------------------------------
static ara_status stage_and_sort(ara_ctx* ctx, const double* ylt, int64_t n, const double** d_y,
                                 const uint32_t** d_order) {
  CUDA_TRY(ctx, cudaSetDevice(ctx->device));
  if (n >= ((int64_t)1 << 32)) return fail(ctx, ARA_ERR_INVALID_ARG, "YLT too long");
  ara_status s = ensure_sort(ctx, n);
  if (s != ARA_OK) return s;
  const double* dy = ylt;
  if (!is_device_ptr(ylt)) {
    s = ensure_ylt_tmp(ctx, n);
    if (s != ARA_OK) return s;
    CUDA_TRY(ctx, cudaMemcpyAsync(ctx->d_ylt_tmp, ylt, sizeof(double) * (size_t)n,
                                  cudaMemcpyHostToDevice, ctx->stream));
    dy = ctx->d_ylt_tmp;
  }
  int which = 0;
  cudaError_t e = sort_ylt_desc(dy, n, ctx->sort, &which, ctx->stream);
  if (e == cudaErrorInvalidValue) return fail(ctx, ARA_ERR_INVALID_ARG, "NaN in the YLT");
  CUDA_TRY(ctx, e);
  *d_y = dy;
  *d_order = ctx->sort.vals[which];
  return ARA_OK;
}

static ara_status risk_measures_impl(ara_ctx* ctx, const double* ylt, int64_t n, int64_t n_total,
                                     const double* rps, int32_t m, double* pml, double* tvar) {
  if (!ctx) return ARA_ERR_INVALID_ARG;
  if (n < 1 || !ylt) return fail(ctx, ARA_ERR_INVALID_ARG, "empty YLT");
  if (n_total < n) return fail(ctx, ARA_ERR_INVALID_ARG, "n_total below the number of values");
  if (m < 0 || m > 128 || (m > 0 && (!rps || !pml || !tvar)))
    return fail(ctx, ARA_ERR_INVALID_ARG, "bad return-period list");
  int64_t ks[128];
  for (int q = 0; q < m; ++q) {
    if (!(rps[q] > 1.0) || !isfinite(rps[q]))
      return fail(ctx, ARA_ERR_INVALID_ARG, "return periods must be finite and > 1");
    ks[q] = tail_count(n_total, rps[q]);
    if (ks[q] > n)
      return fail(ctx, ARA_ERR_INVALID_ARG, "1-in-%g needs the %lld largest of %lld trials, "
                  "only %lld values given", rps[q], (long long)ks[q], (long long)n_total,
                  (long long)n);
  }
  const double* dy;
  const uint32_t* order;
  ara_status s = stage_and_sort(ctx, ylt, n, &dy, &order);
  if (s != ARA_OK) return s;
  if (m == 0) return ARA_OK;
  int64_t* d_k = reinterpret_cast<int64_t*>(ctx->d_misc);
  double* d_pml = reinterpret_cast<double*>(d_k + 128);
  double* d_tvar = d_pml + 128;
  CUDA_TRY(ctx, cudaMemcpyAsync(d_k, ks, sizeof(int64_t) * m, cudaMemcpyHostToDevice, ctx->stream));
  CUDA_TRY(ctx, launch_tail_sums(dy, order, n, d_k, m, d_pml, d_tvar, ctx->stream));
  std::vector<double> hp(m), ht(m);
  CUDA_TRY(ctx, cudaMemcpyAsync(hp.data(), d_pml, sizeof(double) * m, cudaMemcpyDeviceToHost, ctx->stream));
  CUDA_TRY(ctx, cudaMemcpyAsync(ht.data(), d_tvar, sizeof(double) * m, cudaMemcpyDeviceToHost, ctx->stream));
  CUDA_TRY(ctx, cudaStreamSynchronize(ctx->stream));
  for (int q = 0; q < m; ++q) {
    pml[q] = hp[q];
    tvar[q] = ht[q];
  }
  return ARA_OK;
}

ara_status ara_risk_measures(ara_ctx* ctx, const double* ylt, int64_t n, const double* rps,
                             int32_t m, double* pml, double* tvar) {
  return risk_measures_impl(ctx, ylt, n, n, rps, m, pml, tvar);
}

ara_status ara_risk_measures_n(ara_ctx* ctx, const double* values, int64_t n, int64_t n_total,
                               const double* rps, int32_t m, double* pml, double* tvar) {
  return risk_measures_impl(ctx, values, n, n_total, rps, m, pml, tvar);
}

ara_status ara_top_k(ara_ctx* ctx, const double* ylt, int64_t n, int64_t k, double* out) {
  if (!ctx) return ARA_ERR_INVALID_ARG;
  if (n < 1 || !ylt || !out) return fail(ctx, ARA_ERR_INVALID_ARG, "empty YLT or NULL output");
  if (k < 0 || k > n) return fail(ctx, ARA_ERR_INVALID_ARG, "k outside [0, n]");
  const double* dy;
  const uint32_t* order;
  ara_status s = stage_and_sort(ctx, ylt, n, &dy, &order);
  if (s != ARA_OK) return s;
  if (k == 0) return ARA_OK;
  if (n > ctx->sel_cap) {
    dev_free(ctx->d_sel);
    ctx->d_sel = nullptr;
    ctx->sel_cap = 0;
    CUDA_TRY(ctx, dev_alloc(&ctx->d_sel, 2 * n + scan_tmp_words(n)));
    ctx->sel_cap = n;
  }
  uint32_t* flags = ctx->d_sel;
  uint32_t* pos = flags + n;
  uint32_t* tmp = pos + n;
  const bool dev_out = is_device_ptr(out);
  double* d_out = out;
  if (!dev_out) {  // the key buffer the sort is not holding its result in (n * 8 bytes)
    d_out = reinterpret_cast<double*>(order == ctx->sort.vals[0] ? ctx->sort.keys[1]
                                                                  : ctx->sort.keys[0]);
  }
  CUDA_TRY(ctx, launch_top_k_in_index_order(dy, order, n, k, flags, pos, tmp,
                                             scan_tmp_words(n), d_out, ctx->stream));
  if (!dev_out)
    CUDA_TRY(ctx, cudaMemcpyAsync(out, d_out, sizeof(double) * (size_t)k, cudaMemcpyDeviceToHost,
                                  ctx->stream));
  CUDA_TRY(ctx, cudaStreamSynchronize(ctx->stream));
  return ARA_OK;
}

ara_status ara_rank_ylt(ara_ctx* ctx, const double* ylt, int64_t n, int64_t* order) {
  if (!ctx) return ARA_ERR_INVALID_ARG;
  if (n < 1 || !ylt || !order) return fail(ctx, ARA_ERR_INVALID_ARG, "empty YLT or NULL order");
  const double* dy;
  const uint32_t* d_order;
  ara_status s = stage_and_sort(ctx, ylt, n, &dy, &d_order);
  if (s != ARA_OK) return s;
  if (is_device_ptr(order)) {
    CUDA_TRY(ctx, launch_order_to_i64(d_order, n, order, ctx->stream));
  } else {
    // stage through the key buffer the sort is not holding its result in (n * 8 bytes)
    int64_t* tmp = reinterpret_cast<int64_t*>(d_order == ctx->sort.vals[0] ? ctx->sort.keys[1]
                                                                            : ctx->sort.keys[0]);
    CUDA_TRY(ctx, launch_order_to_i64(d_order, n, tmp, ctx->stream));
    CUDA_TRY(ctx, cudaMemcpyAsync(order, tmp, sizeof(int64_t) * (size_t)n, cudaMemcpyDeviceToHost,
                                  ctx->stream));
  }
  CUDA_TRY(ctx, cudaStreamSynchronize(ctx->stream));
  return ARA_OK;
}

// ---- verification trace ------------------------------------------------------------------------
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
  const LayerDev& L = ctx->layers[layer];
  const int64_t cap = std::max<int64_t>(1, Y.max_len * L.n_slots);
  const int64_t total = n * cap;
  if (total > ((int64_t)1 << 27)) return fail(ctx, ARA_ERR_INVALID_ARG, "trace too large");
  if (n == 0) {
    *n_hits = 0;
    return ARA_OK;
  }
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

// ---- learned surrogate ----------------------------------------------------------------------------
namespace {

ara_status mlp_alloc(ara_ctx* ctx) {
  if (ctx->mlp_P) return ARA_OK;
  CUDA_TRY(ctx, dev_alloc(&ctx->mlp_P, kMlpParams));
  CUDA_TRY(ctx, dev_alloc(&ctx->mlp_M, kMlpParams));
  CUDA_TRY(ctx, dev_alloc(&ctx->mlp_V, kMlpParams));
  CUDA_TRY(ctx, dev_alloc(&ctx->mlp_G, kMlpParams));
  CUDA_TRY(ctx, cudaMalloc(&ctx->mlp_W, sizeof(MlpDevWeights)));
  CUDA_TRY(ctx, dev_alloc(&ctx->mlp_bound, kCertCells));
  return ARA_OK;
}

// Uniform(-1/sqrt(fan_in), 1/sqrt(fan_in)) weights and biases, seeded.
void init_params(std::vector<float>& p, uint64_t seed) {
  std::mt19937_64 rng(seed ^ 0x9E3779B97F4A7C15ull);
  std::uniform_real_distribution<double> U(-1.0, 1.0);
  p.assign(kMlpParams, 0.0f);
  const int fans[4][2] = {{kH, 3}, {kH, kH}, {kH, kH}, {1, kH}};
  int o = 0;
  for (auto& f : fans) {
    const double bnd = 1.0 / std::sqrt((double)f[1]);
    for (int i = 0; i < f[0] * f[1] + f[0]; ++i) p[o++] = (float)(bnd * U(rng));
  }
}

struct MlpBuffers {
  MlpScratch s;
  void free_all() {
    dev_free(s.HT0); dev_free(s.HT1); dev_free(s.HT2); dev_free(s.HT3);
    dev_free(s.DZT1); dev_free(s.DZT2); dev_free(s.DZT3);
    s = MlpScratch();
  }
};

cudaError_t mlp_scratch(MlpBuffers& b, int64_t B, cudaStream_t st) {
  b.s.B = B;
  cudaError_t e;
  if ((e = dev_alloc(&b.s.HT0, 8 * B)) != cudaSuccess) return e;
  if ((e = cudaMemsetAsync(b.s.HT0, 0, sizeof(__nv_bfloat16) * 8 * B, st)) != cudaSuccess) return e;
  __nv_bfloat16** big[] = {&b.s.HT1, &b.s.HT2, &b.s.HT3, &b.s.DZT1, &b.s.DZT2, &b.s.DZT3};
  for (auto p : big)
    if ((e = dev_alloc(p, (int64_t)kH * B)) != cudaSuccess) return e;
  return cudaSuccess;
}

float percentile(std::vector<float> v, double q) {
  if (v.empty()) return 0.0f;
  const size_t k = std::min(v.size() - 1, (size_t)(q * (double)(v.size() - 1)));
  std::nth_element(v.begin(), v.begin() + k, v.end());
  return v[k];
}

// Certifies the network held in ctx->mlp_W: fills ctx->mlp_bound.
ara_status mlp_certify(ara_ctx* ctx, int samples, uint64_t seed, ara_surrogate_report* rep,
                       float eps) {
  const int64_t n = kCertCells * samples;
  float *Z = nullptr, *X = nullptr, *Y = nullptr;
  unsigned int* bad = nullptr;
  auto cleanup = [&]() {
    cudaStreamSynchronize(ctx->stream);
    dev_free(Z); dev_free(X); dev_free(Y); dev_free(bad);
  };
  cudaError_t e;
  if ((e = dev_alloc(&Z, 3 * n)) != cudaSuccess || (e = dev_alloc(&X, n)) != cudaSuccess ||
      (e = dev_alloc(&Y, n)) != cudaSuccess || (e = dev_alloc(&bad, 1)) != cudaSuccess ||
      (e = cudaMemsetAsync(bad, 0, sizeof(unsigned int), ctx->stream)) != cudaSuccess ||
      (e = launch_mlp_cert_points(kCertCells, samples, seed, Z, X, bad, ctx->stream)) != cudaSuccess ||
      (e = launch_mlp_eval(ctx->mlp_W, Z, n, Y, ctx->stream)) != cudaSuccess ||
      (e = launch_mlp_cert_reduce(kCertCells, samples, X, Y, ctx->mlp_bound, ctx->stream)) != cudaSuccess) {
    cudaGetLastError();
    cleanup();
    return fail(ctx, ARA_ERR_CUDA, "surrogate certification: %s", cudaGetErrorString(e));
  }
  std::vector<float> b(kCertCells);
  e = cudaMemcpyAsync(b.data(), ctx->mlp_bound, sizeof(float) * kCertCells, cudaMemcpyDeviceToHost,
                      ctx->stream);
  if (e == cudaSuccess) e = cudaStreamSynchronize(ctx->stream);
  cleanup();
  if (e != cudaSuccess) return fail(ctx, ARA_ERR_CUDA, "surrogate certification: %s", cudaGetErrorString(e));
  if (rep) {
    int64_t acc = 0;
    for (float v : b) acc += v <= eps;
    rep->cells_accepted = (double)acc / (double)kCertCells;
    rep->err_median = percentile(b, 0.5);
    rep->err_p99 = percentile(b, 0.99);
  }
  return ARA_OK;
}

// Parameters into a BF16 image: the context's own (params == NULL) or caller values.
ara_status mlp_image(ara_ctx* ctx, const float* params, MlpDevWeights** out, float** tmpP) {
  *tmpP = nullptr;
  if (!params) {
    if (!ctx->mlp_ready) return fail(ctx, ARA_ERR_INVALID_ARG, "no surrogate trained or loaded");
    *out = ctx->mlp_W;
    return ARA_OK;
  }
  MlpDevWeights* w = nullptr;
  CUDA_TRY(ctx, dev_alloc(tmpP, kMlpParams));
  CUDA_TRY(ctx, cudaMalloc(&w, sizeof(MlpDevWeights)));
  CUDA_TRY(ctx, cudaMemcpyAsync(*tmpP, params, sizeof(float) * kMlpParams, cudaMemcpyDefault, ctx->stream));
  CUDA_TRY(ctx, launch_mlp_pack(*tmpP, w, ctx->stream));
  *out = w;
  return ARA_OK;
}

}  // namespace

extern "C" {

ara_status ara_train_surrogate(ara_ctx* ctx, const ara_surrogate_config* cfg,
                               ara_surrogate_report* report) {
  if (!ctx) return ARA_ERR_INVALID_ARG;
  if (!cfg || cfg->n_samples < cfg->batch || cfg->batch < 128 || cfg->batch % 128 != 0 ||
      cfg->steps < 1 || cfg->cert_samples < 8 || !(cfg->lr > 0.0f) || !(cfg->lr_final > 0.0f) ||
      !(cfg->eps > 0.0f))
    return fail(ctx, ARA_ERR_INVALID_ARG, "bad surrogate training configuration");
  CUDA_TRY(ctx, cudaSetDevice(ctx->device));
  ara_status s = mlp_alloc(ctx);
  if (s != ARA_OK) return s;
  ara_surrogate_report rep{};
  const int64_t N = cfg->n_samples / cfg->batch * cfg->batch;
  float *Z = nullptr, *X = nullptr, *T = nullptr, *loss = nullptr;
  unsigned int* bad = nullptr;
  MlpBuffers buf;
  cudaEvent_t ev[4] = {nullptr, nullptr, nullptr, nullptr};
  auto cleanup = [&]() {
    cudaStreamSynchronize(ctx->stream);
    dev_free(Z); dev_free(X); dev_free(T); dev_free(loss); dev_free(bad);
    buf.free_all();
    for (auto& e : ev)
      if (e) cudaEventDestroy(e);
  };
  cudaError_t e = cudaSuccess;
  for (auto& x : ev)
    if (e == cudaSuccess) e = cudaEventCreate(&x);
  const int64_t n_loss = cfg->steps + 1;
  if (e == cudaSuccess) e = dev_alloc(&Z, 3 * N);
  if (e == cudaSuccess) e = dev_alloc(&X, N);
  if (e == cudaSuccess) e = dev_alloc(&T, N);
  if (e == cudaSuccess) e = dev_alloc(&loss, n_loss);
  if (e == cudaSuccess) e = dev_alloc(&bad, 1);
  if (e == cudaSuccess) e = mlp_scratch(buf, cfg->batch, ctx->stream);
  if (e != cudaSuccess) {
    cudaGetLastError();
    cleanup();
    return fail(ctx, ARA_ERR_OOM, "surrogate training buffers: %s", cudaGetErrorString(e));
  }
  std::vector<float> p0;
  init_params(p0, cfg->seed);
  e = cudaMemsetAsync(bad, 0, sizeof(unsigned int), ctx->stream);
  if (e == cudaSuccess) e = cudaMemsetAsync(loss, 0, sizeof(float) * n_loss, ctx->stream);
  if (e == cudaSuccess) e = cudaEventRecord(ev[0], ctx->stream);
  const int64_t gen_chunk = 1 << 24;
  for (int64_t f = 0; f < N && e == cudaSuccess; f += gen_chunk)
    e = launch_mlp_gen(std::min(gen_chunk, N - f), cfg->seed, f, Z + 3 * f, X + f, T + f, bad,
                       ctx->stream);
  if (e == cudaSuccess) e = cudaEventRecord(ev[1], ctx->stream);
  if (e == cudaSuccess)
    e = cudaMemcpyAsync(ctx->mlp_P, p0.data(), sizeof(float) * kMlpParams, cudaMemcpyHostToDevice,
                        ctx->stream);
  for (float* q : {ctx->mlp_M, ctx->mlp_V, ctx->mlp_G})
    if (e == cudaSuccess) e = cudaMemsetAsync(q, 0, sizeof(float) * kMlpParams, ctx->stream);
  if (e == cudaSuccess) e = launch_mlp_pack(ctx->mlp_P, ctx->mlp_W, ctx->stream);
  const int64_t per_epoch = N / cfg->batch;
  const double pi = 3.14159265358979323846;
  for (int64_t step = 1; step <= cfg->steps && e == cudaSuccess; ++step) {
    const int64_t b = (step - 1) % per_epoch;
    e = launch_mlp_step(ctx->mlp_W, Z + 3 * b * cfg->batch, X + b * cfg->batch,
                        T + b * cfg->batch, cfg->batch, buf.s, ctx->mlp_G, loss + step,
                        ctx->stream);
    const double frac = (double)(step - 1) / (double)std::max<int64_t>(1, cfg->steps - 1);
    const float lr = (float)(cfg->lr_final + 0.5 * (cfg->lr - cfg->lr_final) * (1.0 + std::cos(pi * frac)));
    if (e == cudaSuccess)
      e = launch_mlp_adam(ctx->mlp_P, ctx->mlp_M, ctx->mlp_V, ctx->mlp_G, lr, step, ctx->stream);
    if (e == cudaSuccess) e = launch_mlp_pack(ctx->mlp_P, ctx->mlp_W, ctx->stream);
  }
  if (e == cudaSuccess) e = cudaEventRecord(ev[2], ctx->stream);
  std::vector<float> hl(n_loss);
  unsigned int hbad = 0;
  if (e == cudaSuccess)
    e = cudaMemcpyAsync(hl.data(), loss, sizeof(float) * n_loss, cudaMemcpyDeviceToHost, ctx->stream);
  if (e == cudaSuccess)
    e = cudaMemcpyAsync(&hbad, bad, sizeof hbad, cudaMemcpyDeviceToHost, ctx->stream);
  if (e == cudaSuccess) e = cudaStreamSynchronize(ctx->stream);
  if (e != cudaSuccess) {
    cudaGetLastError();
    cleanup();
    return fail(ctx, ARA_ERR_CUDA, "surrogate training: %s", cudaGetErrorString(e));
  }
  ctx->mlp_ready = true;
  ctx->mlp_eps = cfg->eps;
  s = mlp_certify(ctx, cfg->cert_samples, cfg->seed + 1, &rep, cfg->eps);
  if (s != ARA_OK) {
    ctx->mlp_ready = false;
    cleanup();
    return s;
  }
  cudaEventRecord(ev[3], ctx->stream);
  cudaStreamSynchronize(ctx->stream);
  float ms = 0.f;
  cudaEventElapsedTime(&ms, ev[0], ev[1]);
  rep.gen_ms = ms;
  cudaEventElapsedTime(&ms, ev[1], ev[2]);
  rep.train_ms = ms;
  cudaEventElapsedTime(&ms, ev[2], ev[3]);
  rep.cert_ms = ms;
  const int64_t w = std::max<int64_t>(1, cfg->steps / 100);
  double a = 0, z = 0;
  for (int64_t i = 1; i <= w; ++i) {
    a += hl[i];
    z += hl[cfg->steps + 1 - i];
  }
  rep.loss_first = a / w;
  rep.loss_last = z / w;
  rep.bad_targets = hbad;
  cleanup();
  if (report) *report = rep;
  return ARA_OK;
}

ara_status ara_set_surrogate_eps(ara_ctx* ctx, float eps) {
  if (!ctx) return ARA_ERR_INVALID_ARG;
  if (!(eps > 0.0f)) return fail(ctx, ARA_ERR_INVALID_ARG, "eps must be > 0");
  ctx->mlp_eps = eps;
  return ARA_OK;
}

static const uint32_t kBlobMagic = 0x53524741u;  // "AGRS"
struct BlobHeader {
  uint32_t magic, version;
  int32_t n_params, n_cells;
  float eps;
  uint32_t pad[3];
};

ara_status ara_save_surrogate(ara_ctx* ctx, void* blob, size_t cap, size_t* bytes) {
  if (!ctx || !bytes) return ARA_ERR_INVALID_ARG;
  const size_t need = sizeof(BlobHeader) + sizeof(float) * (kMlpParams + kCertCells);
  *bytes = need;
  if (!ctx->mlp_ready) return fail(ctx, ARA_ERR_INVALID_ARG, "no surrogate trained or loaded");
  if (!blob) return ARA_OK;
  if (cap < need) return fail(ctx, ARA_ERR_INVALID_ARG, "blob needs %zu bytes", need);
  CUDA_TRY(ctx, cudaSetDevice(ctx->device));
  BlobHeader h{kBlobMagic, 1, kMlpParams, (int32_t)kCertCells, ctx->mlp_eps, {0, 0, 0}};
  char* o = static_cast<char*>(blob);
  memcpy(o, &h, sizeof h);
  CUDA_TRY(ctx, cudaMemcpyAsync(o + sizeof h, ctx->mlp_P, sizeof(float) * kMlpParams,
                                cudaMemcpyDeviceToHost, ctx->stream));
  CUDA_TRY(ctx, cudaMemcpyAsync(o + sizeof h + sizeof(float) * kMlpParams, ctx->mlp_bound,
                                sizeof(float) * kCertCells, cudaMemcpyDeviceToHost, ctx->stream));
  CUDA_TRY(ctx, cudaStreamSynchronize(ctx->stream));
  return ARA_OK;
}

ara_status ara_load_surrogate(ara_ctx* ctx, const void* blob, size_t bytes) {
  if (!ctx) return ARA_ERR_INVALID_ARG;
  const size_t need = sizeof(BlobHeader) + sizeof(float) * (kMlpParams + kCertCells);
  if (!blob || bytes < need) return fail(ctx, ARA_ERR_INVALID_ARG, "surrogate blob too short");
  BlobHeader h;
  memcpy(&h, blob, sizeof h);
  if (h.magic != kBlobMagic || h.version != 1 || h.n_params != kMlpParams ||
      h.n_cells != (int32_t)kCertCells || !(h.eps > 0.0f))
    return fail(ctx, ARA_ERR_INVALID_ARG, "not a surrogate blob of this library");
  CUDA_TRY(ctx, cudaSetDevice(ctx->device));
  ara_status s = mlp_alloc(ctx);
  if (s != ARA_OK) return s;
  const char* in = static_cast<const char*>(blob);
  CUDA_TRY(ctx, cudaMemcpyAsync(ctx->mlp_P, in + sizeof h, sizeof(float) * kMlpParams,
                                cudaMemcpyHostToDevice, ctx->stream));
  CUDA_TRY(ctx, cudaMemcpyAsync(ctx->mlp_bound, in + sizeof h + sizeof(float) * kMlpParams,
                                sizeof(float) * kCertCells, cudaMemcpyHostToDevice, ctx->stream));
  CUDA_TRY(ctx, launch_mlp_pack(ctx->mlp_P, ctx->mlp_W, ctx->stream));
  CUDA_TRY(ctx, cudaStreamSynchronize(ctx->stream));
  ctx->mlp_eps = h.eps;
  ctx->mlp_ready = true;
  return ARA_OK;
}

ara_status ara_mlp_eval(ara_ctx* ctx, const float* params, const float* z, int64_t n, float* y) {
  if (!ctx) return ARA_ERR_INVALID_ARG;
  if (n < 0 || (n > 0 && (!z || !y))) return fail(ctx, ARA_ERR_INVALID_ARG, "bad arguments");
  if (n == 0) return ARA_OK;
  CUDA_TRY(ctx, cudaSetDevice(ctx->device));
  MlpDevWeights* w = nullptr;
  float* tmpP = nullptr;
  ara_status s = mlp_image(ctx, params, &w, &tmpP);
  const int64_t np = (n + 15) / 16 * 16;
  float *dz = nullptr, *dy = nullptr;
  cudaError_t e = cudaSuccess;
  if (s == ARA_OK) {
    if ((e = dev_alloc(&dz, 3 * np)) == cudaSuccess && (e = dev_alloc(&dy, np)) == cudaSuccess &&
        (e = cudaMemsetAsync(dz, 0, sizeof(float) * 3 * np, ctx->stream)) == cudaSuccess &&
        (e = cudaMemcpyAsync(dz, z, sizeof(float) * 3 * n, cudaMemcpyDefault, ctx->stream)) == cudaSuccess &&
        (e = launch_mlp_eval(w, dz, np, dy, ctx->stream)) == cudaSuccess &&
        (e = cudaMemcpyAsync(y, dy, sizeof(float) * n, cudaMemcpyDefault, ctx->stream)) == cudaSuccess)
      e = cudaStreamSynchronize(ctx->stream);
    if (e != cudaSuccess) s = fail(ctx, ARA_ERR_CUDA, "mlp eval: %s", cudaGetErrorString(e));
  }
  cudaStreamSynchronize(ctx->stream);
  cudaGetLastError();
  dev_free(dz);
  dev_free(dy);
  dev_free(tmpP);
  if (w && w != ctx->mlp_W) dev_free(w);
  return s;
}

ara_status ara_mlp_grad(ara_ctx* ctx, const float* params, const float* z, const float* x,
                        const float* t, int64_t n, float* grad, double* loss) {
  if (!ctx) return ARA_ERR_INVALID_ARG;
  if (n < 16 || n % 16 != 0 || !z || !x || !t || !grad || !loss)
    return fail(ctx, ARA_ERR_INVALID_ARG, "n must be a positive multiple of 16");
  CUDA_TRY(ctx, cudaSetDevice(ctx->device));
  MlpDevWeights* w = nullptr;
  float* tmpP = nullptr;
  ara_status s = mlp_image(ctx, params, &w, &tmpP);
  float *dz = nullptr, *dx = nullptr, *dt = nullptr, *dg = nullptr, *dl = nullptr;
  MlpBuffers buf;
  cudaError_t e = cudaSuccess;
  float hl = 0.0f;
  if (s == ARA_OK) {
    if ((e = dev_alloc(&dz, 3 * n)) == cudaSuccess && (e = dev_alloc(&dx, n)) == cudaSuccess &&
        (e = dev_alloc(&dt, n)) == cudaSuccess && (e = dev_alloc(&dg, kMlpParams)) == cudaSuccess &&
        (e = dev_alloc(&dl, 1)) == cudaSuccess && (e = mlp_scratch(buf, n, ctx->stream)) == cudaSuccess &&
        (e = cudaMemcpyAsync(dz, z, sizeof(float) * 3 * n, cudaMemcpyDefault, ctx->stream)) == cudaSuccess &&
        (e = cudaMemcpyAsync(dx, x, sizeof(float) * n, cudaMemcpyDefault, ctx->stream)) == cudaSuccess &&
        (e = cudaMemcpyAsync(dt, t, sizeof(float) * n, cudaMemcpyDefault, ctx->stream)) == cudaSuccess &&
        (e = cudaMemsetAsync(dg, 0, sizeof(float) * kMlpParams, ctx->stream)) == cudaSuccess &&
        (e = cudaMemsetAsync(dl, 0, sizeof(float), ctx->stream)) == cudaSuccess &&
        (e = launch_mlp_step(w, dz, dx, dt, n, buf.s, dg, dl, ctx->stream)) == cudaSuccess &&
        (e = cudaMemcpyAsync(grad, dg, sizeof(float) * kMlpParams, cudaMemcpyDefault, ctx->stream)) == cudaSuccess &&
        (e = cudaMemcpyAsync(&hl, dl, sizeof(float), cudaMemcpyDeviceToHost, ctx->stream)) == cudaSuccess)
      e = cudaStreamSynchronize(ctx->stream);
    if (e != cudaSuccess) s = fail(ctx, ARA_ERR_CUDA, "mlp grad: %s", cudaGetErrorString(e));
  }
  cudaStreamSynchronize(ctx->stream);
  cudaGetLastError();
  for (float* q : {dz, dx, dt, dg, dl}) dev_free(q);
  buf.free_all();
  dev_free(tmpP);
  if (w && w != ctx->mlp_W) dev_free(w);
  *loss = hl;
  return s;
}

}  // extern "C"
