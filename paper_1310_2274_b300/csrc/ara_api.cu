// ara_api.cu -- the C ABI of libara (include/ara.h): contexts, options, and the staging of YETs,
// ELTs and layers.
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
#include <thread>
#include <vector>

#include "../../include/ara.h"
#include "ara_internal.h"
#include "ara_ctx.h"
#include "ara_philox.cuh"
#include "ara_host.h"

using namespace ara;

void free_layer_on(ara_ctx* c, LayerDev& l, bool ordered, cudaStream_t st) {
  mem_free(c, l.evt, ordered, st);
  mem_free(c, l.tables, ordered, st);
  mem_free(c, l.packed, ordered, st);
  mem_free(c, l.packed_rec, ordered, st);
  mem_free(c, l.corr, ordered, st);
  mem_free(c, l.starts, ordered, st);
  l = LayerDev();
}

void free_layer(ara_ctx* c, LayerDev& l) { free_layer_on(c, l, false, nullptr); }


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
  {  // the pool of object memory (obj_alloc), keeping up to kPoolKeepBytes of freed memory
    cudaMemPoolProps props = {};
    props.allocType = cudaMemAllocationTypePinned;
    props.location.type = cudaMemLocationTypeDevice;
    props.location.id = ctx->device;
    uint64_t keep = kPoolKeepBytes;
    if (cudaMemPoolCreate(&ctx->pool, &props) != cudaSuccess ||
        cudaMemPoolSetAttribute(ctx->pool, cudaMemPoolAttrReleaseThreshold, &keep) !=
            cudaSuccess) {
      cudaGetLastError();
      ara_destroy(ctx);
      return ARA_ERR_CUDA;
    }
  }
  *out = ctx;
  return ARA_OK;
}

void ara_destroy(ara_ctx* ctx) {
  if (!ctx) return;
  cudaSetDevice(ctx->device);
  cudaDeviceSynchronize();
  if (ctx->own_stream) ctx->stream = ctx->own_stream;  // a caller's stream may be gone by now
  if (ctx->pool) {
    for (auto& y : ctx->yets) free_yet(ctx, y);
    for (auto& e : ctx->elts) free_elt(ctx, e);
    for (auto& l : ctx->layers) free_layer(ctx, l);
    if (ctx->stream) cudaStreamSynchronize(ctx->stream);
    cudaMemPoolDestroy(ctx->pool);
    ctx->pool = nullptr;
  }
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
  if (ctx->copy_stream) cudaStreamSynchronize(ctx->copy_stream);
  for (int b = 0; b < kStreamBufs; ++b) {
    dev_free(ctx->d_sids[b]);
    if (ctx->ev_ready[b]) cudaEventDestroy(ctx->ev_ready[b]);
    if (ctx->ev_free[b]) cudaEventDestroy(ctx->ev_free[b]);
  }
  if (ctx->copy_stream) cudaStreamDestroy(ctx->copy_stream);
  dev_free(ctx->d_scratch);
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
      if (value != ARA_SCHED_BAND && value != ARA_SCHED_TRIAL && value != ARA_SCHED_AUTO)
        return fail(ctx, ARA_ERR_INVALID_ARG, "schedule must be ARA_SCHED_AUTO, _BAND or _TRIAL");
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
  // offsets: checked on the device where they and the timestamps are there (the host keeps no
  // copy then), else on the host
  const bool dev_path = is_device_ptr(trial_offsets) && (!timestamps || is_device_ptr(timestamps));
  std::vector<int64_t> off;
  int64_t max_len = 0, n_occ = 0;
  if (dev_path) {
    OffsetCheck oc;
    CUDA_TRY(ctx, launch_check_offsets(trial_offsets, n_trials,
                                       reinterpret_cast<OffsetCheck*>(ctx->d_misc), ctx->stream));
    CUDA_TRY(ctx, cudaMemcpyAsync(&oc, ctx->d_misc, sizeof oc, cudaMemcpyDeviceToHost,
                                  ctx->stream));
    CUDA_TRY(ctx, cudaStreamSynchronize(ctx->stream));
    if (oc.first != 0) return fail(ctx, ARA_ERR_INVALID_ARG, "trial_offsets[0] != 0");
    if (oc.first_decrease >= 0)
      return fail(ctx, ARA_ERR_INVALID_ARG, "trial_offsets decrease at trial %lld",
                  (long long)oc.first_decrease);
    max_len = oc.max_len;
    n_occ = oc.last;
  } else {
    off.resize((size_t)n_trials + 1);
    CUDA_TRY(ctx, cudaMemcpy(off.data(), trial_offsets, sizeof(int64_t) * off.size(),
                             cudaMemcpyDefault));
    if (off[0] != 0) return fail(ctx, ARA_ERR_INVALID_ARG, "trial_offsets[0] != 0");
    for (int64_t i = 0; i < n_trials; ++i) {
      const int64_t len = off[(size_t)i + 1] - off[(size_t)i];
      if (len < 0) return fail(ctx, ARA_ERR_INVALID_ARG, "trial_offsets decrease at trial %lld",
                               (long long)i);
      if (len > max_len) max_len = len;
    }
    n_occ = off[(size_t)n_trials];
  }
  if (n_occ > 0 && (!event_ids || !timestamps))
    return fail(ctx, ARA_ERR_INVALID_ARG, "event_ids or timestamps is NULL");
  if (n_occ >= ((int64_t)1 << 40)) return fail(ctx, ARA_ERR_INVALID_ARG, "YET too large");
  YetDev y;
  y.n_trials = n_trials;
  y.n_occ = n_occ;
  y.catalog = catalog_size;
  y.max_len = max_len;
  // the runs never read timestamps, so they are checked and not kept: host ones on host threads
  // while the ids cross to the device, device ones where they are, by the validation kernel
  const bool ts_on_host = n_occ > 0 && !is_device_ptr(timestamps);
  cudaError_t e;
  if ((e = obj_alloc(ctx, &y.ids, n_occ)) != cudaSuccess ||
      (e = obj_alloc(ctx, &y.offsets, n_trials + 1)) != cudaSuccess) {
    cudaGetLastError();
    free_yet(ctx, y);
    return fail(ctx, ARA_ERR_OOM, "YET of %lld occurrences: %s", (long long)n_occ,
                cudaGetErrorString(e));
  }
  unsigned int host_flags = 0;
  std::thread ts_check;
  if (ts_on_host)
    ts_check = std::thread(
        [&]() { host_flags = validate_timestamps_host(off.data(), timestamps, n_trials); });
  // device offsets are copied where they are; ids in device memory are copied by the validation
  // kernel as it checks them (one pass over them); host ones, even page-locked, by one bulk copy
  // first (the kernel's scattered reads would cross PCIe slower than the copy engine)
  const int64_t* off_src = dev_path ? trial_offsets : off.data();
  const int32_t* r_ids = n_occ > 0 && is_device_ptr(event_ids) ? event_ids : nullptr;
  if ((!r_ids && (e = copy_in(y.ids, event_ids, n_occ, ctx->stream)) != cudaSuccess) ||
      (e = copy_in(y.offsets, off_src, n_trials + 1, ctx->stream)) != cudaSuccess ||
      (e = cudaMemsetAsync(ctx->d_flags, 0, sizeof(unsigned int), ctx->stream)) != cudaSuccess ||
      (e = launch_validate_yet_range(r_ids ? r_ids : y.ids, ts_on_host ? nullptr : timestamps, 0,
                                     y.offsets, 0, n_trials, catalog_size, ctx->d_flags,
                                     ctx->stream, r_ids ? y.ids : nullptr)) != cudaSuccess) {
    cudaGetLastError();
    if (ts_check.joinable()) ts_check.join();
    cudaStreamSynchronize(ctx->stream);
    free_yet(ctx, y);
    return fail(ctx, ARA_ERR_CUDA, "staging YET: %s", cudaGetErrorString(e));
  }
  unsigned int flags = 0;
  e = cudaMemcpyAsync(&flags, ctx->d_flags, sizeof flags, cudaMemcpyDeviceToHost, ctx->stream);
  if (e == cudaSuccess) e = cudaStreamSynchronize(ctx->stream);
  if (ts_check.joinable()) ts_check.join();
  if (e != cudaSuccess) {
    cudaGetLastError();
    free_yet(ctx, y);
    return fail(ctx, ARA_ERR_CUDA, "staging YET: %s", cudaGetErrorString(e));
  }
  flags |= host_flags;
  if (flags) {
    free_yet(ctx, y);
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
  if ((e = obj_alloc(ctx, &y.offsets, n_trials + 1)) != cudaSuccess ||
      (e = copy_in(y.offsets, y.h_off.data(), n_trials + 1, ctx->stream)) != cudaSuccess ||
      (e = cudaStreamSynchronize(ctx->stream)) != cudaSuccess) {
    cudaGetLastError();
    free_yet(ctx, y);
    return fail(ctx, ARA_ERR_CUDA, "staging YET offsets: %s", cudaGetErrorString(e));
  }
  y.live = true;
  ctx->yets.push_back(std::move(y));
  *yet_out = (int32_t)ctx->yets.size() - 1;
  // the first run's leading chunks cross PCIe while the caller stages ELTs and layers
  prefetch_stream(ctx, *yet_out);
  return ARA_OK;
}

ara_status ara_free_yet(ara_ctx* ctx, int32_t yet) {
  if (!ctx) return ARA_ERR_INVALID_ARG;
  if (yet < 0 || yet >= (int32_t)ctx->yets.size() || !ctx->yets[yet].live)
    return fail(ctx, ARA_ERR_BAD_HANDLE, "bad YET handle %d", yet);
  for (auto& e : ctx->elts)
    if (e.live && e.yet == yet) return fail(ctx, ARA_ERR_INVALID_ARG, "YET still has ELTs");
  CUDA_TRY(ctx, cudaSetDevice(ctx->device));
  CUDA_TRY(ctx, cudaDeviceSynchronize());  // no stream may still read the YET
  if (ctx->yets[yet].host && ctx->copy_stream) {
    // copies of its ids (ahead of a run, or of a run that stopped on an error) end before the
    // caller may release the arrays
    if (ctx->pf_yet == yet) ctx->pf_yet = -1;
    CUDA_TRY(ctx, cudaStreamSynchronize(ctx->copy_stream));
  }
  free_yet(ctx, ctx->yets[yet]);
  return ARA_OK;
}

// ---- ELT ------------------------------------------------------------------------------------
ara_status ara_add_elts(ara_ctx* ctx, int32_t yet, int32_t n_elts, const int64_t* n,
                        const int32_t* const* event_ids, const double* const* mean,
                        const double* const* sd, const double* const* sd_corr,
                        const double* const* max_exposure, int32_t* elts_out) {
  if (!ctx) return ARA_ERR_INVALID_ARG;
  if (n_elts < 0) return fail(ctx, ARA_ERR_INVALID_ARG, "n_elts < 0");
  if (n_elts > 0 && (!elts_out || !n || !event_ids || !mean || !sd || !max_exposure))
    return fail(ctx, ARA_ERR_INVALID_ARG, "NULL argument");
  if (yet < 0 || yet >= (int32_t)ctx->yets.size() || !ctx->yets[yet].live)
    return fail(ctx, ARA_ERR_BAD_HANDLE, "bad YET handle %d", yet);
  for (int32_t j = 0; j < n_elts; ++j) {
    if (n[j] < 0 || n[j] >= ((int64_t)1 << 31))
      return fail(ctx, ARA_ERR_INVALID_ARG, "bad record count of ELT %d", j);
    if (n[j] > 0 && (!event_ids[j] || !mean[j] || !sd[j] || !max_exposure[j]))
      return fail(ctx, ARA_ERR_INVALID_ARG, "NULL array of ELT %d", j);
  }
  if (n_elts == 0) return ARA_OK;
  ara_status s = set_device(ctx);
  if (s != ARA_OK) return s;
  const YetDev& y = ctx->yets[yet];
  const bool defer = ctx->table_policy == ARA_TABLES_ON_DEMAND;
  auto sdc_of = [&](int32_t j) { return sd_corr ? sd_corr[j] : nullptr; };
  // staging scratch: each ELT's check flags and uncertified count, the duplicate marks, and the
  // input copies of the largest batch of kMaxPrepJobs ELTs (reused batch after batch: the stream
  // orders them); sized once, before any work is queued
  size_t temps = 0;
  for (int32_t b = 0; b < n_elts; b += kMaxPrepJobs) {
    size_t t = 0;
    for (int32_t j = b; j < std::min(n_elts, b + kMaxPrepJobs); ++j)
      t += scratch_bytes<double>(n[j]) * (sdc_of(j) ? 4 : 3);
    temps = std::max(temps, t);
  }
  const size_t scratch = scratch_bytes<unsigned int>(n_elts) +
                         scratch_bytes<unsigned long long>(n_elts) +
                         scratch_bytes<unsigned int>(y.catalog) + temps;
  std::vector<EltDev> es((size_t)n_elts);
  auto undo = [&]() {
    cudaGetLastError();
    cudaStreamSynchronize(ctx->stream);
    for (auto& e : es) free_elt(ctx, e);
  };
  cudaError_t err = cudaSuccess;
  for (int32_t j = 0; j < n_elts && err == cudaSuccess; ++j) {
    EltDev& e = es[(size_t)j];
    e.yet = yet;
    e.n = n[j];
    if ((err = obj_alloc(ctx, &e.ids, e.n)) == cudaSuccess &&
        (err = obj_alloc(ctx, &e.recs, e.n)) == cudaSuccess &&
        (defer || (err = obj_alloc(ctx, &e.tables, e.n * kTablePieces)) == cudaSuccess) && sdc_of(j))
      err = obj_alloc(ctx, &e.corr, e.n);
  }
  if (err == cudaSuccess) err = ensure_scratch(ctx, scratch);
  if (err != cudaSuccess) {
    undo();
    return fail(ctx, ARA_ERR_OOM, "%d ELTs: %s", n_elts, cudaGetErrorString(err));
  }
  ScratchCarver sc{ctx->d_scratch};
  unsigned int* d_flags = sc.take<unsigned int>(n_elts);
  unsigned long long* d_uncert = sc.take<unsigned long long>(n_elts);
  unsigned int* d_dup = sc.take<unsigned int>(y.catalog);
  std::vector<unsigned int> flags((size_t)n_elts, 0u);
  std::vector<unsigned long long> uncert((size_t)n_elts, 0ull);
  err = cudaMemsetAsync(d_flags, 0, sizeof(unsigned int) * (size_t)n_elts, ctx->stream);
  if (err == cudaSuccess)
    err = cudaMemsetAsync(d_uncert, 0, sizeof(unsigned long long) * (size_t)n_elts, ctx->stream);
  // the records of each batch of kMaxPrepJobs ELTs checked and converted in one launch
  for (int32_t b = 0; b < n_elts && err == cudaSuccess; b += kMaxPrepJobs) {
    PrepJobs jobs{};
    jobs.n = std::min(kMaxPrepJobs, n_elts - b);
    ScratchCarver tc = sc;
    for (int k = 0; k < jobs.n && err == cudaSuccess; ++k) {
      const int32_t j = b + k;
      EltDev& e = es[(size_t)j];
      const int64_t nj = e.n;
      double* d_mean = tc.take<double>(nj);
      double* d_sd = tc.take<double>(nj);
      double* d_mx = tc.take<double>(nj);
      double* d_sdc = sdc_of(j) ? tc.take<double>(nj) : nullptr;
      // inputs the device can read where they are (device memory, mapped page-locked host
      // memory) are read in place by the staging kernel, which also writes the ids' device copy;
      // the others are copied first.  (Reads over PCIe by the kernel do not queue behind other
      // copies, such as the ids a host-resident YET copies ahead.)
      const int32_t* r_ids = device_readable(event_ids[j]);
      const double* r_mean = device_readable(mean[j]);
      const double* r_sd = device_readable(sd[j]);
      const double* r_sdc = sdc_of(j) ? device_readable(sdc_of(j)) : nullptr;
      const double* r_mx = device_readable(max_exposure[j]);
      if ((!r_ids && (err = copy_in(e.ids, event_ids[j], nj, ctx->stream)) != cudaSuccess) ||
          (!r_mean && (err = copy_in(d_mean, mean[j], nj, ctx->stream)) != cudaSuccess) ||
          (!r_sd && (err = copy_in(d_sd, sd[j], nj, ctx->stream)) != cudaSuccess) ||
          (sdc_of(j) && !r_sdc &&
           (err = copy_in(d_sdc, sdc_of(j), nj, ctx->stream)) != cudaSuccess) ||
          (!r_mx && (err = copy_in(d_mx, max_exposure[j], nj, ctx->stream)) != cudaSuccess))
        break;
      jobs.ids[k] = r_ids ? r_ids : e.ids;
      jobs.ids_out[k] = r_ids ? e.ids : nullptr;
      jobs.mean[k] = r_mean ? r_mean : d_mean;
      jobs.sd[k] = r_sd ? r_sd : d_sd;
      jobs.sdc[k] = sdc_of(j) ? (r_sdc ? r_sdc : d_sdc) : nullptr;
      jobs.mx[k] = r_mx ? r_mx : d_mx;
      jobs.recs[k] = e.recs;
      jobs.corr[k] = e.corr;
      jobs.first[k + 1] = jobs.first[k] + nj;
    }
    if (err == cudaSuccess)
      err = cudaMemsetAsync(d_dup, 0, sizeof(unsigned int) * (size_t)y.catalog, ctx->stream);
    if (err == cudaSuccess)
      err = launch_prepare_elts(jobs, y.catalog, d_dup, d_flags + b, ctx->stream);
  }
  // tables at staging (ARA_TABLES_EAGER): all the ELTs' in one launch (kMaxTableJobs a launch)
  for (int32_t b = 0; !defer && b < n_elts && err == cudaSuccess; b += kMaxTableJobs) {
    TableJobs jobs{};
    jobs.n = std::min(kMaxTableJobs, n_elts - b);
    for (int k = 0; k < jobs.n; ++k) {
      const EltDev& e = es[(size_t)(b + k)];
      jobs.recs[k] = e.recs;
      jobs.tables[k] = e.tables;
      jobs.first[k + 1] = jobs.first[k] + e.n;
    }
    err = launch_build_tables(jobs, d_uncert + b, ctx->stream);
  }
  if (err == cudaSuccess)
    err = cudaMemcpyAsync(flags.data(), d_flags, sizeof(unsigned int) * (size_t)n_elts,
                          cudaMemcpyDeviceToHost, ctx->stream);
  if (err == cudaSuccess)
    err = cudaMemcpyAsync(uncert.data(), d_uncert, sizeof(unsigned long long) * (size_t)n_elts,
                          cudaMemcpyDeviceToHost, ctx->stream);
  if (err == cudaSuccess) err = cudaStreamSynchronize(ctx->stream);
  if (err != cudaSuccess) {
    const ara_status st = err == cudaErrorMemoryAllocation ? ARA_ERR_OOM : ARA_ERR_CUDA;
    undo();
    return fail(ctx, st, "staging ELTs: %s", cudaGetErrorString(err));
  }
  for (int32_t j = 0; j < n_elts; ++j)
    if (flags[(size_t)j]) {
      const unsigned int f = flags[(size_t)j];
      undo();
      return fail(ctx, ARA_ERR_INVALID_ARG, "ELT %d rejected:%s%s%s%s", j,
                  (f & 8) ? " event id outside the catalogue" : "",
                  (f & 16) ? " mean <= 0, an sd < 0 or non-finite value" : "",
                  (f & 32) ? " max_exposure <= mean with sd > 0" : "",
                  (f & 64) ? " duplicate event id" : "");
    }
  for (int32_t j = 0; j < n_elts; ++j) {
    EltDev& e = es[(size_t)j];
    e.n_uncertified = (int64_t)uncert[(size_t)j];
    e.live = true;
    ctx->elts.push_back(e);
    elts_out[j] = (int32_t)ctx->elts.size() - 1;
  }
  return ARA_OK;
}

ara_status ara_add_elt_corr(ara_ctx* ctx, int32_t yet, int64_t n, const int32_t* event_ids,
                            const double* mean, const double* sd_indep, const double* sd_corr,
                            const double* max_exposure, int32_t* elt_out) {
  if (!ctx) return ARA_ERR_INVALID_ARG;
  if (!elt_out) return fail(ctx, ARA_ERR_INVALID_ARG, "elt_out is NULL");
  return ara_add_elts(ctx, yet, 1, &n, &event_ids, &mean, &sd_indep, &sd_corr, &max_exposure,
                      elt_out);
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
  CUDA_TRY(ctx, cudaDeviceSynchronize());  // no stream may still read the ELT
  free_elt(ctx, ctx->elts[elt]);
  return ARA_OK;
}

// ---- layer ------------------------------------------------------------------------------------
}  // extern "C"

// Builds a layer; wide = true forces 16-byte index entries (two mask words) whatever the ELT
// count, the form the batched serving kernel takes.
ara_status ara_build_layer(ara_ctx* ctx, const int32_t* elts, int32_t n_elts, double occ_ret,
                           double occ_lim, double agg_ret, double agg_lim, bool wide,
                           cudaStream_t st, bool may_build_band, bool ordered,
                           LayerDev* out, bool starts) {
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
  const TablePiece** d_src = nullptr;
  const float** d_ssrc = nullptr;  // start-table sources (layers packed with start tables)
  // temporaries: stream-ordered ones on a serving stream, else staging scratch (the table source
  // pointers sized for every record of the layer's ELTs, which bounds the packed count)
  auto cleanup = [&]() {
    if (!ordered) {
      cudaStreamSynchronize(st);
      return;
    }
    mem_free(ctx, d_mask, ordered, st);
    mem_free(ctx, d_cnt, ordered, st);
    mem_free(ctx, d_base, ordered, st);
    mem_free(ctx, d_tmp, ordered, st);
    mem_free(ctx, d_src, ordered, st);
    mem_free(ctx, d_ssrc, ordered, st);
  };
  const int64_t evt_words = C * (MW == 1 ? 2 : 4);
  if (ordered) {
    err = mem_alloc(ctx, &d_mask, C * MW, ordered, st);
    if (err == cudaSuccess) err = mem_alloc(ctx, &d_cnt, C, ordered, st);
    if (err == cudaSuccess) err = mem_alloc(ctx, &d_base, C, ordered, st);
    if (err == cudaSuccess) err = mem_alloc(ctx, &d_tmp, tmp_words, ordered, st);
  } else {
    int64_t records = 0;
    for (int j = 0; j < n_elts; ++j) records += ctx->elts[elts[j]].n;
    err = ensure_scratch(ctx, scratch_bytes<uint32_t>(C * MW) + 2 * scratch_bytes<uint32_t>(C) +
                                  scratch_bytes<uint32_t>(tmp_words) +
                                  scratch_bytes<const TablePiece*>(records) +
                                  (starts ? scratch_bytes<const float*>(records) : 0));
    if (err == cudaSuccess) {
      ScratchCarver sc{ctx->d_scratch};
      d_mask = sc.take<uint32_t>(C * MW);
      d_cnt = sc.take<uint32_t>(C);
      d_base = sc.take<uint32_t>(C);
      d_tmp = sc.take<uint32_t>(tmp_words);
      d_src = sc.take<const TablePiece*>(records);
      if (starts) d_ssrc = sc.take<const float*>(records);
    }
  }
  if (err != cudaSuccess || (err = mem_alloc(ctx, &L.evt, evt_words, ordered, st)) != cudaSuccess) {
    cudaGetLastError();
    cleanup();
    free_layer_on(ctx, L, ordered, st);
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
    free_layer_on(ctx, L, ordered, st);
    return fail(ctx, ARA_ERR_CUDA, "layer index: %s", cudaGetErrorString(err));
  }
  L.n_packed = (int64_t)last[0] + (int64_t)last[1];
  // packed records, then the records' tables copied into packed order (one gather per hit);
  // correlated weights only when some ELT of the layer has a correlated SD
  bool has_corr = false, all_tables = true, all_starts = starts;
  for (int j = 0; j < n_elts; ++j) {
    has_corr = has_corr || ctx->elts[elts[j]].corr != nullptr;
    all_tables = all_tables && ctx->elts[elts[j]].tables != nullptr;
    all_starts = all_starts && ctx->elts[elts[j]].starts != nullptr;
  }
  if ((err = mem_alloc(ctx, &L.packed, L.n_packed, ordered, st)) != cudaSuccess ||
      (err = mem_alloc(ctx, &L.packed_rec, L.n_packed, ordered, st)) != cudaSuccess ||
      (all_tables && (err = mem_alloc(ctx, &L.tables, L.n_packed * kTablePieces, ordered, st)) !=
                         cudaSuccess) ||
      (ordered && (err = mem_alloc(ctx, &d_src, L.n_packed, ordered, st)) != cudaSuccess) ||
      (has_corr && (err = mem_alloc(ctx, &L.corr, L.n_packed, ordered, st)) != cudaSuccess) ||
      (all_starts &&
       (err = mem_alloc(ctx, &L.starts, L.n_packed * kStartFloats, ordered, st)) != cudaSuccess) ||
      (all_starts && ordered && (err = mem_alloc(ctx, &d_ssrc, L.n_packed, ordered, st)) !=
                                    cudaSuccess)) {
    cudaGetLastError();
    cleanup();
    free_layer_on(ctx, L, ordered, st);
    return fail(ctx, ARA_ERR_OOM, "layer records and tables: %s", cudaGetErrorString(err));
  }
  for (int j = 0; j < n_elts && err == cudaSuccess; ++j)
    err = launch_layer_scatter(ctx->elts[elts[j]], j, MW, L.evt, L.packed, d_src, L.packed_rec,
                               L.corr, all_starts ? d_ssrc : nullptr, st);
  if (err == cudaSuccess && all_tables) err = launch_gather_tables(L.n_packed, d_src, L.tables, st);
  if (err == cudaSuccess && all_starts)
    err = launch_gather_starts(L.n_packed, d_ssrc, L.starts, st);
  // the largest event-loss bound sizes the grid of the exact year sums (d_cnt is free by now)
  unsigned int ev_bits = 0u;
  if (err == cudaSuccess) err = launch_layer_event_bound(L.evt, MW, C, L.packed, d_cnt, st);
  if (err == cudaSuccess)
    err = cudaMemcpyAsync(&ev_bits, d_cnt, sizeof(unsigned int), cudaMemcpyDeviceToHost, st);
  if (err == cudaSuccess) err = cudaStreamSynchronize(st);
  cleanup();
  if (err != cudaSuccess) {
    cudaGetLastError();
    free_layer_on(ctx, L, ordered, st);
    return fail(ctx, ARA_ERR_CUDA, "layer records: %s", cudaGetErrorString(err));
  }
  memcpy(&L.ev_bound, &ev_bits, sizeof(float));
  // band-major copy of the YET at this layer's band width (one per width and YET): used if it
  // exists, else made by a run of the table inversion once the schedule asks for it (at once
  // under ARA_SCHED_BAND, once it pays under ARA_SCHED_AUTO; a Newton pass never makes one)
  const int log2w = ctx->band_log2w > 0 ? ctx->band_log2w : choose_band_log2w(C, L.n_packed);
  bool banded = false;
  for (const auto& v : ctx->yets[yet].bands) banded = banded || v.log2w == log2w;
  if (banded)
    L.band_log2w = log2w;
  else if (may_build_band)
    L.band_want = log2w;
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
  CUDA_TRY(ctx, cudaDeviceSynchronize());  // no stream may still read the layer
  free_layer(ctx, ctx->layers[layer]);
  return ARA_OK;
}

}  // extern "C"
