// ara_risk.cu -- ordering of year losses and the risk measures of paper §2.4 through the C ABI
// (PML/TVaR, ranks, top-k for trial shards).
#include <cuda_runtime.h>
#include <math.h>
#include <string.h>

#include <algorithm>
#include <cmath>
#include <vector>

#include "../../include/ara.h"
#include "ara_ctx.h"
#include "ara_host.h"
#include "ara_internal.h"
#include "ara_philox.cuh"

using namespace ara;

extern "C" {

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

}  // extern "C"
