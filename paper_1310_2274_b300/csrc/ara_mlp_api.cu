// ara_mlp_api.cu -- the learned surrogate through the C ABI: training, certification, save and
// load, evaluation and gradients of the network.
#include <random>
#include <string.h>
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
  unsigned int n_bad = 0;
  e = cudaMemcpyAsync(b.data(), ctx->mlp_bound, sizeof(float) * kCertCells, cudaMemcpyDeviceToHost,
                      ctx->stream);
  if (e == cudaSuccess)
    e = cudaMemcpyAsync(&n_bad, bad, sizeof(unsigned int), cudaMemcpyDeviceToHost, ctx->stream);
  if (e == cudaSuccess) e = cudaStreamSynchronize(ctx->stream);
  cleanup();
  if (e != cudaSuccess) return fail(ctx, ARA_ERR_CUDA, "surrogate certification: %s", cudaGetErrorString(e));
  if (rep) {
    int64_t acc = 0;
    for (float v : b) acc += v <= eps;
    rep->cells_accepted = (double)acc / (double)kCertCells;
    rep->err_median = percentile(b, 0.5);
    rep->err_p99 = percentile(b, 0.99);
    rep->bad_targets += n_bad;
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
  rep.bad_targets += hbad;  // plus the certification points counted by mlp_certify
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
