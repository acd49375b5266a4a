// ara_mlp.cu -- training, evaluation and certification of the learned surrogate (ara_mlp.cuh).
//
// Training data: (alpha, beta, u) drawn from a counter-based stream (half log-uniform over the
// box [0.1, 50]^2, half the ELT value law's moment-matched parameters), the target x from the
// exact inversion polished in binary64.  Loss per sample: 100 (sigmoid(20 y) - x)^2 +
// 1e-3 (y - clip(logit x, +-30)/20)^2 (absolute error in x, which is what a loss sees, plus a weak
// pull on logit x that keeps the tails from saturating).
//
// One optimisation step = fwd_bwd (per 16-row tile per warp: forward with MMA, loss gradient,
// backward through the layers with MMA on transposed weights; activations and layer gradients are
// written transposed for the next kernel; bias gradients reduced in the warp) -> wgrad (split-K
// MMA over the batch for dW = dZ^T H, one m-tile per warp) -> adam (master FP32 weights) -> pack
// (BF16 shared-memory image for the next step).
#include <cuda_bf16.h>
#include <cuda_runtime.h>
#include <math.h>
#include <stdint.h>

#include "ara_internal.h"
#include "ara_mlp.cuh"
#include "ara_philox.cuh"
#include "ara_table.cuh"

namespace ara {

namespace {

constexpr float kLossX = 100.0f;
constexpr float kLossLogit = 1e-3f;
constexpr double kLn01 = -2.302585092994046;   // ln 0.1
constexpr double kLn50 = 3.912023005428146;    // ln 50

__device__ __forceinline__ void copy_smem(void* dst, const void* src, int bytes) {
  const uint4* s = reinterpret_cast<const uint4*>(src);
  uint4* d = reinterpret_cast<uint4*>(dst);
  for (int i = threadIdx.x; i < bytes / 16; i += blockDim.x) d[i] = s[i];
}

__device__ __forceinline__ float logit_clip(double lnx, double ln1mx) {
  double v = lnx - ln1mx;
  v = fmin(fmax(v, -30.0), 30.0);
  return (float)v;
}

// ---- training data ----------------------------------------------------------------------------
__global__ void gen_kernel(int64_t n, uint64_t seed, int64_t first, float* Z, float* X, float* T,
                           unsigned int* bad) {
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  const int64_t id = first + i;
  U4 c;
  c.x = (uint32_t)id; c.y = (uint32_t)((uint64_t)id >> 32); c.z = 0x5EEDu; c.w = 0x7A1Au;
  const U4 w = philox4x32_10(c, (uint32_t)seed, (uint32_t)(seed >> 32));
  const double u1 = word_to_uniform(w.x), u2 = word_to_uniform(w.y), u3 = word_to_uniform(w.z);
  const float u = word_to_uniform(w.w);
  double a = exp(kLn01 + u1 * (kLn50 - kLn01)), b = exp(kLn01 + u3 * (kLn50 - kLn01));
  if (id & 1) {  // the ELT value law: sd = mean U(0.3,1.2), max = mean U(3,10)
    const double s = 0.3 + 0.9 * u1, m = 3.0 + 7.0 * u2;
    const double k = (m - 1.0) / (s * s) - 1.0;
    const double a2 = k / m, b2 = (1.0 - 1.0 / m) * k;
    if (a2 >= 0.1 && a2 <= 50.0 && b2 >= 0.1 && b2 <= 50.0) { a = a2; b = b2; }
  }
  double lnx, ln1mx;
  if (!ara_exact_quantile_logs(a, b, u, &lnx, &ln1mx)) atomicAdd(bad, 1u);
  Z[3 * i + 0] = (float)((log(a) - kLnCenter) / kLnHalf);
  Z[3 * i + 1] = (float)((log(b) - kLnCenter) / kLnHalf);
  Z[3 * i + 2] = (logf(u) - log1pf(-u)) / kLogitScale;
  X[i] = (float)exp(lnx);
  T[i] = logit_clip(lnx, ln1mx) / kOutScale;
}

// ---- forward + backward per tile ----------------------------------------------------------------
__device__ __forceinline__ void store_t2(__nv_bfloat16* HT, int64_t B, int col, int64_t row,
                                         uint32_t packed) {
  const __nv_bfloat162 v = *reinterpret_cast<const __nv_bfloat162*>(&packed);
  HT[(int64_t)col * B + row] = v.x;
  HT[(int64_t)(col + 1) * B + row] = v.y;
}

// Writes an A-fragment set (4 k-tiles) transposed: HT[feature][row].
__device__ __forceinline__ void store_frag_t(__nv_bfloat16* HT, int64_t B, int64_t r0, int g, int t,
                                             const uint32_t (&h)[4][4]) {
#pragma unroll
  for (int kk = 0; kk < 4; ++kk) {
    store_t2(HT, B, kk * 16 + 2 * t, r0 + g, h[kk][0]);
    store_t2(HT, B, kk * 16 + 2 * t, r0 + g + 8, h[kk][1]);
    store_t2(HT, B, kk * 16 + 8 + 2 * t, r0 + g, h[kk][2]);
    store_t2(HT, B, kk * 16 + 8 + 2 * t, r0 + g + 8, h[kk][3]);
  }
}

// dz (C layout, FP32) -> bias-gradient partials, transposed BF16 store, and A fragments.
__device__ __forceinline__ void dz_out(const float (&dz)[8][4], __nv_bfloat16* DZT, int64_t B,
                                       int64_t r0, int g, int t, float (&db)[8][2],
                                       uint32_t (&a)[4][4]) {
#pragma unroll
  for (int nn = 0; nn < 8; ++nn) {
    db[nn][0] += dz[nn][0] + dz[nn][2];
    db[nn][1] += dz[nn][1] + dz[nn][3];
  }
#pragma unroll
  for (int kk = 0; kk < 4; ++kk) {
    a[kk][0] = pack_bf16(dz[2 * kk][0], dz[2 * kk][1]);
    a[kk][1] = pack_bf16(dz[2 * kk][2], dz[2 * kk][3]);
    a[kk][2] = pack_bf16(dz[2 * kk + 1][0], dz[2 * kk + 1][1]);
    a[kk][3] = pack_bf16(dz[2 * kk + 1][2], dz[2 * kk + 1][3]);
  }
  store_frag_t(DZT, B, r0, g, t, a);
}

__global__ void __launch_bounds__(128) fwd_bwd_kernel(
    const MlpDevWeights* __restrict__ Wd, const float* __restrict__ Z, const float* __restrict__ X,
    const float* __restrict__ T, int64_t B, float inv_B, __nv_bfloat16* HT0, __nv_bfloat16* HT1,
    __nv_bfloat16* HT2, __nv_bfloat16* HT3, __nv_bfloat16* DZT1, __nv_bfloat16* DZT2,
    __nv_bfloat16* DZT3, float* grad, float* loss_acc) {
  __shared__ __align__(16) MlpSmem W;
  __shared__ __align__(16) MlpSmemBwd Wb;
  copy_smem(&W, &Wd->fwd, sizeof(MlpSmem));
  copy_smem(&Wb, &Wd->bwd, sizeof(MlpSmemBwd));
  __syncthreads();
  const int lane = threadIdx.x & 31, g = lane >> 2, t = lane & 3;
  const int64_t warp = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  const int64_t nwarps = ((int64_t)gridDim.x * blockDim.x) >> 5;
  float db1[8][2] = {}, db2[8][2] = {}, db3[8][2] = {}, dw4[8][2] = {};
  float db4 = 0.f, loss = 0.f;
  for (int64_t tile = warp; tile < B / 16; tile += nwarps) {
    const int64_t r0 = tile * 16;
    float zr0[3], zr8[3];
#pragma unroll
    for (int c = 0; c < 3; ++c) {
      zr0[c] = Z[(r0 + g) * 3 + c];
      zr8[c] = Z[(r0 + g + 8) * 3 + c];
    }
    float pre1[8][4], pre2[8][4], pre3[8][4];
    uint32_t h1[4][4], h2[4][4];
    float y0, y8;
    mlp_tile_forward_train(W, zr0, zr8, g, t, &y0, &y8, pre1, pre2, pre3, h1, h2, nullptr);
    // dL/dy for rows g and g + 8
    float dy[2];
#pragma unroll
    for (int h = 0; h < 2; ++h) {
      const int64_t r = r0 + g + 8 * h;
      const float y = h ? y8 : y0;
      const float s = 1.0f / (1.0f + __expf(-kOutScale * y));
      const float dx = s - X[r];
      const float dt = y - T[r];
      dy[h] = (2.0f * kLossX * dx * s * (1.0f - s) * kOutScale + 2.0f * kLossLogit * dt) * inv_B;
      if (t == 0) loss += (kLossX * dx * dx + kLossLogit * dt * dt) * inv_B;
    }
    // transposed activations: layer inputs for the weight gradients
    if (t == 0) {
#pragma unroll
      for (int c = 0; c < 3; ++c) {
        HT0[(int64_t)c * B + r0 + g] = __float2bfloat16_rn(zr0[c]);
        HT0[(int64_t)c * B + r0 + g + 8] = __float2bfloat16_rn(zr8[c]);
      }
    }
    store_frag_t(HT1, B, r0, g, t, h1);
    store_frag_t(HT2, B, r0, g, t, h2);
    // output layer (FP32): dW4 += dy silu(a3), db4 += dy; dH3 = dy W4, dZ3 = dH3 silu'(a3)
    float dz[8][4];
#pragma unroll
    for (int nn = 0; nn < 8; ++nn) {
      dw4[nn][0] += dy[0] * silu_f(pre3[nn][0]) + dy[1] * silu_f(pre3[nn][2]);
      dw4[nn][1] += dy[0] * silu_f(pre3[nn][1]) + dy[1] * silu_f(pre3[nn][3]);
    }
    if (t == 0) db4 += dy[0] + dy[1];
#pragma unroll
    for (int nn = 0; nn < 8; ++nn) {
      const int c = nn * 8 + 2 * t;
      dz[nn][0] = dy[0] * W.w4[c] * silu_grad_f(pre3[nn][0]);
      dz[nn][1] = dy[0] * W.w4[c + 1] * silu_grad_f(pre3[nn][1]);
      dz[nn][2] = dy[1] * W.w4[c] * silu_grad_f(pre3[nn][2]);
      dz[nn][3] = dy[1] * W.w4[c + 1] * silu_grad_f(pre3[nn][3]);
    }
    uint32_t a[4][4];
    dz_out(dz, DZT3, B, r0, g, t, db3, a);
    float acc[8][4];
    layer64(acc, a, Wb.w3t, g, t);  // dH2 = dZ3 W3
#pragma unroll
    for (int nn = 0; nn < 8; ++nn)
#pragma unroll
      for (int q = 0; q < 4; ++q) dz[nn][q] = acc[nn][q] * silu_grad_f(pre2[nn][q]);
    dz_out(dz, DZT2, B, r0, g, t, db2, a);
    layer64(acc, a, Wb.w2t, g, t);  // dH1 = dZ2 W2
#pragma unroll
    for (int nn = 0; nn < 8; ++nn)
#pragma unroll
      for (int q = 0; q < 4; ++q) dz[nn][q] = acc[nn][q] * silu_grad_f(pre1[nn][q]);
    dz_out(dz, DZT1, B, r0, g, t, db1, a);
  }
  // reduce the per-lane partials over the 8 row groups (lanes with equal t), then one atomic each
#pragma unroll
  for (int nn = 0; nn < 8; ++nn)
#pragma unroll
    for (int e = 0; e < 2; ++e) {
#pragma unroll
      for (int d = 4; d < 32; d <<= 1) {
        db1[nn][e] += __shfl_xor_sync(0xFFFFFFFFu, db1[nn][e], d);
        db2[nn][e] += __shfl_xor_sync(0xFFFFFFFFu, db2[nn][e], d);
        db3[nn][e] += __shfl_xor_sync(0xFFFFFFFFu, db3[nn][e], d);
        dw4[nn][e] += __shfl_xor_sync(0xFFFFFFFFu, dw4[nn][e], d);
      }
    }
  if (g == 0) {
#pragma unroll
    for (int nn = 0; nn < 8; ++nn)
#pragma unroll
      for (int e = 0; e < 2; ++e) {
        const int c = nn * 8 + 2 * t + e;
        atomicAdd(grad + kOffB1 + c, db1[nn][e]);
        atomicAdd(grad + kOffB2 + c, db2[nn][e]);
        atomicAdd(grad + kOffB3 + c, db3[nn][e]);
        atomicAdd(grad + kOffW4 + c, dw4[nn][e]);
      }
  }
#pragma unroll
  for (int d = 1; d < 32; d <<= 1) {
    db4 += __shfl_xor_sync(0xFFFFFFFFu, db4, d);
    loss += __shfl_xor_sync(0xFFFFFFFFu, loss, d);
  }
  if (lane == 0) {
    atomicAdd(grad + kOffB4, db4);
    atomicAdd(loss_acc, loss);
  }
}

// dW[o][i] += sum over rows r of DZT[o][r] * HT[i][r] for r in this block's chunk.
// One warp per 16 output rows (4 warps = 64 outputs); n_tiles = 8 (64 inputs) or 1 (3 inputs).
template <int NT>
__global__ void __launch_bounds__(128) wgrad_kernel(const __nv_bfloat16* __restrict__ DZT,
                                                    const __nv_bfloat16* __restrict__ HT,
                                                    int n_in, int64_t B, int64_t chunk,
                                                    float* dW) {
  constexpr int n_tiles = NT;
  const int lane = threadIdx.x & 31, g = lane >> 2, t = lane & 3, w = threadIdx.x >> 5;
  const int64_t k_begin = (int64_t)blockIdx.x * chunk;
  const int64_t k_end = min(B, k_begin + chunk);
  float acc[NT][4] = {};
  const __nv_bfloat16* arow0 = DZT + (int64_t)(16 * w + g) * B;
  const __nv_bfloat16* arow8 = DZT + (int64_t)(16 * w + g + 8) * B;
  for (int64_t k0 = k_begin; k0 < k_end; k0 += 16) {
    uint32_t a[4];
    a[0] = *reinterpret_cast<const uint32_t*>(arow0 + k0 + 2 * t);
    a[1] = *reinterpret_cast<const uint32_t*>(arow8 + k0 + 2 * t);
    a[2] = *reinterpret_cast<const uint32_t*>(arow0 + k0 + 8 + 2 * t);
    a[3] = *reinterpret_cast<const uint32_t*>(arow8 + k0 + 8 + 2 * t);
#pragma unroll
    for (int nn = 0; nn < n_tiles; ++nn) {
      const __nv_bfloat16* brow = HT + (int64_t)(nn * 8 + g) * B + k0;
      const uint32_t b0 = *reinterpret_cast<const uint32_t*>(brow + 2 * t);
      const uint32_t b1 = *reinterpret_cast<const uint32_t*>(brow + 8 + 2 * t);
      mma_bf16(acc[nn], a, b0, b1);
    }
  }
#pragma unroll
  for (int nn = 0; nn < n_tiles; ++nn) {
    const int c = nn * 8 + 2 * t;
    const int o0 = 16 * w + g, o8 = o0 + 8;
    if (c < n_in) {
      atomicAdd(dW + o0 * n_in + c, acc[nn][0]);
      atomicAdd(dW + o8 * n_in + c, acc[nn][2]);
    }
    if (c + 1 < n_in) {
      atomicAdd(dW + o0 * n_in + c + 1, acc[nn][1]);
      atomicAdd(dW + o8 * n_in + c + 1, acc[nn][3]);
    }
  }
}

__global__ void adam_kernel(float* P, float* M, float* V, float* G, int n, float lr, float b1,
                            float b2, float eps, float bc1, float bc2) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  const float g = G[i];
  const float m = b1 * M[i] + (1.0f - b1) * g;
  const float v = b2 * V[i] + (1.0f - b2) * g * g;
  M[i] = m;
  V[i] = v;
  P[i] -= lr * (m / bc1) / (sqrtf(v / bc2) + eps);
  G[i] = 0.0f;
}

// FP32 parameter vector -> BF16 shared-memory images (forward and backward).
__global__ void pack_kernel(const float* __restrict__ P, MlpDevWeights* Wd) {
  MlpSmem& F = Wd->fwd;
  MlpSmemBwd& Bw = Wd->bwd;
  const __nv_bfloat16 zero = __float2bfloat16_rn(0.0f);
  for (int i = threadIdx.x + blockIdx.x * blockDim.x; i < kH * kLd;
       i += blockDim.x * gridDim.x) {
    const int r = i / kLd, c = i % kLd;
    // W1 in columns 0..2 and, for the lo parts of the inference inputs, again in 3..5
    if (c < 24) F.w1[r][c] = c < 6 ? __float2bfloat16_rn(P[kOffW1 + r * 3 + c % 3]) : zero;
    F.w2[r][c] = c < kH ? __float2bfloat16_rn(P[kOffW2 + r * kH + c]) : zero;
    F.w3[r][c] = c < kH ? __float2bfloat16_rn(P[kOffW3 + r * kH + c]) : zero;
    Bw.w2t[r][c] = c < kH ? __float2bfloat16_rn(P[kOffW2 + c * kH + r]) : zero;
    Bw.w3t[r][c] = c < kH ? __float2bfloat16_rn(P[kOffW3 + c * kH + r]) : zero;
    if (c == 0) {
      F.b1[r] = P[kOffB1 + r];
      F.b2[r] = P[kOffB2 + r];
      F.b3[r] = P[kOffB3 + r];
      F.w4[r] = P[kOffW4 + r];
    }
    if (i == 0) {
      F.b4 = P[kOffB4];
      F.pad[0] = F.pad[1] = F.pad[2] = 0.0f;
    }
  }
}

// y = net(z) for n rows (n a multiple of 16; the caller pads).
__global__ void __launch_bounds__(128) eval_kernel(const MlpDevWeights* __restrict__ Wd,
                                                   const float* __restrict__ Z, int64_t n, float* Y) {
  __shared__ __align__(16) MlpSmem W;
  copy_smem(&W, &Wd->fwd, sizeof(MlpSmem));
  __syncthreads();
  const int lane = threadIdx.x & 31, g = lane >> 2, t = lane & 3;
  const int64_t warp = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  const int64_t nwarps = ((int64_t)gridDim.x * blockDim.x) >> 5;
  for (int64_t tile = warp; tile < n / 16; tile += nwarps) {
    const int64_t r0 = tile * 16;
    float zr0[3], zr8[3];
#pragma unroll
    for (int c = 0; c < 3; ++c) {
      zr0[c] = Z[(r0 + g) * 3 + c];
      zr8[c] = Z[(r0 + g + 8) * 3 + c];
    }
    float y0, y8;
    mlp_tile_forward(W, zr0, zr8, g, t, &y0, &y8);
    if (t == 0) {
      Y[r0 + g] = y0;
      Y[r0 + g + 8] = y8;
    }
  }
}

// ---- certification --------------------------------------------------------------------------------
// Cell (i0, i1, i2) of the kCert0 x kCert1 x kCert2 grid over the normalised inputs in [-1, 1]^3;
// kCertSamples stratified points per cell (the cell's corners first, then counter-based points).
__global__ void cert_points_kernel(int64_t n_cells, int samples, uint64_t seed, float* Z, float* X,
                                   unsigned int* bad) {
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n_cells * samples) return;
  const int64_t cell = i / samples;
  const int s = (int)(i % samples);
  const int i2 = (int)(cell % kCert2), i1 = (int)((cell / kCert2) % kCert1),
            i0 = (int)(cell / ((int64_t)kCert2 * kCert1));
  double f0, f1, f2;
  if (s < 8) {  // corners (shrunk by 1e-6 into the cell)
    f0 = (s & 1) ? 1.0 - 1e-6 : 1e-6;
    f1 = (s & 2) ? 1.0 - 1e-6 : 1e-6;
    f2 = (s & 4) ? 1.0 - 1e-6 : 1e-6;
  } else {
    U4 c;
    c.x = (uint32_t)i; c.y = (uint32_t)((uint64_t)i >> 32); c.z = 0xCE27u; c.w = 0x1u;
    const U4 w = philox4x32_10(c, (uint32_t)seed, (uint32_t)(seed >> 32));
    f0 = word_to_uniform(w.x); f1 = word_to_uniform(w.y); f2 = word_to_uniform(w.z);
  }
  const double z0 = -1.0 + 2.0 * (i0 + f0) / kCert0;
  const double z1 = -1.0 + 2.0 * (i1 + f1) / kCert1;
  const double z2 = -1.0 + 2.0 * (i2 + f2) / kCert2;
  const double a = exp(kLnCenter + kLnHalf * z0), b = exp(kLnCenter + kLnHalf * z1);
  // u on the binary32 uniform grid nearest to logit^-1(z2 * scale)
  double u = 1.0 / (1.0 + exp(-z2 * kLogitScale));
  u = fmin(fmax(u, 0x1p-24), 1.0 - 0x1p-24);
  const float uf = (float)(ldexp(2.0 * floor(ldexp(u, 23)) + 1.0, -24));
  double lnx, ln1mx;
  const bool ok = ara_exact_quantile_logs(a, b, uf, &lnx, &ln1mx);
  if (!ok) atomicAdd(bad, 1u);
  Z[3 * i + 0] = (float)((log(a) - kLnCenter) / kLnHalf);
  Z[3 * i + 1] = (float)((log(b) - kLnCenter) / kLnHalf);
  Z[3 * i + 2] = (logf(uf) - log1pf(-uf)) / kLogitScale;
  // no reference where the exact inversion failed: NaN makes the cell's bound 1 (rejected)
  X[i] = ok ? (float)exp(lnx) : __int_as_float(0x7FC00000);
}

__global__ void cert_reduce_kernel(int64_t n_cells, int samples, const float* X, const float* Y,
                                   float* bound) {
  const int64_t cell = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (cell >= n_cells) return;
  float m = 0.0f;
  for (int s = 0; s < samples; ++s) {
    const int64_t i = cell * samples + s;
    const float xs = 1.0f / (1.0f + __expf(-kOutScale * Y[i]));
    const float e = fabsf(xs - X[i]);
    m = (e == e) ? fmaxf(m, e) : 1.0f;
  }
  bound[cell] = m;
}

}  // namespace

cudaError_t launch_mlp_gen(int64_t n, uint64_t seed, int64_t first, float* Z, float* X, float* T,
                           unsigned int* bad, cudaStream_t st) {
  if (n == 0) return cudaSuccess;
  gen_kernel<<<(unsigned)((n + 127) / 128), 128, 0, st>>>(n, seed, first, Z, X, T, bad);
  count_launches(1);
  return cudaGetLastError();
}

cudaError_t launch_mlp_pack(const float* P, MlpDevWeights* Wd, cudaStream_t st) {
  pack_kernel<<<(kH * kLd + 255) / 256, 256, 0, st>>>(P, Wd);
  count_launches(1);
  return cudaGetLastError();
}

cudaError_t launch_mlp_step(const MlpDevWeights* Wd, const float* Z, const float* X,
                            const float* T, int64_t B, MlpScratch& s, float* grad, float* loss_acc,
                            cudaStream_t st) {
  const int blocks = (int)std::min<int64_t>((B / 16 + 3) / 4, 148 * 8);
  fwd_bwd_kernel<<<blocks, 128, 0, st>>>(Wd, Z, X, T, B, 1.0f / (float)B, s.HT0, s.HT1, s.HT2,
                                         s.HT3, s.DZT1, s.DZT2, s.DZT3, grad, loss_acc);
  count_launches(1);
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return e;
  const int64_t chunk = 512;
  const unsigned gk = (unsigned)((B + chunk - 1) / chunk);
  wgrad_kernel<8><<<gk, 128, 0, st>>>(s.DZT3, s.HT2, kH, B, chunk, grad + kOffW3);
  wgrad_kernel<8><<<gk, 128, 0, st>>>(s.DZT2, s.HT1, kH, B, chunk, grad + kOffW2);
  wgrad_kernel<1><<<gk, 128, 0, st>>>(s.DZT1, s.HT0, 3, B, chunk, grad + kOffW1);
  count_launches(3);
  return cudaGetLastError();
}

cudaError_t launch_mlp_adam(float* P, float* M, float* V, float* G, float lr, int64_t step,
                            cudaStream_t st) {
  const float b1 = 0.9f, b2 = 0.999f;
  const float bc1 = 1.0f - powf(b1, (float)step), bc2 = 1.0f - powf(b2, (float)step);
  adam_kernel<<<(kMlpParams + 255) / 256, 256, 0, st>>>(P, M, V, G, kMlpParams, lr, b1, b2, 1e-8f,
                                                        bc1, bc2);
  count_launches(1);
  return cudaGetLastError();
}

cudaError_t launch_mlp_eval(const MlpDevWeights* Wd, const float* Z, int64_t n, float* Y,
                            cudaStream_t st) {
  if (n == 0) return cudaSuccess;
  const int blocks = (int)std::min<int64_t>((n / 16 + 3) / 4, 148 * 16);
  eval_kernel<<<blocks, 128, 0, st>>>(Wd, Z, n, Y);
  count_launches(1);
  return cudaGetLastError();
}

cudaError_t launch_mlp_cert_points(int64_t n_cells, int samples, uint64_t seed, float* Z, float* X,
                                   unsigned int* bad, cudaStream_t st) {
  const int64_t n = n_cells * samples;
  cert_points_kernel<<<(unsigned)((n + 127) / 128), 128, 0, st>>>(n_cells, samples, seed, Z, X,
                                                                  bad);
  count_launches(1);
  return cudaGetLastError();
}

cudaError_t launch_mlp_cert_reduce(int64_t n_cells, int samples, const float* X, const float* Y,
                                   float* bound, cudaStream_t st) {
  cert_reduce_kernel<<<(unsigned)((n_cells + 255) / 256), 256, 0, st>>>(n_cells, samples, X, Y,
                                                                        bound);
  count_launches(1);
  return cudaGetLastError();
}

}  // namespace ara
