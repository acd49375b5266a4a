// ara_mlp.cuh -- the learned surrogate of InvCDF_beta: a 3 -> 64 -> 64 -> 64 -> 1 SiLU network
// evaluated and trained with warp-level BF16 tensor-core MMA (m16n8k16, FP32 accumulate).
//
// Inputs (normalised): z0 = (ln a - kLnCenter) / kLnHalf, z1 = (ln b - kLnCenter) / kLnHalf,
// z2 = logit(u) / kLogitScale; output y with logit(x) = kOutScale * y.  The three hidden layers
// run on the tensor cores with BF16 weights and FP32 accumulation (FP32 master copies live with
// the optimiser); training rounds inputs and activations to BF16, inference carries them as hi +
// lo BF16 pairs (below); the 64 -> 1 output layer is an FP32 dot product on the FP32 layer-3
// activations.  SiLU is evaluated as z * (1 + tanh(z/2)) / 2 with the hardware tanh.
//
// Register dataflow: the FP32 accumulator fragment of a layer (16 rows x 8 outputs per n-tile)
// has exactly the layout of the next layer's A fragment (16 rows x 16 inputs per k-tile) once two
// adjacent n-tiles are packed to BF16 pairs, so activations never leave registers.
#pragma once

#include <cuda_bf16.h>
#include <stdint.h>

namespace ara {

constexpr int kH = 64;                    // hidden width
constexpr int kMlpParams = 3 * kH + kH + 2 * (kH * kH + kH) + kH + 1;  // 8,641
constexpr float kLnCenter = 0.8047190f;   // (ln 0.1 + ln 50) / 2
constexpr float kLnHalf = 3.1073040f;     // (ln 50 - ln 0.1) / 2
constexpr float kLogitScale = 16.635532f; // logit(1 - 2^-24)
constexpr float kOutScale = 20.0f;
constexpr float kBoxLo = 0.1f, kBoxHi = 50.0f;  // trained (alpha, beta) box

// Weights as the kernels hold them in shared memory: BF16, rows padded to kLd elements so that
// the B-fragment loads of a warp touch 32 distinct banks.  Transposed copies serve backward.
constexpr int kLd = 72;
struct MlpSmem {               // forward (inference) weights, ~22 KB
  __nv_bfloat16 w1[kH][24];   // [out][in]: W1 in columns 0..2 and again in 3..5, 0 to 16 (+8 pad)
  __nv_bfloat16 w2[kH][kLd];  // [out][in]
  __nv_bfloat16 w3[kH][kLd];
  float w4[kH];               // output layer in FP32 on the FP32 layer-3 activations
  float b1[kH], b2[kH], b3[kH];
  float b4;
  float pad[3];
};
struct MlpSmemBwd {            // extra weights of the backward pass, ~18 KB
  __nv_bfloat16 w2t[kH][kLd]; // [in][out]
  __nv_bfloat16 w3t[kH][kLd];
};

// FP32 parameter vector layout (the optimiser's master copy): W1[64,3], b1[64], W2[64,64], b2,
// W3[64,64], b3, W4[64], b4.
constexpr int kOffW1 = 0, kOffB1 = kOffW1 + kH * 3, kOffW2 = kOffB1 + kH, kOffB2 = kOffW2 + kH * kH,
              kOffW3 = kOffB2 + kH, kOffB3 = kOffW3 + kH * kH, kOffW4 = kOffB3 + kH,
              kOffB4 = kOffW4 + kH;

#ifdef __CUDACC__

__device__ __forceinline__ uint32_t pack_bf16(float lo, float hi) {
  const __nv_bfloat162 v = __floats2bfloat162_rn(lo, hi);
  return *reinterpret_cast<const uint32_t*>(&v);
}

__device__ __forceinline__ void mma_bf16(float (&d)[4], const uint32_t (&a)[4], uint32_t b0,
                                         uint32_t b1) {
  asm volatile(
      "mma.sync.aligned.m16n8k16.row.col.f32.bf16.bf16.f32 {%0,%1,%2,%3}, {%4,%5,%6,%7}, "
      "{%8,%9}, {%0,%1,%2,%3};"
      : "+f"(d[0]), "+f"(d[1]), "+f"(d[2]), "+f"(d[3])
      : "r"(a[0]), "r"(a[1]), "r"(a[2]), "r"(a[3]), "r"(b0), "r"(b1));
}

__device__ __forceinline__ float tanh_approx(float x) {
  float y;
  asm("tanh.approx.f32 %0, %1;" : "=f"(y) : "f"(x));
  return y;
}
__device__ __forceinline__ float silu_f(float z) {
  return 0.5f * z * (1.0f + tanh_approx(0.5f * z));
}
// d silu / dz with the same tanh form: s = (1 + tanh(z/2))/2, silu' = s (1 + z (1 - s))
__device__ __forceinline__ float silu_grad_f(float z) {
  const float s = 0.5f * (1.0f + tanh_approx(0.5f * z));
  return s * (1.0f + z * (1.0f - s));
}

// One hidden layer for a 16-row tile: acc[nn][4] = A (16 x 64) * W^T + 0, W = w[64][kLd].
__device__ __forceinline__ void layer64(float (&acc)[8][4], const uint32_t (&a)[4][4],
                                        const __nv_bfloat16 (*w)[kLd], int g, int t) {
#pragma unroll
  for (int nn = 0; nn < 8; ++nn) {
    acc[nn][0] = acc[nn][1] = acc[nn][2] = acc[nn][3] = 0.f;
#pragma unroll
    for (int kk = 0; kk < 4; ++kk) {
      const __nv_bfloat16* row = &w[nn * 8 + g][kk * 16 + 2 * t];
      const uint32_t b0 = *reinterpret_cast<const uint32_t*>(row);
      const uint32_t b1 = *reinterpret_cast<const uint32_t*>(row + 8);
      mma_bf16(acc[nn], a[kk], b0, b1);
    }
  }
}

// bias + SiLU on an accumulator tile, packed as the next layer's A fragments; pre-activations
// optionally kept (pre != nullptr) for the backward pass.
__device__ __forceinline__ void act_pack(float (&acc)[8][4], const float* bias, uint32_t (&a)[4][4],
                                         int t, float (*pre)[4]) {
#pragma unroll
  for (int nn = 0; nn < 8; ++nn) {
    const float bb0 = bias[nn * 8 + 2 * t], bb1 = bias[nn * 8 + 2 * t + 1];
    acc[nn][0] += bb0; acc[nn][1] += bb1; acc[nn][2] += bb0; acc[nn][3] += bb1;
    if (pre) {
      pre[nn][0] = acc[nn][0]; pre[nn][1] = acc[nn][1];
      pre[nn][2] = acc[nn][2]; pre[nn][3] = acc[nn][3];
    }
  }
#pragma unroll
  for (int kk = 0; kk < 4; ++kk) {
    a[kk][0] = pack_bf16(silu_f(acc[2 * kk][0]), silu_f(acc[2 * kk][1]));
    a[kk][1] = pack_bf16(silu_f(acc[2 * kk][2]), silu_f(acc[2 * kk][3]));
    a[kk][2] = pack_bf16(silu_f(acc[2 * kk + 1][0]), silu_f(acc[2 * kk + 1][1]));
    a[kk][3] = pack_bf16(silu_f(acc[2 * kk + 1][2]), silu_f(acc[2 * kk + 1][3]));
  }
}

// Input fragment of layer 1 from the tile's rows: row r's z comes from lane src(r).  zr0/zr8 are
// the (z0, z1, z2) of rows g and g + 8 (already gathered by the caller).
__device__ __forceinline__ void input_frag(uint32_t (&a)[4], const float (&zr0)[3],
                                           const float (&zr8)[3], int t) {
  a[0] = t == 0 ? pack_bf16(zr0[0], zr0[1]) : (t == 1 ? pack_bf16(zr0[2], 0.f) : 0u);
  a[1] = t == 0 ? pack_bf16(zr8[0], zr8[1]) : (t == 1 ? pack_bf16(zr8[2], 0.f) : 0u);
  a[2] = 0u;
  a[3] = 0u;
}

// Output layer y = W4 . silu(a3) + b4 in FP32 from the layer-3 accumulator (bias included): this
// lane holds columns nn*8 + 2t, +1 of rows g and g + 8; the row's sum is gathered across its
// four lanes, so every lane of the row group returns it.
__device__ __forceinline__ void output_layer(const MlpSmem& W, const float (&acc)[8][4], int t,
                                             float* y0, float* y8) {
  float s0 = 0.f, s8 = 0.f;
#pragma unroll
  for (int nn = 0; nn < 8; ++nn) {
    const float w0 = W.w4[nn * 8 + 2 * t], w1 = W.w4[nn * 8 + 2 * t + 1];
    s0 = fmaf(w0, silu_f(acc[nn][0]), fmaf(w1, silu_f(acc[nn][1]), s0));
    s8 = fmaf(w0, silu_f(acc[nn][2]), fmaf(w1, silu_f(acc[nn][3]), s8));
  }
  s0 += __shfl_xor_sync(0xFFFFFFFFu, s0, 1);
  s0 += __shfl_xor_sync(0xFFFFFFFFu, s0, 2);
  s8 += __shfl_xor_sync(0xFFFFFFFFu, s8, 1);
  s8 += __shfl_xor_sync(0xFFFFFFFFu, s8, 2);
  *y0 = s0 + W.b4;
  *y8 = s8 + W.b4;
}

// Training forward pass of a 16-row tile (inputs and layer-1/2 activations rounded to BF16 once,
// the arithmetic the backward pass differentiates).  Returns y for rows g (*y0) and g + 8 (*y8)
// in all four lanes of the row group.  pre1..pre3 receive pre-activations when non-null.
__device__ __forceinline__ void mlp_tile_forward_train(const MlpSmem& W, const float (&zr0)[3],
                                                 const float (&zr8)[3], int g, int t, float* y0,
                                                 float* y8, float (*pre1)[4] = nullptr,
                                                 float (*pre2)[4] = nullptr,
                                                 float (*pre3)[4] = nullptr,
                                                 uint32_t (*h1o)[4] = nullptr,
                                                 uint32_t (*h2o)[4] = nullptr,
                                                 uint32_t (*h3o)[4] = nullptr) {
  uint32_t a0[4];
  input_frag(a0, zr0, zr8, t);
  float acc[8][4];
#pragma unroll
  for (int nn = 0; nn < 8; ++nn) {
    acc[nn][0] = acc[nn][1] = acc[nn][2] = acc[nn][3] = 0.f;
    const __nv_bfloat16* row = &W.w1[nn * 8 + g][2 * t];
    const uint32_t b0 = *reinterpret_cast<const uint32_t*>(row);
    const uint32_t b1 = *reinterpret_cast<const uint32_t*>(row + 8);
    mma_bf16(acc[nn], a0, b0, b1);
  }
  uint32_t h[4][4];
  act_pack(acc, W.b1, h, t, pre1);
  if (h1o) {
#pragma unroll
    for (int kk = 0; kk < 4; ++kk)
#pragma unroll
      for (int q = 0; q < 4; ++q) h1o[kk][q] = h[kk][q];
  }
  layer64(acc, h, W.w2, g, t);
  act_pack(acc, W.b2, h, t, pre2);
  if (h2o) {
#pragma unroll
    for (int kk = 0; kk < 4; ++kk)
#pragma unroll
      for (int q = 0; q < 4; ++q) h2o[kk][q] = h[kk][q];
  }
  layer64(acc, h, W.w3, g, t);
  act_pack(acc, W.b3, h, t, pre3);
  if (h3o) {
#pragma unroll
    for (int kk = 0; kk < 4; ++kk)
#pragma unroll
      for (int q = 0; q < 4; ++q) h3o[kk][q] = h[kk][q];
  }
  output_layer(W, acc, t, y0, y8);
}

// ---- inference: A operands carried as BF16 pairs ------------------------------------------------
// One BF16 A operand keeps 8 significant bits: an input or activation moves by up to 2^-9 of
// itself, and for the logit-u input that alone moves x by about 1e-3 near the median.  Inference
// (evaluation, certification, the trial kernel) therefore carries every A value v as
// hi = bf16(v) and lo = bf16(v - hi) (v - hi is exact in FP32), hi + lo within 2^-17 of v.  Layer 1
// takes the lo parts of its three inputs in K columns 3..5, whose weights repeat W1 (the training
// pass keeps those input columns zero); layers 2 and 3 run their MMAs on the hi and then on the lo
// fragments into one FP32 accumulator.  Weights stay the trained BF16 values.

// Two FP32 values as hi and lo BF16 pairs (low half: v0).
__device__ __forceinline__ void split_pack(float v0, float v1, uint32_t& hi, uint32_t& lo) {
  const __nv_bfloat162 h = __floats2bfloat162_rn(v0, v1);
  const float2 hf = __bfloat1622float2(h);
  const __nv_bfloat162 l = __floats2bfloat162_rn(v0 - hf.x, v1 - hf.y);
  hi = *reinterpret_cast<const uint32_t*>(&h);
  lo = *reinterpret_cast<const uint32_t*>(&l);
}

// Layer-1 A fragment: K columns 0..2 the hi parts of (z0, z1, z2), 3..5 their lo parts.
__device__ __forceinline__ void input_frag_split(uint32_t (&a)[4], const float (&zr0)[3],
                                                 const float (&zr8)[3], int t) {
  float h0[3], l0[3], h8[3], l8[3];
#pragma unroll
  for (int c = 0; c < 3; ++c) {
    h0[c] = __bfloat162float(__float2bfloat16_rn(zr0[c]));
    l0[c] = zr0[c] - h0[c];
    h8[c] = __bfloat162float(__float2bfloat16_rn(zr8[c]));
    l8[c] = zr8[c] - h8[c];
  }
  // lane t holds K columns 2t, 2t + 1 of rows g (a[0]) and g + 8 (a[1])
  a[0] = t == 0 ? pack_bf16(h0[0], h0[1])
                : (t == 1 ? pack_bf16(h0[2], l0[0]) : (t == 2 ? pack_bf16(l0[1], l0[2]) : 0u));
  a[1] = t == 0 ? pack_bf16(h8[0], h8[1])
                : (t == 1 ? pack_bf16(h8[2], l8[0]) : (t == 2 ? pack_bf16(l8[1], l8[2]) : 0u));
  a[2] = 0u;
  a[3] = 0u;
}

// bias + SiLU on an accumulator tile, as the next layer's hi and lo A fragments.
__device__ __forceinline__ void act_pack_split(float (&acc)[8][4], const float* bias,
                                               uint32_t (&hi)[4][4], uint32_t (&lo)[4][4], int t) {
#pragma unroll
  for (int nn = 0; nn < 8; ++nn) {
    const float bb0 = bias[nn * 8 + 2 * t], bb1 = bias[nn * 8 + 2 * t + 1];
    acc[nn][0] += bb0; acc[nn][1] += bb1; acc[nn][2] += bb0; acc[nn][3] += bb1;
  }
#pragma unroll
  for (int kk = 0; kk < 4; ++kk) {
    split_pack(silu_f(acc[2 * kk][0]), silu_f(acc[2 * kk][1]), hi[kk][0], lo[kk][0]);
    split_pack(silu_f(acc[2 * kk][2]), silu_f(acc[2 * kk][3]), hi[kk][1], lo[kk][1]);
    split_pack(silu_f(acc[2 * kk + 1][0]), silu_f(acc[2 * kk + 1][1]), hi[kk][2], lo[kk][2]);
    split_pack(silu_f(acc[2 * kk + 1][2]), silu_f(acc[2 * kk + 1][3]), hi[kk][3], lo[kk][3]);
  }
}

// acc += A (16 x 64) * W^T for one hidden layer (acc not cleared).
__device__ __forceinline__ void layer64_add(float (&acc)[8][4], const uint32_t (&a)[4][4],
                                            const __nv_bfloat16 (*w)[kLd], int g, int t) {
#pragma unroll
  for (int nn = 0; nn < 8; ++nn) {
#pragma unroll
    for (int kk = 0; kk < 4; ++kk) {
      const __nv_bfloat16* row = &w[nn * 8 + g][kk * 16 + 2 * t];
      const uint32_t b0 = *reinterpret_cast<const uint32_t*>(row);
      const uint32_t b1 = *reinterpret_cast<const uint32_t*>(row + 8);
      mma_bf16(acc[nn], a[kk], b0, b1);
    }
  }
}

// Inference forward pass of a 16-row tile: y for rows g (*y0) and g + 8 (*y8) in all four lanes
// of the row group.
__device__ __forceinline__ void mlp_tile_forward(const MlpSmem& W, const float (&zr0)[3],
                                                 const float (&zr8)[3], int g, int t, float* y0,
                                                 float* y8) {
  uint32_t a0[4];
  input_frag_split(a0, zr0, zr8, t);
  float acc[8][4];
#pragma unroll
  for (int nn = 0; nn < 8; ++nn) {
    acc[nn][0] = acc[nn][1] = acc[nn][2] = acc[nn][3] = 0.f;
    const __nv_bfloat16* row = &W.w1[nn * 8 + g][2 * t];
    const uint32_t b0 = *reinterpret_cast<const uint32_t*>(row);
    const uint32_t b1 = *reinterpret_cast<const uint32_t*>(row + 8);
    mma_bf16(acc[nn], a0, b0, b1);
  }
  uint32_t hh[4][4], hl[4][4];
  act_pack_split(acc, W.b1, hh, hl, t);
  layer64(acc, hh, W.w2, g, t);
  layer64_add(acc, hl, W.w2, g, t);
  act_pack_split(acc, W.b2, hh, hl, t);
  layer64(acc, hh, W.w3, g, t);
  layer64_add(acc, hl, W.w3, g, t);
#pragma unroll
  for (int nn = 0; nn < 8; ++nn) {
    const float bb0 = W.b3[nn * 8 + 2 * t], bb1 = W.b3[nn * 8 + 2 * t + 1];
    acc[nn][0] += bb0; acc[nn][1] += bb1; acc[nn][2] += bb0; acc[nn][3] += bb1;
  }
  output_layer(W, acc, t, y0, y8);
}

#endif  // __CUDACC__

// The weights as kept in device memory between kernels, already in the shared-memory layout so
// that a block copies them with plain 16-byte loads.
struct MlpDevWeights {
  MlpSmem fwd;
  MlpSmemBwd bwd;
};

}  // namespace ara
