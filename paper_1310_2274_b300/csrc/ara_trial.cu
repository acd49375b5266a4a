// ara_trial.cu -- Algorithm 1 of the paper for one layer: one warp per trial.
//
// Per trial (paper §2.2, Algorithm 1; §2.3 terms; §3.3 secondary uncertainty):
//   for each event in timestamp order, for each ELT of the layer holding it:
//       u = Philox(trial, event position, ELT handle);  loss = max_l * InvCDF_beta(u; a, b)
//   l = sum of the event's losses (layer order), o = min(max(l - OccR, 0), OccL)
//   S = sum of o over the year;  YLT[trial] = min(max(S - AggR, 0), AggL)
//
// Schedule (designed for SIMT on sm_103a, not the paper's thread-per-trial):
//   * A warp walks its trial in chunks of 128 occurrences; lane l reads occurrences
//     c + 32v + l (v = 0..3), so each of the four id loads is one coalesced 128-byte line.
//   * Each occurrence reads its 8/16-byte lookup entry (record base + ELT mask); hits are counted
//     with popc and laid out in event order by a warp scan, giving the chunk's hit list.
//   * The hit list is processed 32 hits per round, one hit per lane, so the inversion (the time
//     sink) runs with every lane busy however sparse the hits are.  A lane finds its hit's event
//     by binary search of the chunk's hit prefix in shared memory and its ELT by the n-th set bit
//     of the mask.
//   * An event's losses (contiguous in the hit list) are summed by a segmented warp scan; the
//     tail lane adds the segment to the event's shared accumulator.  The order is fixed by the
//     data, so results do not depend on the launch configuration.
//   * Occurrence terms are applied per event in FP32; the year sum S is carried per lane in FP64
//     (or Kahan-compensated FP32) and reduced across the warp at the end.
#include <cuda_runtime.h>
#include <stdint.h>

#include "ara_ibeta.cuh"
#include "ara_internal.h"
#include "ara_philox.cuh"

namespace ara {

namespace {

constexpr int kWarpsPerBlock = 8;
constexpr int kV = 4;             // occurrences per lane per chunk
constexpr int kChunk = 32 * kV;   // occurrences per chunk

struct AccF64 {
  double s = 0.0;
  __device__ void add(float o) { s += (double)o; }
  __device__ void warp_reduce() {
#pragma unroll
    for (int d = 16; d >= 1; d >>= 1) s += __shfl_xor_sync(0xFFFFFFFFu, s, d);
  }
  __device__ double value() const { return s; }
};

// Kahan-compensated binary32: the running sum is s - c.
struct AccKahan {
  float s = 0.f, c = 0.f;
  __device__ void add(float o) {
    const float y = __fsub_rn(o, c);
    const float t = __fadd_rn(s, y);
    c = __fsub_rn(__fsub_rn(t, s), y);
    s = t;
  }
  __device__ void warp_reduce() {
#pragma unroll
    for (int d = 16; d >= 1; d >>= 1) {
      const float s2 = __shfl_xor_sync(0xFFFFFFFFu, s, d);
      const float c2 = __shfl_xor_sync(0xFFFFFFFFu, c, d);
      // TwoSum(s, s2) = t + e exactly; the combined sum is t + e - c - c2.
      const float t = __fadd_rn(s, s2);
      const float bb = __fsub_rn(t, s);
      const float e = __fadd_rn(__fsub_rn(s, __fsub_rn(t, bb)), __fsub_rn(s2, bb));
      c = __fsub_rn(__fadd_rn(c, c2), e);
      s = t;
    }
  }
  __device__ double value() const { return (double)s - (double)c; }
};

template <int MW>
struct Entry;
template <>
struct Entry<1> {
  uint32_t base;
  uint32_t m0;
  __device__ static Entry load(const uint32_t* evt, int32_t e) {
    const uint2 v = __ldg(reinterpret_cast<const uint2*>(evt) + e);
    Entry r;
    r.base = v.x;
    r.m0 = v.y;
    return r;
  }
  __device__ int count() const { return __popc(m0); }
};
template <>
struct Entry<2> {
  uint32_t base;
  uint32_t m0, m1;
  __device__ static Entry load(const uint32_t* evt, int32_t e) {
    const uint4 v = __ldg(reinterpret_cast<const uint4*>(evt) + e);
    Entry r;
    r.base = v.x;
    r.m0 = v.y;
    r.m1 = v.z;
    return r;
  }
  __device__ int count() const { return __popc(m0) + __popc(m1); }
};

// Bit position of the n-th (0-based) set bit of m (n < popc(m)): clear the n lowest set bits.
__device__ __forceinline__ int nth_set_bit(uint32_t m, int n) {
  for (int i = 0; i < n; ++i) m &= m - 1u;
  return __ffs(m) - 1;
}

__device__ __forceinline__ BetaRec load_rec(const BetaRec* p) {
  const float4* q = reinterpret_cast<const float4*>(p);
  const float4 u = __ldg(q);
  const float4 v = __ldg(q + 1);
  BetaRec r;
  r.a = u.x; r.b = u.y; r.mx = u.z; r.L0 = u.w;
  r.p0 = v.x; r.lnx0 = v.y; r.lny0 = v.z; r.lns = v.w;
  return r;
}

template <int MW, class Acc, bool TRACE>
__global__ void __launch_bounds__(kWarpsPerBlock * 32)
    trial_kernel(const __grid_constant__ TrialParams P) {
  __shared__ int32_t s_excl[kWarpsPerBlock][kChunk];
  __shared__ uint32_t s_base[kWarpsPerBlock][kChunk];
  __shared__ uint32_t s_mask[kWarpsPerBlock][MW][kChunk];
  __shared__ float s_lsum[kWarpsPerBlock][kChunk];

  const int lane = threadIdx.x & 31;
  const int wib = threadIdx.x >> 5;
  const int64_t w = (int64_t)blockIdx.x * kWarpsPerBlock + wib;
  if (w >= P.n) return;  // whole warp leaves together; no block-wide barrier follows
  const int64_t trial = P.t0 + w;
  const int64_t beg = P.offsets[trial];
  const int64_t end = P.offsets[trial + 1];

  int32_t* excl = s_excl[wib];
  uint32_t* sbase = s_base[wib];
  float* lsum = s_lsum[wib];

  Acc acc;
  int32_t trace_n = 0;
  unsigned int nc = 0;
  unsigned int n_inv = 0, n_it = 0, n_cf = 0, n_hit = 0;

  for (int64_t c = beg; c < end; c += kChunk) {
    // ---- stream ids, look up entries, lay out the chunk's hits in event order ---------------
    int32_t run = 0;
#pragma unroll
    for (int v = 0; v < kV; ++v) {
      const int64_t q = c + v * 32 + lane;
      Entry<MW> en;
      en.base = 0;
      en.m0 = 0;
      if constexpr (MW == 2) en.m1 = 0;
      if (q < end) en = Entry<MW>::load(P.evt, __ldg(P.ids + q));
      const int cnt = en.count();
      int incl = cnt;
#pragma unroll
      for (int d = 1; d < 32; d <<= 1) {
        const int t = __shfl_up_sync(0xFFFFFFFFu, incl, d);
        if (lane >= d) incl += t;
      }
      const int idx = v * 32 + lane;
      excl[idx] = run + incl - cnt;
      sbase[idx] = en.base;
      s_mask[wib][0][idx] = en.m0;
      if constexpr (MW == 2) s_mask[wib][1][idx] = en.m1;
      lsum[idx] = 0.f;
      run += __shfl_sync(0xFFFFFFFFu, incl, 31);
    }
    __syncwarp();

    // ---- 32 hits per round: uniform draw, inverse beta, per-event segmented sum ------------
    for (int32_t r0 = 0; r0 < run; r0 += 32) {
      const int32_t g = r0 + lane;
      const bool has = g < run;
      int ev = 0;
      float loss = 0.f;
      if (has) {
        // largest event index whose exclusive prefix is <= g
#pragma unroll
        for (int step = kChunk / 2; step >= 1; step >>= 1)
          if (excl[ev + step] <= g) ev += step;
        const int nth = g - excl[ev];
        int slot;
        if constexpr (MW == 1) {
          slot = nth_set_bit(s_mask[wib][0][ev], nth);
        } else {
          const uint32_t m0 = s_mask[wib][0][ev];
          const int c0 = __popc(m0);
          slot = nth < c0 ? nth_set_bit(m0, nth) : 32 + nth_set_bit(s_mask[wib][1][ev], nth - c0);
        }
        const uint32_t pos = sbase[ev] + (uint32_t)nth;
        const BetaRec rec = load_rec(P.recs + pos);
        const uint32_t k = (uint32_t)(c - beg) + (uint32_t)ev;
        float u = 0.f, x = __int_as_float(0x7FC00000);
        if (rec.a > 0.f) {
          u = su_uniform(P.seed, trial, k, P.handles[slot]);
          const IbetaResult ib = ara_inv_beta(rec, u);
          x = ib.x;
          nc += ib.converged ? 0u : 1u;
          n_inv += 1u;
          n_it += (unsigned)ib.iters;
          n_cf += (unsigned)ib.cf_terms;
          loss = rec.mx * x;
        } else {
          loss = rec.mx;  // sd = 0: the mean (primary uncertainty only)
          if (TRACE) u = su_uniform(P.seed, trial, k, P.handles[slot]);
        }
        if constexpr (TRACE) {
          const int32_t th = trace_n + g;
          if (th < P.trace_cap) {
            const int64_t o = w * P.trace_cap + th;
            P.tr_k[o] = (int32_t)k;
            P.tr_j[o] = slot;
            P.tr_rec[o] = (int32_t)P.rec_idx[pos];
            P.tr_u[o] = u;
            P.tr_x[o] = x;
            P.tr_loss[o] = loss;
          }
        }
      }
      // segmented inclusive scan over lanes: segments are the runs of equal ev
      const int seg = has ? ev : -1;
      float val = loss;
#pragma unroll
      for (int d = 1; d < 32; d <<= 1) {
        const float nv = __shfl_up_sync(0xFFFFFFFFu, val, d);
        const int ns = __shfl_up_sync(0xFFFFFFFFu, seg, d);
        if (lane >= d && ns == seg) val += nv;
      }
      const int next_seg = __shfl_down_sync(0xFFFFFFFFu, seg, 1);
      const bool tail = has && (lane == 31 || next_seg != seg);
      if (tail) lsum[ev] += val;
      __syncwarp();
    }
    if constexpr (TRACE) trace_n += run;
    n_hit += (lane == 0) ? (unsigned)run : 0u;

    // ---- occurrence terms and the year's running sum -----------------------------------------
#pragma unroll
    for (int v = 0; v < kV; ++v) {
      const int64_t q = c + v * 32 + lane;
      if (q < end) {
        const float l = lsum[v * 32 + lane];
        const float o = fminf(fmaxf(l - P.occ_ret, 0.f), P.occ_lim);
        acc.add(o);
      }
    }
    __syncwarp();
  }

  acc.warp_reduce();
  nc = __reduce_add_sync(0xFFFFFFFFu, nc);
  n_inv = __reduce_add_sync(0xFFFFFFFFu, n_inv);
  n_it = __reduce_add_sync(0xFFFFFFFFu, n_it);
  n_cf = __reduce_add_sync(0xFFFFFFFFu, n_cf);
  if (lane == 0) {
    const double S = acc.value();
    P.ylt[w] = fmin(fmax(S - P.agg_ret, 0.0), P.agg_lim);
    if (nc) atomicAdd(P.not_conv, (unsigned long long)nc);
    atomicAdd(P.stats + 0, (unsigned long long)n_inv);
    atomicAdd(P.stats + 1, (unsigned long long)n_it);
    atomicAdd(P.stats + 2, (unsigned long long)n_cf);
    atomicAdd(P.stats + 3, (unsigned long long)n_hit);
    if constexpr (TRACE) P.tr_count[w] = trace_n;
  }
}

template <int MW, class Acc, bool TRACE>
cudaError_t launch_one(const TrialParams& p, cudaStream_t st) {
  const int64_t blocks = (p.n + kWarpsPerBlock - 1) / kWarpsPerBlock;
  if (blocks == 0) return cudaSuccess;
  trial_kernel<MW, Acc, TRACE><<<(unsigned)blocks, kWarpsPerBlock * 32, 0, st>>>(p);
  count_launches(1);
  return cudaGetLastError();
}

}  // namespace

cudaError_t launch_trial(const TrialParams& p, int mask_words, int precision, bool trace,
                         cudaStream_t st) {
  if (trace) {
    return mask_words == 1 ? launch_one<1, AccF64, true>(p, st)
                           : launch_one<2, AccF64, true>(p, st);
  }
  if (precision == 1) {
    return mask_words == 1 ? launch_one<1, AccKahan, false>(p, st)
                           : launch_one<2, AccKahan, false>(p, st);
  }
  return mask_words == 1 ? launch_one<1, AccF64, false>(p, st)
                         : launch_one<2, AccF64, false>(p, st);
}

}  // namespace ara
