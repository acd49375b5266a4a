// ara_trial_common.cuh -- device pieces shared by the trial-major and the band-major kernels of
// Algorithm 1: year-sum accumulators, L2 cache policies, lookup-entry loads, record loads.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include "ara_ibeta.cuh"
#include "ara_internal.h"

namespace ara {
namespace {

// Year-sum accumulators.  make() starts a sum for the launch item P; add() takes one
// occurrence's result; warp_reduce() combines the 32 lanes; value() is the year sum S.
//
// AccExact (ARA_ACC_FP64): each binary32 occurrence result is rounded to a multiple of the
// item's grid unit 2^e and summed exactly in 64-bit integers.  e is chosen per launch so that the
// longest trial times the largest occurrence result the layer's records allow (the sum of an
// event's loss bounds less OccR, at most OccL) fits in 2^62 units; S = units x 2^e is rounded
// once to binary64.  The integer sum is independent of the order and grouping of the additions,
// so every schedule gives the same S.
struct AccExact {
  unsigned long long s = 0;
  float qs = 1.0f;    // 2^-e
  double unit = 1.0;  // 2^e
  __device__ static AccExact make(const TrialParams& P) {
    AccExact a;
    a.qs = P.q_scale;
    a.unit = P.q_unit;
    return a;
  }
  __device__ static unsigned long long units(float o, float qs) {
    return __float2ull_rn(o * qs);  // o >= 0; the scaling by 2^-e is exact
  }
  __device__ void add(float o) { s += units(o, qs); }
  __device__ void warp_reduce() {
#pragma unroll
    for (int d = 16; d >= 1; d >>= 1) s += __shfl_xor_sync(0xFFFFFFFFu, s, d);
  }
  __device__ double value() const { return (double)s * unit; }
};

// ARA_ACC_KAHAN32: Kahan-compensated binary32 in occurrence order per lane, lanes combined by
// TwoSum; the running sum is s - c.
struct AccKahan {
  float s = 0.f, c = 0.f;
  __device__ static AccKahan make(const TrialParams&) { return AccKahan(); }
  __device__ void add(float o) {
    const float y = __fsub_rn(o, c);
    const float t = __fadd_rn(s, y);
    c = __fsub_rn(__fsub_rn(t, s), y);
    s = t;
  }
  // TwoSum(s, o.s) = t + e exactly; the combined sum is t + e - c - o.c.
  __device__ void merge(const AccKahan& o) {
    const float t = __fadd_rn(s, o.s);
    const float bb = __fsub_rn(t, s);
    const float e = __fadd_rn(__fsub_rn(s, __fsub_rn(t, bb)), __fsub_rn(o.s, bb));
    c = __fsub_rn(__fadd_rn(c, o.c), e);
    s = t;
  }
  __device__ void warp_reduce() {
#pragma unroll
    for (int d = 16; d >= 1; d >>= 1) {
      AccKahan o;
      o.s = __shfl_xor_sync(0xFFFFFFFFu, s, d);
      o.c = __shfl_xor_sync(0xFFFFFFFFu, c, d);
      merge(o);
    }
  }
  __device__ double value() const { return (double)s - (double)c; }
};

// L2 residency (sm_100+ cache policies).  Per launch the kernel streams the 3.2 GB event-id
// stream and, on the table path, one random 32-byte table piece per hit from tables of several
// GB; both are read once and marked evict-first.  The lookup index and the record headers
// (~45 MB, reused every few microseconds) are marked evict-last so the stream does not push them
// out of the 126 MB L2.
struct L2Policies {
  unsigned long long keep, stream;
  __device__ static L2Policies make() {
    L2Policies p;
    asm volatile("createpolicy.fractional.L2::evict_last.b64 %0, 1.0;" : "=l"(p.keep));
    asm volatile("createpolicy.fractional.L2::evict_first.b64 %0, 1.0;" : "=l"(p.stream));
    return p;
  }
};

__device__ __forceinline__ int32_t ld_stream_s32(const int32_t* p, unsigned long long pol) {
  int32_t v;
  asm volatile("ld.global.nc.L1::no_allocate.L2::cache_hint.s32 %0, [%1], %2;"
               : "=r"(v) : "l"(p), "l"(pol));
  return v;
}
// Gathers of 8 or 16 bytes at random addresses (index entries, records, start pieces), with an L2
// policy; a miss fills 64 bytes rather than the default 128.
__device__ __forceinline__ uint2 ld_pol_u2(const uint2* p, unsigned long long pol) {
  uint2 v;
  asm volatile("ld.global.nc.L2::cache_hint.L2::64B.v2.u32 {%0,%1}, [%2], %3;"
               : "=r"(v.x), "=r"(v.y) : "l"(p), "l"(pol));
  return v;
}
__device__ __forceinline__ uint4 ld_pol_u4(const uint4* p, unsigned long long pol) {
  uint4 v;
  asm volatile("ld.global.nc.L2::cache_hint.L2::64B.v4.u32 {%0,%1,%2,%3}, [%4], %5;"
               : "=r"(v.x), "=r"(v.y), "=r"(v.z), "=r"(v.w) : "l"(p), "l"(pol));
  return v;
}

template <int MW>
struct Entry;
template <>
struct Entry<1> {
  uint32_t base;
  uint32_t m0;
  __device__ static Entry load(const uint32_t* evt, int32_t e, unsigned long long pol) {
    const uint2 v = ld_pol_u2(reinterpret_cast<const uint2*>(evt) + e, pol);
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
  __device__ static Entry load(const uint32_t* evt, int32_t e, unsigned long long pol) {
    const uint4 v = ld_pol_u4(reinterpret_cast<const uint4*>(evt) + e, pol);
    Entry r;
    r.base = v.x;
    r.m0 = v.y;
    r.m1 = v.z;
    return r;
  }
  __device__ int count() const { return __popc(m0) + __popc(m1); }
};

// The uniform a hit's inversion receives (paper §3.2).  u is the hit's own uniform (z_(Prog,E));
// with a correlated weight cc > 0 the occurrence's shared uniform uc (z_(E)) enters through
// v = sqrt(1 - cc^2) Phi^-1(u) + cc Phi^-1(uc), z = Phi(v); the table receives the tail side and
// q = Phi(-|v|), which keeps its precision where z is close to 1.  cc = 0 returns u itself.
struct SuDraw {
  bool lower;  // z < 1/2
  float q;     // min(z, 1 - z)
  float z;
};
__device__ __forceinline__ SuDraw su_draw(float u, float uc, float cc) {
  SuDraw d;
  if (!(cc > 0.0f)) {
    d.lower = u < 0.5f;
    d.q = d.lower ? u : 1.0f - u;
    d.z = u;
    return d;
  }
  const float v = sqrtf(fmaxf(1.0f - cc * cc, 0.0f)) * normcdfinvf(u) + cc * normcdfinvf(uc);
  d.lower = v < 0.0f;
  d.q = normcdff(-fabsf(v));
  d.z = d.lower ? d.q : 1.0f - d.q;
  return d;
}

// Bit position of the n-th (0-based) set bit of m (n < popc(m)): clear the n lowest set bits,
// then find the lowest.  n is the hit's rank within its event, almost always 0 or 1, so this
// short loop beats a general n-th-bit search (1.6% of the band kernel's time).
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


// A hit's 32-byte record and its start-table piece (one 32-byte sector) under an L2 policy:
// evict-last for records, which both schedules reuse from L2 (57 MB at paper scale); the band
// schedule keeps its band's start tables too, the trial-major schedule streams them (919 MB
// swept at random).
__device__ __forceinline__ BetaRec load_rec_policy(const BetaRec* p, unsigned long long pol) {
  const uint4 a = ld_pol_u4(reinterpret_cast<const uint4*>(p), pol);
  const uint4 b = ld_pol_u4(reinterpret_cast<const uint4*>(p) + 1, pol);
  BetaRec r;
  r.a = __uint_as_float(a.x); r.b = __uint_as_float(a.y);
  r.mx = __uint_as_float(a.z); r.L0 = __uint_as_float(a.w);
  r.p0 = __uint_as_float(b.x); r.lnx0 = __uint_as_float(b.y);
  r.lny0 = __uint_as_float(b.z); r.lns = __uint_as_float(b.w);
  return r;
}

// ara_start_logit with the piece loaded under the policy pol.
__device__ __forceinline__ float start_logit_policy(const float* st, float u,
                                                    unsigned long long pol) {
  float tau;
  const int k = ara_start_piece(u, &tau);
  const uint4* c4 = reinterpret_cast<const uint4*>(st + k * kStartStride);
  const uint4 a = ld_pol_u4(c4, pol);
  const uint2 b = ld_pol_u2(reinterpret_cast<const uint2*>(c4 + 1), pol);
  return ara_start_poly(make_float2(__uint_as_float(a.x), __uint_as_float(a.y)),
                        make_float2(__uint_as_float(a.z), __uint_as_float(a.w)),
                        make_float2(__uint_as_float(b.x), __uint_as_float(b.y)), tau);
}

// The Newton inversion for the rare record whose table failed certification (and for the
// surrogate's rejected cells), kept out of line so that its registers do not weigh on the table
// path; ONE_CF as for ara_inv_beta.
template <bool ONE_CF>
__device__ __noinline__ IbetaResult newton_fallback(const BetaRec* p, float u) {
  return ara_inv_beta<ONE_CF>(load_rec(p), u);
}

}  // namespace
}  // namespace ara
