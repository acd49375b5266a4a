// ara_philox.cuh -- counter-based uniforms for secondary uncertainty.
//
// The paper draws its uncertainty from pre-stored uniforms z_(Prog,E) per occurrence and z_(E)
// per XELT record (§3.1).  Here a single uniform per (trial, event position, ELT) is generated
// on the fly by Philox4x32-10 (Salmon, Moraes, Dror & Shaw, "Parallel Random Numbers: As Easy
// as 1, 2, 3", SC'11): ten rounds of two 32x32->64 multiplications by the constants
// 0xD2511F53 and 0xCD9E8D57, word permutation and xor with the key, the key advanced between
// rounds by the Weyl increments 0x9E3779B9 and 0xBB67AE85.  With one standard deviation per
// record (sigma_C = 0) the normal-copula combination of §3.2 returns its input uniform
// unchanged, so the uniform feeds the beta inversion directly.
#pragma once

#include <stdint.h>

namespace ara {

struct U4 {
  uint32_t x, y, z, w;
};

__device__ __forceinline__ U4 philox4x32_10(U4 c, uint32_t k0, uint32_t k1) {
#pragma unroll
  for (int r = 0; r < 10; ++r) {
    const uint32_t lo0 = 0xD2511F53u * c.x;
    const uint32_t hi0 = __umulhi(0xD2511F53u, c.x);
    const uint32_t lo1 = 0xCD9E8D57u * c.z;
    const uint32_t hi1 = __umulhi(0xCD9E8D57u, c.z);
    U4 n;
    n.x = hi1 ^ c.y ^ k0;
    n.y = lo1;
    n.z = hi0 ^ c.w ^ k1;
    n.w = lo0;
    c = n;
    k0 += 0x9E3779B9u;
    k1 += 0xBB67AE85u;
  }
  return c;
}

// The same generator with the round keys given (rk0[r], rk1[r] = key words of round r), so that
// a kernel can take them from its launch parameters instead of advancing the key per call.
__device__ __forceinline__ U4 philox4x32_10_rk(U4 c, const uint32_t* rk0, const uint32_t* rk1) {
#pragma unroll
  for (int r = 0; r < 10; ++r) {
    const uint64_t p0 = (uint64_t)0xD2511F53u * c.x;  // one 32x32 -> 64-bit product each
    const uint64_t p1 = (uint64_t)0xCD9E8D57u * c.z;
    U4 n;
    n.x = (uint32_t)(p1 >> 32) ^ c.y ^ rk0[r];
    n.y = (uint32_t)p1;
    n.z = (uint32_t)(p0 >> 32) ^ c.w ^ rk1[r];
    n.w = (uint32_t)p0;
    c = n;
  }
  return c;
}

// Round keys of the key (seed_lo, seed_hi), as philox4x32_10 advances them.
inline void philox_round_keys(uint64_t seed, uint32_t* rk0, uint32_t* rk1) {
  uint32_t k0 = (uint32_t)(seed & 0xFFFFFFFFu), k1 = (uint32_t)(seed >> 32);
  for (int r = 0; r < 10; ++r) {
    rk0[r] = k0;
    rk1[r] = k1;
    k0 += 0x9E3779B9u;
    k1 += 0xBB67AE85u;
  }
}

// Upper 23 bits j of w -> (2j+1) 2^-24: exact in binary32, in [2^-24, 1 - 2^-24], and the grid is
// symmetric so 1 - u is exact as well.
__device__ __forceinline__ float word_to_uniform(uint32_t w) {
  return __uint2float_rn(((w >> 9) << 1) | 1u) * 5.9604644775390625e-8f;  // * 2^-24
}

// Uniform of occurrence k of trial i in the ELT with handle elt:
// counter (k, i_lo, elt/4, i_hi), key (seed_lo, seed_hi), output word elt mod 4.
__device__ __forceinline__ float su_uniform(uint64_t seed, int64_t trial, uint32_t k, int32_t elt) {
  U4 c;
  c.x = k;
  c.y = (uint32_t)((uint64_t)trial & 0xFFFFFFFFu);
  c.z = (uint32_t)elt >> 2;
  c.w = (uint32_t)((uint64_t)trial >> 32);
  const U4 o = philox4x32_10(c, (uint32_t)(seed & 0xFFFFFFFFu), (uint32_t)(seed >> 32));
  const int q = elt & 3;
  const uint32_t w = q == 0 ? o.x : (q == 1 ? o.y : (q == 2 ? o.z : o.w));
  return word_to_uniform(w);
}

// su_uniform with precomputed round keys.
__device__ __forceinline__ float su_uniform_rk(const uint32_t* rk0, const uint32_t* rk1,
                                               int64_t trial, uint32_t k, int32_t elt) {
  U4 c;
  c.x = k;
  c.y = (uint32_t)((uint64_t)trial & 0xFFFFFFFFu);
  c.z = (uint32_t)elt >> 2;
  c.w = (uint32_t)((uint64_t)trial >> 32);
  const U4 o = philox4x32_10_rk(c, rk0, rk1);
  const int q = elt & 3;
  const uint32_t w = q == 0 ? o.x : (q == 1 ? o.y : (q == 2 ? o.z : o.w));
  return word_to_uniform(w);
}

// The correlated (event-occurrence) uniform of occurrence k of trial i, shared by every ELT and
// layer (paper §3.1, z_(E)): counter (k, i_lo, 0xFFFFFFFF, i_hi), a group no ELT handle reaches,
// output word 0.
__device__ __forceinline__ float su_uniform_corr_rk(const uint32_t* rk0, const uint32_t* rk1,
                                                    int64_t trial, uint32_t k) {
  U4 c;
  c.x = k;
  c.y = (uint32_t)((uint64_t)trial & 0xFFFFFFFFu);
  c.z = 0xFFFFFFFFu;
  c.w = (uint32_t)((uint64_t)trial >> 32);
  return word_to_uniform(philox4x32_10_rk(c, rk0, rk1).x);
}

}  // namespace ara
