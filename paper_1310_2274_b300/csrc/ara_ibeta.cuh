// ara_ibeta.cuh -- FP32 inverse of the regularised incomplete beta function, for one lane.
//
// Paper §3.3: Loss = max_l * InvCDF_beta(z; alpha, beta), where InvCDF_beta is the functional
// inverse of I_x(alpha, beta) = B(x; alpha, beta) / B(alpha, beta).  This is the time sink of
// the method (paper §5.1: most of the secondary-uncertainty time is spent in it).
//
// Formulation (chosen for SIMT execution in binary32):
//   * Per-record constants are computed once, in FP64, when an ELT is staged: alpha, beta and
//       L0 = alpha ln x0 + beta ln y0 - ln B(alpha, beta),   x0 = alpha/(alpha+beta), y0 = 1-x0.
//     With them the beta prefactor x^a y^b / B(a,b) = exp(L0 + a ln(x/x0) + b ln(y/y0)), whose
//     exponent is O(1) near the bulk of the distribution, so binary32 keeps it accurate without
//     any per-hit lgamma (the cancellation of large log-gamma values happens once, in FP64).
//   * I_x(a,b) = prefactor * K / a with K the continued fraction of DLMF 8.17.22, evaluated
//     back-to-front-free by the forward (Wallis) three-term recurrence after an equivalence
//     transformation that clears every division: partial numerators
//       alpha_1 = -(a+b) x,  alpha_{2m+1} = -(a+m)(a+b+m) x,  alpha_{2m} = m(b-m) x,
//     partial denominators a+n.  Numerator and denominator are rescaled by exact powers of two.
//     Past x = (a+1)/(a+b+2) the symmetric fraction for I_{1-x}(b,a) is used (DLMF 8.17.4).
//   * The root of I_x = p is found by Newton's method in t = ln x from a start given by the
//     small-x limit of DLMF 8.17.22 or, for a, b > 1, by the normal approximation of
//     Abramowitz & Stegun 26.5.22 with the normal quantile of A&S 26.2.23.  The tail below the
//     mean is always the one solved (the other through 1 - u, exact on the uniform grid).
//   * Iterations are capped; a lane that reaches the cap reports it (no trap, no spin).
#pragma once

#ifndef ARA_HD
#ifdef __CUDACC__
#define ARA_HD __host__ __device__ __forceinline__
#else
#include <cmath>
#define ARA_HD inline
#endif
#endif

#include <stdint.h>

#ifndef __CUDACC__
#include <cmath>
#include <cstring>
using std::isfinite;
struct float4 {
  float x, y, z, w;
};
#endif

namespace ara {
ARA_HD float4 ara_make_float4(float x, float y, float z, float w) {
  float4 v;
  v.x = x; v.y = y; v.z = z; v.w = w;
  return v;
}
}  // namespace ara

namespace ara {

struct IbetaResult {
  float x;        // quantile in [0,1]
  float t;        // ln of the unknown actually solved for (x, or 1-x when the tail flipped);
                  // finite even where that unknown underflows binary32
  int iters;      // Newton iterations used
  int cf_terms;   // continued-fraction terms summed
  bool converged;
};

constexpr int kIbetaMaxIter = 12;
constexpr int kCfMaxTerms = 160;

// Multiply by 2^-e exactly, e taken from the exponent field of s (s finite, nonzero).
ARA_HD float ara_pow2_scale_of(float s) {
#ifdef __CUDA_ARCH__
  int bits = __float_as_int(s);
#else
  int bits;
  memcpy(&bits, &s, 4);
#endif
  int e = ((bits >> 23) & 0xFF) - 127;
  int sb = (127 - e) << 23;  // 2^-e as binary32 (e in [-126, 127])
  float r;
#ifdef __CUDA_ARCH__
  r = __int_as_float(sb);
#else
  memcpy(&r, &sb, 4);
#endif
  return r;
}

// K(a,b,x) = 1/(1 + d1/(1 + d2/(...))) of DLMF 8.17.22 by the Wallis recurrence on the
// division-free equivalent fraction T = 1 + alpha_1/(beta_1 + alpha_2/(beta_2 + ...)), K = 1/T.
// Converges quickly for x < (a+1)/(a+b+2).  Returns K; *terms counts recurrence steps.
ARA_HD float ara_beta_cf(float a, float b, float x, int* terms) {
  const float apb = a + b;
  // T_n = A_n / B_n.  A_{-1} = 1, A_0 = 1; B_{-1} = 0, B_0 = 1.
  float Am2 = 1.0f, Am1 = 1.0f, Bm2 = 0.0f, Bm1 = 1.0f;
  float prev = 1.0f;
  float res = 1.0f;
  int n = 1;
  for (; n <= kCfMaxTerms; n += 2) {
    // odd step n = 2m+1: alpha = -(a+m)(a+b+m) x  (alpha_1 = -(a+b) x: the a cancels)
    const float m = 0.5f * (float)(n - 1);
    const float al_odd = (n == 1) ? -apb * x : -(a + m) * (apb + m) * x;
    const float be_odd = a + (float)n;
    float A = be_odd * Am1 + al_odd * Am2;
    float B = be_odd * Bm1 + al_odd * Bm2;
    Am2 = Am1; Bm2 = Bm1; Am1 = A; Bm1 = B;
    // even step n+1 = 2(m+1): alpha = (m+1)(b-m-1) x
    const float m2 = m + 1.0f;
    const float al_even = m2 * (b - m2) * x;
    const float be_even = a + (float)(n + 1);
    A = be_even * Am1 + al_even * Am2;
    B = be_even * Bm1 + al_even * Bm2;
    Am2 = Am1; Bm2 = Bm1; Am1 = A; Bm1 = B;
    // exact power-of-two rescale keeps the recurrence inside binary32 range
    const float sc = ara_pow2_scale_of(Am1);
    Am1 *= sc; Am2 *= sc; Bm1 *= sc; Bm2 *= sc;
    if (((n + 1) & 3) == 0 || n + 2 > kCfMaxTerms) {
      res = Bm1 / Am1;
      if (fabsf(res - prev) <= 1.2e-7f * fabsf(res)) { n += 2; break; }
      prev = res;
    }
  }
  if (terms) *terms += n - 1;
  return res;
}

// Normal quantile for the upper tail probability q in (0, 1/2]: the deviate t with
// Q(t) = q, by the rational approximation A&S 26.2.23 (|error| < 4.5e-4).  Used only for a start.
ARA_HD float ara_norm_upper_quantile(float q) {
  const float t = sqrtf(-2.0f * logf(q));
  const float num = 2.515517f + t * (0.802853f + t * 0.010328f);
  const float den = 1.0f + t * (1.432788f + t * (0.189269f + t * 0.001308f));
  return t - num / den;
}

// One ELT record as the device uses it (32 bytes, one L2 sector).  All fields are derived once
// per record, in FP64, from (mean, sd, max) when an ELT is staged (paper §3.3):
//   a, b   alpha and beta of the moment-matched beta distribution (sd clamped as in §3.3);
//          a = 0 marks a record with sd = 0, whose loss is the mean (primary uncertainty only);
//   mx     max_l, the scale of the loss (for a = 0: the mean itself);
//   L0     a ln x0 + b ln y0 - ln B(a,b), x0 = a/(a+b), y0 = b/(a+b) (symmetric in a, b);
//   p0     I_{x0}(a,b), the probability below the mean: u <= p0 puts the root below x0;
//   lnx0, lny0, lns   ln x0, ln y0, ln(a+b).
struct BetaRec {
  float a, b, mx, L0;
  float p0, lnx0, lny0, lns;
};

// Solve I_x(a,b) = u for x, x in [0,1].
//
// Newton's method on G(t) = ln I_{e^t}(a,b) - ln p in t = ln x.  Below the threshold
// x = (a+1)/(a+b+2), I_x = P K / a with P the prefactor, so G = E + ln(K/a) - ln p and
// G'(t) = x f(x) / I_x = a / ((1-x) K): no exponential is needed.  In the lower tail G is nearly
// linear in t (I_x ~ x^a), which is where Newton in x fails for a < 1.
//
// The tail is chosen per record: if u > p0 the root lies above the mean, and the symmetric
// problem I_y(b,a) = 1 - u (exact on the uniform grid) is solved for y = 1 - x instead, so the
// unknown solved for is always below the mean of its distribution.
ARA_HD IbetaResult ara_inv_beta(const BetaRec& rec, float u) {
  IbetaResult r;
  r.iters = 0;
  r.cf_terms = 0;
  r.converged = true;
  r.t = 0.0f;
  const bool flip = u > rec.p0;
  const float p = flip ? 1.0f - u : u;
  const float a = flip ? rec.b : rec.a;
  const float b = flip ? rec.a : rec.b;
  const float lnx0 = flip ? rec.lny0 : rec.lnx0;
  const float lny0 = flip ? rec.lnx0 : rec.lny0;
  const float L0 = rec.L0;
  const float s = a + b;
  const float lna = lnx0 + rec.lns;
  const float lnp = logf(p);

  // ---- start --------------------------------------------------------------------------------
  // small-x limit of DLMF 8.17.22 (K -> 1, y -> 1): ln p = L0 + a ln(x/x0) - b ln y0 - ln a
  float t = lnx0 + (lnp + lna - L0 + b * lny0) / a;
  if (a > 1.0f && b > 1.0f) {
    // A&S 26.5.22: x ~ a / (a + b e^{2w}), with yp the upper-tail normal deviate of p.
    const float yp = ara_norm_upper_quantile(fminf(p, 0.5f));
    const float ypl = p > 0.5f ? -ara_norm_upper_quantile(1.0f - p) : yp;
    const float lam = (ypl * ypl - 3.0f) / 6.0f;
    const float h = 2.0f / (1.0f / (2.0f * a - 1.0f) + 1.0f / (2.0f * b - 1.0f));
    const float w = ypl * sqrtf(fmaxf(h + lam, 0.0f)) / h -
                    (1.0f / (2.0f * b - 1.0f) - 1.0f / (2.0f * a - 1.0f)) *
                        (lam + 5.0f / 6.0f - 2.0f / (3.0f * h));
    t = lna - logf(a + b * expf(2.0f * w));
  }
  t = fminf(t, lnx0);  // the root is below the mean
  // Below e^-69 ~ 1e-30 the loss max_l * x is far under every term of a year loss.
  if (!(t > -69.0f)) { r.x = flip ? 1.0f : 0.0f; r.t = t; return r; }

  // ---- Newton iterations in t ---------------------------------------------------------------
  const float thr = (a + 1.0f) / (s + 2.0f);
  bool done = false;
  int it = 0;
  float x = expf(t);
  for (; it < kIbetaMaxIter; ++it) {
    const float y = 1.0f - x;
    // E = ln(x^a y^b / B(a,b)) = L0 + a ln(x/x0) + b ln(y/y0), w = (x - x0)(a + b)
    const float w = fmaf(x, s, -a);
    const float rx = w / a;   // x/x0 - 1
    const float ry = -w / b;  // y/y0 - 1
    const float lnrx = rx > -0.5f ? log1pf(rx) : t - lnx0;
    const float lnry = ry > -0.5f ? log1pf(ry) : logf(y) - lny0;
    const float E = L0 + a * lnrx + b * lnry;
    float G, dG;
    if (x < thr) {
      const float K = ara_beta_cf(a, b, x, &r.cf_terms);
      G = E + logf(K) - lna - lnp;
      dG = a / (y * K);
    } else {
      const float P = expf(E);
      const float J = P * ara_beta_cf(b, a, y, &r.cf_terms) / b;  // I_{1-x}(b,a)
      G = log1pf(-J) - lnp;
      dG = P / (y * (1.0f - J));
    }
    float tn = t - G / dG;
    if (!(tn < 0.0f)) tn = 0.5f * t;  // a step past x = 1 is halved toward it
    const float step = fabsf(tn - t);
    t = tn;
    x = expf(t);
    if (step <= 3.0e-5f) { done = true; ++it; break; }
    if (!(t > -69.0f)) { done = true; ++it; x = 0.0f; break; }
  }
  r.iters = it;
  r.converged = done;
  r.t = t;
  r.x = flip ? 1.0f - x : x;
  return r;
}

// ---- certified per-record quantile tables ---------------------------------------------------------
//
// Each record's (alpha, beta) is fixed and is met hundreds of times per run, so its quantile
// function is tabulated once, when the ELT is staged.  The two tails are tabulated separately:
// below the mean (u <= p0) the table maps t = sqrt(-2 ln u) to r = ln x; above it, t =
// sqrt(-2 ln(1-u)) to r = ln(1-x).  In t the quantile's log is smooth and nearly quadratic in the
// tails (ln x ~ (ln u)/a), so kTableIntervals quintic Hermite pieces per tail, built from r and its
// first two derivatives at uniformly spaced knots, reproduce it to ~1e-8; every piece is checked
// at its midpoint when the table is built, and a record whose table misses the bound keeps the
// Newton inversion.  One piece is 6 binary32 coefficients of a polynomial in the local coordinate
// tau in [0,1], padded to 32 bytes (one sector); the record header is 16 bytes.
constexpr int kTableIntervals = 32;
// t at the smallest uniform on the grid, 2^-24: sqrt(48 ln 2)
constexpr float kTableTHi = 5.76832104f;

// A record's table header: 32 bytes, one L2 sector.  The spans of both tails are computed once
// when the table is built, by the same binary32 code (ara_table_span) the builder used, so the
// evaluation and the builder agree on the piece boundaries exactly.
struct TableRec {
  float mx;          // loss scale (the mean itself for a sd = 0 record)
  float p0;          // I_{x0}(a,b); negative marks a sd = 0 record
  float tlo[2];      // table start in t of the lower and the upper tail
  float ih[2];       // inverse piece widths of the two tails
  const float4* iv;  // 2 * kTableIntervals pieces (lower then upper), 2 float4 each; NULL: no table
};
static_assert(sizeof(TableRec) == 32, "a table header is one 32-byte sector");

// Start of a tail's table in t and its inverse piece width, from the tail's mean probability
// pe (p0 for the lower tail, 1 - p0 for the upper).
ARA_HD void ara_table_span(float pe, float* tlo, float* invh) {
  *tlo = sqrtf(-2.0f * logf(pe));
  *invh = (float)kTableIntervals / (kTableTHi - *tlo);
}

ARA_HD float ara_exp2_fast(float r) {
#ifdef __CUDA_ARCH__
  float v;
  asm("ex2.approx.ftz.f32 %0, %1;" : "=f"(v) : "f"(r));  // relative error about 2^-22
  return v;
#else
  return exp2f(r);
#endif
}

// Quantile from a certified table (iv != NULL, p0 >= 0).  Pieces hold log2 x as quintics in
// tau, the position inside the piece.  KEEP chooses the piece load's L2 policy: evict-last when
// the pieces are reused while they are cached (band-major schedule), evict-first when the tables
// are swept at random and a piece is rarely met twice before eviction (trial-major schedule).
template <bool KEEP = false>
ARA_HD float ara_table_quantile(const TableRec& tr, float u) {
  const bool lower = u <= tr.p0;
  const float q = lower ? u : 1.0f - u;  // exact on the uniform grid
  const float t = sqrtf(-2.0f * logf(q));
  const float tlo = lower ? tr.tlo[0] : tr.tlo[1];
  const float ih = lower ? tr.ih[0] : tr.ih[1];
  float pos = fminf(fmaxf((t - tlo) * ih, 0.0f), (float)kTableIntervals);
  const int k = pos < (float)(kTableIntervals - 1) ? (int)pos : kTableIntervals - 1;
  const float tau = pos - (float)k;
  const float4* c = tr.iv + 2 * ((lower ? 0 : kTableIntervals) + k);
#ifdef __CUDA_ARCH__
  // one 32-byte load, streamed: bypasses L1 and is first in line for eviction from L2
  float4 c0, c1;
  if constexpr (KEEP) {
    asm volatile(
        "ld.global.nc.L1::no_allocate.L2::evict_last.v8.f32 {%0,%1,%2,%3,%4,%5,%6,%7}, [%8];"
        : "=f"(c0.x), "=f"(c0.y), "=f"(c0.z), "=f"(c0.w), "=f"(c1.x), "=f"(c1.y), "=f"(c1.z),
          "=f"(c1.w)
        : "l"(c));
  } else {
    asm volatile(
        "ld.global.nc.L1::no_allocate.L2::evict_first.v8.f32 {%0,%1,%2,%3,%4,%5,%6,%7}, [%8];"
        : "=f"(c0.x), "=f"(c0.y), "=f"(c0.z), "=f"(c0.w), "=f"(c1.x), "=f"(c1.y), "=f"(c1.z),
          "=f"(c1.w)
        : "l"(c));
  }
#else
  const float4 c0 = c[0];
  const float4 c1 = c[1];
#endif
  const float r2 = fmaf(tau, fmaf(tau, fmaf(tau, fmaf(tau, fmaf(tau, c1.y, c1.x), c0.w), c0.z),
                                  c0.y),
                        c0.x);
  const float v = ara_exp2_fast(r2);
  return lower ? v : 1.0f - v;
}

}  // namespace ara
