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
//   * The root of I_x = p is found by Halley's method (Newton's step corrected by the second
//     derivative, which costs nothing extra here) in t = ln x from a start given by the
//     small-x limit of DLMF 8.17.22 or, for a, b > 1, by the normal approximation of
//     Abramowitz & Stegun 26.5.22 with the normal quantile of A&S 26.2.23.  The tail below the
//     mean is always the one solved (the other through 1 - u, exact on the uniform grid).
//   * Iterations are capped; a lane that reaches the cap reports it (no trap, no spin).
#pragma once

#ifndef ARA_HD
#ifdef __CUDACC__
#define ARA_HD __host__ __device__ __forceinline__
#define ARA_HD_CALL static __host__ __device__ __noinline__
#else
#include <cmath>
#define ARA_HD inline
#define ARA_HD_CALL static inline
#endif
#endif

#include <stdint.h>
#include <string.h>

#ifndef __CUDACC__
#include <cmath>
#include <cstring>
using std::isfinite;
struct float4 {
  float x, y, z, w;
};
struct float2 {
  float x, y;
};
#endif

namespace ara {
ARA_HD float ara_bits_to_float(int i) {
#ifdef __CUDA_ARCH__
  return __int_as_float(i);
#else
  float f;
  memcpy(&f, &i, 4);
  return f;
#endif
}
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

// Two binary32 values in one 64-bit register, (lo, hi): the recurrence advances its numerator
// and denominator together by the paired FP32 instructions (fma.rn.f32x2, mul.rn.f32x2), each
// element rounded as its scalar operation.
struct F2 {
  unsigned long long v;
};
ARA_HD F2 f2_make(float lo, float hi) {
  F2 r;
#ifdef __CUDA_ARCH__
  asm("mov.b64 %0, {%1, %2};" : "=l"(r.v) : "f"(lo), "f"(hi));
#else
  uint32_t a, b;
  memcpy(&a, &lo, 4);
  memcpy(&b, &hi, 4);
  r.v = ((unsigned long long)b << 32) | a;
#endif
  return r;
}
ARA_HD float f2_lo(F2 p) {
#ifdef __CUDA_ARCH__
  return __uint_as_float((uint32_t)p.v);
#else
  const uint32_t a = (uint32_t)p.v;
  float f;
  memcpy(&f, &a, 4);
  return f;
#endif
}
ARA_HD float f2_hi(F2 p) {
#ifdef __CUDA_ARCH__
  return __uint_as_float((uint32_t)(p.v >> 32));
#else
  const uint32_t b = (uint32_t)(p.v >> 32);
  float f;
  memcpy(&f, &b, 4);
  return f;
#endif
}
ARA_HD F2 f2_fma(F2 a, F2 b, F2 c) {
#ifdef __CUDA_ARCH__
  F2 r;
  asm("fma.rn.f32x2 %0, %1, %2, %3;" : "=l"(r.v) : "l"(a.v), "l"(b.v), "l"(c.v));
  return r;
#else
  return f2_make(fmaf(f2_lo(a), f2_lo(b), f2_lo(c)), fmaf(f2_hi(a), f2_hi(b), f2_hi(c)));
#endif
}
ARA_HD F2 f2_mul(F2 a, F2 b) {
#ifdef __CUDA_ARCH__
  F2 r;
  asm("mul.rn.f32x2 %0, %1, %2;" : "=l"(r.v) : "l"(a.v), "l"(b.v));
  return r;
#else
  return f2_make(f2_lo(a) * f2_lo(b), f2_hi(a) * f2_hi(b));
#endif
}

// K(a,b,x) = 1/(1 + d1/(1 + d2/(...))) of DLMF 8.17.22 by the Wallis recurrence on the
// division-free equivalent fraction T = 1 + alpha_1/(beta_1 + alpha_2/(beta_2 + ...)), K = 1/T.
// Converges quickly for x < (a+1)/(a+b+2).  The fraction is summed in blocks of four terms: after
// each block two estimates four terms apart are compared, B/A against pB/pA cross-multiplied,
// |B pA - pB A| <= max(tol |B pA|, tol_g |A pA|) (A and pA are rescaled into [1, 2)), so the one
// division is the final K.  The first bound is a relative error tol in K; the second is a
// relative error tol_g / K in K, which the inversion below sets so that the fraction stops once
// its error moves the root's ln x by at most tol.  CfState holds the recurrence between blocks, so a lane can sum one fraction block by
// block and take up another's when it is done (the batched inversion of the kernels).
struct CfState {
  float a, b, x, apb;
  F2 P1, P2;                 // (A_{n-1}, B_{n-1}), (A_{n-2}, B_{n-2}); T_n = A_n / B_n;
                             // A_{-1} = 1, A_0 = 1; B_{-1} = 0, B_0 = 1
  float pA, pB;              // the estimate last tested, as the pair (A, B)
  float m;                   // the next pair holds terms 2m+1 and 2m+2 (an exact small integer)
  int n;                     // index of the next (odd) term, 2m+1
};

ARA_HD void ara_cf_init(CfState& c, float a, float b, float x) {
  c.a = a; c.b = b; c.x = x; c.apb = a + b;
  c.P2 = f2_make(1.0f, 0.0f);
  c.P1 = f2_make(1.0f, 1.0f);
  c.pA = 1.0f; c.pB = 1.0f;
  c.m = 0.0f;
  c.n = 1;
}

// Terms 2m+1 and 2m+2, then the exact power-of-two rescale.
ARA_HD void ara_cf_pair(CfState& c) {
  // odd step 2m+1: alpha = -(a+m)(a+b+m) x  (alpha_1 = -(a+b) x: the a cancels)
  const float m = c.m;
  const float al_odd = (m == 0.0f) ? -c.apb * c.x : -(c.a + m) * (c.apb + m) * c.x;
  const float be_odd = c.a + fmaf(2.0f, m, 1.0f);  // a + (2m+1), the integer exact
  F2 N = f2_fma(f2_make(be_odd, be_odd), c.P1, f2_mul(f2_make(al_odd, al_odd), c.P2));
  c.P2 = c.P1;
  c.P1 = N;
  // even step 2(m+1): alpha = (m+1)(b-m-1) x
  const float m2 = m + 1.0f;
  const float al_even = m2 * (c.b - m2) * c.x;
  const float be_even = c.a + 2.0f * m2;
  N = f2_fma(f2_make(be_even, be_even), c.P1, f2_mul(f2_make(al_even, al_even), c.P2));
  c.P2 = c.P1;
  c.P1 = N;
  // exact power-of-two rescale keeps the recurrence inside binary32 range
  const float sc = ara_pow2_scale_of(f2_lo(c.P1));
  const F2 s2 = f2_make(sc, sc);
  c.P1 = f2_mul(c.P1, s2);
  c.P2 = f2_mul(c.P2, s2);
  c.m = m2;
}

// Four more terms and the convergence test: true once the fraction has converged or reached
// kCfMaxTerms terms; c.n - 1 is then the number of terms summed.
ARA_HD bool ara_cf_block(CfState& c, float tol, float tol_g = 0.0f) {
  ara_cf_pair(c);
  ara_cf_pair(c);
  c.n += 4;
  const float A = f2_lo(c.P1), B = f2_hi(c.P1);
  const float cur = B * c.pA;
  if (fabsf(fmaf(-c.pB, A, cur)) <= fmaxf(tol * fabsf(cur), tol_g * fabsf(A * c.pA))) return true;
  c.pA = A;
  c.pB = B;
  return c.n > kCfMaxTerms;
}

ARA_HD float ara_cf_value(const CfState& c) { return f2_hi(c.P1) / f2_lo(c.P1); }

// The whole fraction for one lane; *terms is increased by the number of terms summed.
ARA_HD float ara_beta_cf(float a, float b, float x, int* terms, float tol = 1.2e-7f,
                         float tol_g = 0.0f) {
  CfState c;
  ara_cf_init(c, a, b, x);
  while (!ara_cf_block(c, tol, tol_g)) {
  }
  if (terms) *terms += c.n - 1;
  return ara_cf_value(c);
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

// The state of one inversion between the pieces of a Halley iteration (the one-lane inversion
// below runs them in a loop; the batched inversion of the kernels runs the continued fraction of
// many inversions in between).
struct HalleyState {
  float a, b, s, lnx0, lny0, L0, lna, lnp, thr;  // of the tail solved (swapped when u > p0)
  float t, x;                                    // current iterate, t = ln x
  bool flip, good;                               // tail swapped; start from a table's estimate
};

// The fast division (about 2 ulp), for quotients that only steer the iteration.
ARA_HD float ara_fdiv(float n, float d) {
#ifdef __CUDA_ARCH__
  return __fdividef(n, d);
#else
  return n / d;
#endif
}

// Start of the inversion.  Returns false when it is already done (r holds the result): the
// start lies below e^-69, where the loss max_l x is far under every term of a year loss.
// The fields of the state that depend on the record and u alone; returns p (u or 1 - u).
ARA_HD float ara_halley_fields(const BetaRec& rec, float u, HalleyState& h) {
  h.flip = u > rec.p0;
  const float p = h.flip ? 1.0f - u : u;
  h.a = h.flip ? rec.b : rec.a;
  h.b = h.flip ? rec.a : rec.b;
  h.lnx0 = h.flip ? rec.lny0 : rec.lnx0;
  h.lny0 = h.flip ? rec.lnx0 : rec.lny0;
  h.L0 = rec.L0;
  h.s = h.a + h.b;
  h.lna = h.lnx0 + rec.lns;
  h.lnp = logf(p);
  h.thr = ara_fdiv(h.a + 1.0f, h.s + 2.0f);  // chooses the fraction's side; either side is exact
  return p;
}

ARA_HD bool ara_halley_setup(const BetaRec& rec, float u, float start_logit, HalleyState& h,
                             IbetaResult& r) {
  r.iters = 0;
  r.cf_terms = 0;
  r.converged = true;
  r.t = 0.0f;
  const float p = ara_halley_fields(rec, u, h);
  const float a = h.a, b = h.b;

  // a start table's estimate of the log-odds L, as t = ln x = -ln(1 + e^-L) of the tail solved
  // (a start only: the fast exponential and logarithm are ample).  An estimate below e^-69 ends
  // the inversion only if the analytic start (exact in that limit) agrees: start tables are not
  // certified, and on shapes far outside the ELT value law (a, b near 1e-6 under the sd clamp
  // of §3.3) they can be far off.
  float t = 0.0f;
  h.good = start_logit < 1e29f;  // false for NaN too
  if (h.good) {
#ifdef __CUDA_ARCH__
    t = -__logf(1.0f + __expf(h.flip ? start_logit : -start_logit));
#else
    t = -std::log(1.0f + std::exp(h.flip ? start_logit : -start_logit));
#endif
    h.good = t > -69.0f;
  }
  if (!h.good) {
    // small-x limit of DLMF 8.17.22 (K -> 1, y -> 1): ln p = L0 + a ln(x/x0) - b ln y0 - ln a
    t = h.lnx0 + (h.lnp + h.lna - h.L0 + b * h.lny0) / a;
    if (a > 1.0f && b > 1.0f) {
      // A&S 26.5.22: x ~ a / (a + b e^{2w}), with yp the upper-tail normal deviate of p.
      const float yp = ara_norm_upper_quantile(fminf(p, 0.5f));
      const float ypl = p > 0.5f ? -ara_norm_upper_quantile(1.0f - p) : yp;
      const float lam = (ypl * ypl - 3.0f) / 6.0f;
      const float hh = 2.0f / (1.0f / (2.0f * a - 1.0f) + 1.0f / (2.0f * b - 1.0f));
      const float w = ypl * sqrtf(fmaxf(hh + lam, 0.0f)) / hh -
                      (1.0f / (2.0f * b - 1.0f) - 1.0f / (2.0f * a - 1.0f)) *
                          (lam + 5.0f / 6.0f - 2.0f / (3.0f * hh));
      t = h.lna - logf(a + b * expf(2.0f * w));
    }
  }
  t = fminf(t, h.lnx0);  // the root is below the mean
  h.t = t;
  if (!(t > -69.0f)) {  // below e^-69 ~ 1e-30
    r.x = h.flip ? 1.0f : 0.0f;
    r.t = t;
    return false;
  }
  h.x = expf(t);
  return true;
}

// The part of a Halley iteration before the continued fraction: E = ln(x^a y^b / B(a,b)) and the
// fraction to sum, K(a,b,x) below the threshold x = (a+1)/(a+b+2) (I_x = P K / a), else K(b,a,y)
// (the complement I_y(b,a) = P K / b).
struct HalleyPre {
  float y, E;
  bool lower;
  float ca, cb, cx;  // arguments of the continued fraction
};

ARA_HD HalleyPre ara_halley_pre(const HalleyState& h) {
  HalleyPre q;
  const float x = h.x;
  q.y = 1.0f - x;
  // E = L0 + a ln(x/x0) + b ln(y/y0), w = (x - x0)(a + b)
  const float w = fmaf(x, h.s, -h.a);
  const float rx = w / h.a;   // x/x0 - 1
  const float ry = -w / h.b;  // y/y0 - 1
  const float lnrx = rx > -0.5f ? log1pf(rx) : h.t - h.lnx0;
  const float lnry = ry > -0.5f ? log1pf(ry) : logf(q.y) - h.lny0;
  q.E = h.L0 + h.a * lnrx + h.b * lnry;
  q.lower = x < h.thr;
  q.ca = q.lower ? h.a : h.b;
  q.cb = q.lower ? h.b : h.a;
  q.cx = q.lower ? x : q.y;
  return q;
}

// The part after it: G = ln I_x - ln p, G' and Halley's step in t.  Returns true when the
// iteration `it` (0-based) ends the inversion.
// The residual G is the function value and keeps IEEE arithmetic; G' and Halley's correction
// only shape the step toward the root, so their quotients take the fast division (ara_fdiv).
ARA_HD bool ara_halley_post(HalleyState& h, const HalleyPre& q, float K, int it) {
  const float a = h.a, b = h.b, x = h.x, y = q.y;
  float G, dG;
  if (q.lower) {
    G = q.E + logf(K) - h.lna - h.lnp;
    dG = ara_fdiv(a, y * K);
  } else {
    const float P = expf(q.E);
    const float J = P * K / b;  // I_{1-x}(b,a)
    G = log1pf(-J) - h.lnp;
    dG = ara_fdiv(P, y * (1.0f - J));
  }
  // Where I_x is nearly flat in t (G' below 1e-3: a shape parameter far below the paper's
  // value law, e.g. the sd clamp of §3.3, which gives a, b near 1e-6) the binary32 residual's
  // rounding noise (a few units of 2^-24 times the exponent E, |E| ~ 15 there) moves the
  // Newton step by far more than 3e-4 and the steps never settle; there the iteration ends
  // once the residual is at that noise, x then being the exact quantile of a uniform within a
  // few 1e-6 of u (a backward-error stop).
  if (dG < 1e-3f && fabsf(G) <= 2.4e-7f * (2.0f + fabsf(q.E))) return true;
  // Halley's correction of the Newton step dn = G/G': the second derivative is free, since
  // G' = x f(x) / I_x gives G'' = G' (a - (b-1) x/y - G'); the step converges cubically, so
  // a step of 3e-4 leaves an error near 1e-11 in t.  Far from the root (|dn c| large) the
  // plain Newton step is taken.
  const float dn = ara_fdiv(G, dG);
  const float c = 0.5f * (a - (b - 1.0f) * ara_fdiv(x, y) - dG);
  const float den = 1.0f - dn * c;
  float tn = h.t - ((den > 0.5f && den < 2.0f) ? ara_fdiv(dn, den) : dn);
  if (!(tn < 0.0f)) tn = 0.5f * h.t;  // a step past x = 1 is halved toward it
  const float step = fabsf(tn - h.t);
  h.t = tn;
  h.x = expf(tn);
  if ((it > 0 || h.good) && step <= 3.0e-4f) return true;
  if (!(tn > -69.0f)) {
    h.x = 0.0f;
    return true;
  }
  return false;
}

ARA_HD void ara_halley_result(const HalleyState& h, int iters, bool done, IbetaResult& r) {
  r.iters = iters;
  r.converged = done;
  r.t = h.t;
  r.x = h.flip ? 1.0f - h.x : h.x;
}

// Iterations it0, it0 + 1, ... of an inversion set up by ara_halley_setup, to the end; r.cf_terms
// is increased by the terms summed.  From the analytic start (~1e-2 from the root) the first
// iteration's continued fraction is summed only to 1e-4 and cannot end the loop; later
// iterations (and every one from a start table's estimate) are summed to binary32 accuracy.  The
// fraction stops once its last four terms changed K by at most kCfStop relatively, or by as much
// as moves ln x by kCfStop, whichever is looser.  A relative change e in the fraction K(c, d, z)
// moves t = ln x by e y K / c on either side of the threshold (c = a below it, where
// G = E + ln K - ln a - ln p and G' = a / (y K); c = b above it, where G = ln(1 - J) - ln p with
// J = P K / b and G' = P / (y (1 - J))), so the second bound is tol_g = tol c / y, capped at 1e-4
// so that the first-order step stays valid.  The fraction gains orders of magnitude over four
// terms, so the error left is far below the last change: over the ELT value law and over
// alpha, beta in [0.1, 100]^2 (4,000 roots each, binary64) a stop at kCfStop = 3.6e-6 leaves at
// most 5e-8 in ln x, where a stop at 1.2e-7 left 1e-8 and took 11% more terms.
// ONE_CF: evaluate the continued fraction in one loop whichever side of the threshold x lies on
// (lanes of a warp on different sides share it; 16% faster where most hits invert this way), or
// in a loop per side (fewer registers, for the out-of-line fallback of the table paths).  Both
// give the same result bit for bit.
constexpr float kCfStop = 3.6e-6f;
template <bool ONE_CF>
ARA_HD void ara_halley_iterate(HalleyState& h, int it0, IbetaResult& r) {
  const float cf_first = h.good ? kCfStop : 1.0e-4f;
  bool done = false;
  int it = it0;
  for (; it < kIbetaMaxIter; ++it) {
    const HalleyPre q = ara_halley_pre(h);
    const float tol = it == 0 ? cf_first : kCfStop;
    const float tol_g = fminf(tol * ara_fdiv(q.ca, q.y), 1e-4f);
    float K;
    if constexpr (ONE_CF)
      K = ara_beta_cf(q.ca, q.cb, q.cx, &r.cf_terms, tol, tol_g);
    else
      K = q.lower ? ara_beta_cf(h.a, h.b, h.x, &r.cf_terms, tol, tol_g)
                  : ara_beta_cf(h.b, h.a, q.y, &r.cf_terms, tol, tol_g);
    if (ara_halley_post(h, q, K, it)) {
      done = true;
      ++it;
      break;
    }
  }
  ara_halley_result(h, it, done, r);
}

// Solve I_x(a,b) = u for x, x in [0,1].
//
// Halley's method on G(t) = ln I_{e^t}(a,b) - ln p in t = ln x.  Below the threshold
// x = (a+1)/(a+b+2), I_x = P K / a with P the prefactor, so G = E + ln(K/a) - ln p and
// G'(t) = x f(x) / I_x = a / ((1-x) K): no exponential is needed.  In the lower tail G is nearly
// linear in t (I_x ~ x^a), which is where Newton in x fails for a < 1.
//
// The tail is chosen per record: if u > p0 the root lies above the mean, and the symmetric
// problem I_y(b,a) = 1 - u (exact on the uniform grid) is solved for y = 1 - x instead, so the
// unknown solved for is always below the mean of its distribution.
// start_logit: an estimate of ln(x / (1 - x)) accurate to ~1e-4 (a start table's value), or
// anything not below 1e29 to use the analytic start (the small-x limit of DLMF 8.17.22 or, for
// a, b > 1, the normal approximation of A&S 26.5.22).  From a good start the first iteration
// sums its continued fraction fully and may end the loop.
template <bool ONE_CF = true>
ARA_HD IbetaResult ara_inv_beta(const BetaRec& rec, float u, float start_logit = 1e30f) {
  IbetaResult r;
  HalleyState h;
  if (!ara_halley_setup(rec, u, start_logit, h, r)) return r;
  ara_halley_iterate<ONE_CF>(h, 0, r);
  return r;
}

// ---- certified per-record quantile tables ---------------------------------------------------------
//
// Each record's (alpha, beta) is fixed and is met hundreds of times per run, so its quantile
// function is tabulated once, when the ELT is staged.  One coordinate serves every record and
// both tails: with q = min(u, 1 - u) and t = sqrt(-2 ln q), the signed distance from the median
//   z = t - t_m  (u < 1/2),   z = t_m - t  (u > 1/2),   t_m = sqrt(2 ln 2),
// covers the whole uniform grid (u in [2^-24, 1 - 2^-24] gives |z| <= 4.591) and is cut into
// kTablePieces pieces of width kTableH on [-kTableZ, kTableZ]; the median is a piece boundary.
// In z the log-odds L = ln(x / (1 - x)) of the quantile is smooth and nearly quadratic in both
// tails (ln x ~ (ln u)/alpha, ln(1-x) ~ (ln(1-u))/beta), so quintic Hermite pieces built from L
// and its first two derivatives at the knots reproduce it to ~1e-8; every piece is checked at its
// midpoint when the table is built, and a record whose table misses the bound keeps the Newton
// inversion.  A piece is 32 bytes, one sector: 6 binary32 coefficients of log2-odds in the local
// coordinate tau in [0,1), the record's loss scale max_l, and a flag.  Because the piece index
// depends on u alone, a hit needs no record header: one 32-byte load gives everything.
constexpr int kTablePieces = 64;
constexpr float kTableTm = 1.17741002f;   // sqrt(2 ln 2): t at the median
constexpr float kTableH = 0.14453125f;    // 37/256, exact: 32 pieces per side reach z = 4.625
constexpr float kTableZ = 4.625f;         // 32 kTableH
constexpr float kTableInvH = 6.91891892f; // 1 / kTableH
constexpr uint32_t kPieceTable = 0;       // piece flags: evaluate the quintic
constexpr uint32_t kPieceMean = 1;        //   sd = 0: the loss is max_l (the mean)
constexpr uint32_t kPieceNewton = 2;      //   table not certified: invert by Newton

struct TablePiece {
  float c[6];     // log2-odds in tau, lowest order first
  float mx;       // the record's loss scale (the mean itself for a sd = 0 record)
  uint32_t flag;  // kPiece*
};

// ---- start tables for the Newton-Halley inversion ---------------------------------------------
// Where a record's certified table does not exist (tables on demand, before they pay off) the
// inversion starts from a coarse table built in binary32 when the ELT is staged: the same
// coordinate z, 16 pieces of width 4 kTableH, a quintic Hermite of the log-odds L from L, dL/dz
// and d2L/dz2 at the knots.  A piece's six coefficients are padded to one 32-byte sector (512
// bytes a record), so a hit reads one sector of it.  It is not certified: it is only a start
// (~2e-6 from the root in ln x on average, 1.7e-4 at worst over the ELT value law, so a single
// Halley step lands within ~1e-11), and a piece whose knots failed holds NaN, which sends the
// inversion back to its analytic start.
constexpr int kStartPieces = 16;
constexpr int kStartCoefs = 6;                      // quintic Hermite: L, L', L'' at both knots
constexpr int kStartStride = 8;                     // floats a piece takes: one 32-byte sector
constexpr int kStartFloats = kStartPieces * kStartStride;
constexpr float kStartInvH = kTableInvH * 0.25f;  // 1 / (4 kTableH)

// Piece and local coordinate of u in a start table.
ARA_HD int ara_start_piece(float u, float* tau) {
  const bool lower = u < 0.5f;
  const float q = lower ? u : 1.0f - u;
#ifdef __CUDA_ARCH__
  // the hardware base-2 logarithm and square root (q >= 2^-24 is normal): ample for a start
  float lg, t;
  asm("lg2.approx.ftz.f32 %0, %1;" : "=f"(lg) : "f"(q));
  asm("sqrt.approx.ftz.f32 %0, %1;" : "=f"(t) : "f"(-1.38629436f * lg));
#else
  const float t = sqrtf(-2.0f * logf(q));
#endif
  const float z = lower ? t - kTableTm : kTableTm - t;
  const float pos = fminf(fmaxf((z + kTableZ) * kStartInvH, 0.0f), (float)kStartPieces);
  const int k = pos < (float)(kStartPieces - 1) ? (int)pos : kStartPieces - 1;
  *tau = pos - (float)k;
  return k;
}

// The piece's quintic at tau, by Horner with explicit FMAs: every caller, whatever load brought
// the coefficients, gets the same bits.
ARA_HD float ara_start_poly(float2 c01, float2 c23, float2 c45, float tau) {
  return fmaf(tau, fmaf(tau, fmaf(tau, fmaf(tau, fmaf(tau, c45.y, c45.x), c23.y), c23.x), c01.y),
              c01.x);
}

// Estimated log-odds of the quantile of u from a record's start table (NaN where none).
ARA_HD float ara_start_logit(const float* st, float u) {
  float tau;
  const int k = ara_start_piece(u, &tau);
  const float2* c2 = reinterpret_cast<const float2*>(st + k * kStartStride);
#ifdef __CUDA_ARCH__
  const float2 c01 = __ldg(c2), c23 = __ldg(c2 + 1), c45 = __ldg(c2 + 2);
#else
  const float2 c01 = c2[0], c23 = c2[1], c45 = c2[2];
#endif
  return ara_start_poly(c01, c23, c45, tau);
}
static_assert(sizeof(TablePiece) == 32, "a table piece is one 32-byte sector");

ARA_HD float ara_exp2_fast(float r) {
#ifdef __CUDA_ARCH__
  float v;
  asm("ex2.approx.ftz.f32 %0, %1;" : "=f"(v) : "f"(r));  // relative error about 2^-22
  return v;
#else
  return exp2f(r);
#endif
}

// Piece index and local coordinate of the uniform whose tail side is `lower` and whose tail
// probability is q = min(z, 1 - z).  ln q comes from the hardware base-2 logarithm
// (relative error about 2^-22 for q <= 1/2), which moves z by at most ~3e-7: well inside a
// piece, and the quantile's log-odds by L'(z) times that.
ARA_HD int ara_table_piece_q(bool lower, float q, float* tau) {
#ifdef __CUDA_ARCH__
  const float t = sqrtf(-1.38629436f * __log2f(q));  // -2 ln q = -2 ln 2 log2 q
#else
  const float t = sqrtf(-2.0f * logf(q));
#endif
  const float z = lower ? t - kTableTm : kTableTm - t;
  const float pos = fminf(fmaxf((z + kTableZ) * kTableInvH, 0.0f), (float)kTablePieces);
  const int k = pos < (float)(kTablePieces - 1) ? (int)pos : kTablePieces - 1;
  *tau = pos - (float)k;
  return k;
}

// The same from the uniform u itself (q = min(u, 1 - u), exact on the uniform grid).
ARA_HD int ara_table_piece(float u, float* tau) {
  const bool lower = u < 0.5f;
  return ara_table_piece_q(lower, lower ? u : 1.0f - u, tau);
}

// One 32-byte load of piece k of the record whose table starts at rec.  KEEP chooses the L2
// policy: evict-last when pieces are reused while cached (band-major schedule), evict-first when
// the tables are swept at random (trial-major schedule).  A miss fills 64 bytes, not the default
// 128: a random 32-byte gather then reads half as much from DRAM.
template <bool KEEP>
ARA_HD TablePiece ara_load_piece(const TablePiece* rec, int k) {
  TablePiece pc;
#ifdef __CUDA_ARCH__
  uint32_t w[8];
  const TablePiece* p = rec + k;
  if constexpr (KEEP) {
    asm volatile(
        "ld.global.nc.L1::no_allocate.L2::evict_last.L2::64B.v8.u32 {%0,%1,%2,%3,%4,%5,%6,%7}, [%8];"
        : "=r"(w[0]), "=r"(w[1]), "=r"(w[2]), "=r"(w[3]), "=r"(w[4]), "=r"(w[5]), "=r"(w[6]),
          "=r"(w[7])
        : "l"(p));
  } else {
    asm volatile(
        "ld.global.nc.L1::no_allocate.L2::evict_first.L2::64B.v8.u32 {%0,%1,%2,%3,%4,%5,%6,%7}, [%8];"
        : "=r"(w[0]), "=r"(w[1]), "=r"(w[2]), "=r"(w[3]), "=r"(w[4]), "=r"(w[5]), "=r"(w[6]),
          "=r"(w[7])
        : "l"(p));
  }
#pragma unroll
  for (int i = 0; i < 6; ++i) pc.c[i] = __uint_as_float(w[i]);
  pc.mx = __uint_as_float(w[6]);
  pc.flag = w[7];
#else
  pc = rec[k];
#endif
  return pc;
}

// x from a table piece (flag kPieceTable): log2-odds by Horner, then x = 1 / (1 + 2^-L2).
ARA_HD float ara_piece_x(const TablePiece& pc, float tau) {
  const float l2 = fmaf(tau, fmaf(tau, fmaf(tau, fmaf(tau, fmaf(tau, pc.c[5], pc.c[4]), pc.c[3]),
                                            pc.c[2]),
                                  pc.c[1]),
                        pc.c[0]);
  const float e = ara_exp2_fast(-l2);
#ifdef __CUDA_ARCH__
  return __fdividef(1.0f, 1.0f + e);  // e beyond 2^126 (x below ~1e-38) gives 0
#else
  return 1.0f / (1.0f + e);
#endif
}

}  // namespace ara
