// ara_table.cuh -- construction of the certified per-record quantile tables (host and device).
//
// Knots are placed at z_i = -kTableZ + i kTableH (i = 0..kTablePieces), z the signed distance
// from the median in t = sqrt(-2 ln q), q = min(u, 1 - u).  The quantile at a knot comes from
// the binary32 Newton-Halley inversion on the record's own tail (u <= p0: x itself; u > p0: 1 - x
// of the swapped record, so x near 1 keeps its precision), started from the Taylor step of the
// knot before it; the log-odds L = ln x - ln(1-x) and its first two derivatives in z follow from
// the beta density; each piece's quintic Hermite coefficients are stored as log2-odds.  Each
// piece is then checked at its midpoint against the same inversion started from the piece
// itself; a record keeps its table only if every midpoint agrees to kTableTol in L (so in
// x/(1-x) relatively) plus the binary32 rounding of L and the inversion's own rounding.  A table
// is thus the binary32 Newton-Halley inversion, tabulated: its error against the exact quantile
// is that inversion's (mean 2.3e-7 relative in x over the ELT value law) plus at most kTableTol.
//
// Derivatives (g = dL/du = B(a,b) / (x^a (1-x)^b), t = t_m + |z|, u(z) with du/dz = -t q):
//   L'  = -t q g,
//   L'' = L'^2 (b x - a (1 - x)) - s (t^2 - 1) L' / t,   s = +1 for z > 0, -1 for z < 0;
// L'' jumps at the median (z = 0), which is a piece boundary: each side uses its own value.
#pragma once

#include "ara_ibeta.cuh"

namespace ara {

constexpr double kTableTol = 1e-6;
// The binary32 check's allowance for its reference's own rounding: the inversion's residual
// ln I - ln p carries up to kTableNoiseUlps units of 2^-24 of the magnitude of its terms (the
// prefactor's L0, a ln(x/x0), b ln(y/y0), ln p, the fraction), which moves its L by that times
// dL/d(ln p) = |L'| / t (about 1/a in a lower tail: the binary32 inversion of a record with a
// shape parameter near 0.1 is itself only good to ~1e-5 there).  Capped at kTableNoiseCap: a
// record whose inversion is worse conditioned still keeps the Newton inversion.
constexpr float kTableNoiseUlps = 16.0f;
constexpr float kTableNoiseCap = 1e-5f;

// ---- quantiles polished in binary64 (staging constants, the learned surrogate's targets) --------
// A value hi + lo of two binary32 numbers (|lo| <= ulp(hi)/2, ~48 significant bits): the FP64 pipe
// of this part is 1/64 of the FP32 one, so the polish's continued fraction runs in pairs of
// binary32 (Dekker's and Knuth's error-free sum and product, the product through an FMA).  The
// additions and products are the round-to-nearest intrinsics on the device, so that the compiler
// never fuses them into FMAs, which would break the error-free transformations.
struct DF {
  float hi, lo;
};
#ifdef __CUDA_ARCH__
ARA_HD float df_add_rn(float a, float b) { return __fadd_rn(a, b); }
ARA_HD float df_sub_rn(float a, float b) { return __fsub_rn(a, b); }
ARA_HD float df_mul_rn(float a, float b) { return __fmul_rn(a, b); }
#else
ARA_HD float df_add_rn(float a, float b) { return a + b; }
ARA_HD float df_sub_rn(float a, float b) { return a - b; }
ARA_HD float df_mul_rn(float a, float b) { return a * b; }
#endif
ARA_HD DF df_from(double d) {
  DF r;
  r.hi = (float)d;
  r.lo = (float)(d - (double)r.hi);
  return r;
}
ARA_HD double df_to(DF a) { return (double)a.hi + (double)a.lo; }
// s + e with |s| >= |e| (or s = 0), renormalised
ARA_HD DF df_quick(float s, float e) {
  DF r;
  r.hi = df_add_rn(s, e);
  r.lo = df_sub_rn(e, df_sub_rn(r.hi, s));
  return r;
}
ARA_HD DF df_add(DF a, DF b) {
  const float s = df_add_rn(a.hi, b.hi);
  const float bb = df_sub_rn(s, a.hi);
  float e = df_add_rn(df_sub_rn(a.hi, df_sub_rn(s, bb)), df_sub_rn(b.hi, bb));
  e = df_add_rn(e, df_add_rn(a.lo, b.lo));
  return df_quick(s, e);
}
ARA_HD DF df_add_f(DF a, float b) {
  const float s = df_add_rn(a.hi, b);
  const float bb = df_sub_rn(s, a.hi);
  float e = df_add_rn(df_sub_rn(a.hi, df_sub_rn(s, bb)), df_sub_rn(b, bb));
  e = df_add_rn(e, a.lo);
  return df_quick(s, e);
}
ARA_HD DF df_neg(DF a) {
  a.hi = -a.hi;
  a.lo = -a.lo;
  return a;
}
ARA_HD DF df_mul(DF a, DF b) {
  const float p = df_mul_rn(a.hi, b.hi);
  float e = fmaf(a.hi, b.hi, -p);
  e = fmaf(a.hi, b.lo, e);
  e = fmaf(a.lo, b.hi, e);
  return df_quick(p, e);
}
ARA_HD DF df_mul_f(DF a, float b) {
  const float p = df_mul_rn(a.hi, b);
  float e = fmaf(a.hi, b, -p);
  e = fmaf(a.lo, b, e);
  return df_quick(p, e);
}
ARA_HD DF df_scale(DF a, float s) {  // s a power of two: exact
  a.hi *= s;
  a.lo *= s;
  return a;
}

// K = 1/(1 + d1/(1 + ...)) of DLMF 8.17.22 in double-float by the Wallis recurrence of the
// division-free equivalent fraction (numerators -(a+b)x, -(a+m)(a+b+m)x, m(b-m)x; denominators
// a+n), rescaled by a power of two every step pair.  Converged when B/A moved by at most 1e-10
// relative since the previous pair, tested without a division: |B pA - pB A| <= 1e-10 |B pA|
// (pA, pB: the previous pair at the same scale).
ARA_HD double ara_beta_cf_f64(double a64, double b64, double x64) {
  const DF a = df_from(a64), b = df_from(b64), x = df_from(x64);
  const DF apb = df_add(a, b);
  DF Am2 = {1.0f, 0.0f}, Am1 = {1.0f, 0.0f}, Bm2 = {0.0f, 0.0f}, Bm1 = {1.0f, 0.0f};
  DF pA = Am1, pB = Bm1;
  for (int n = 1; n < 4000; n += 2) {
    const float m = 0.5f * (float)(n - 1);  // exact
    const DF al_odd = (n == 1) ? df_neg(df_mul(apb, x))
                               : df_neg(df_mul(df_mul(df_add_f(a, m), df_add_f(apb, m)), x));
    const DF be_odd = df_add_f(a, (float)n);
    DF A = df_add(df_mul(be_odd, Am1), df_mul(al_odd, Am2));
    DF B = df_add(df_mul(be_odd, Bm1), df_mul(al_odd, Bm2));
    Am2 = Am1; Bm2 = Bm1; Am1 = A; Bm1 = B;
    const float m2 = m + 1.0f;
    const DF al_even = df_mul(df_mul_f(df_add_f(b, -m2), m2), x);
    const DF be_even = df_add_f(a, (float)(n + 1));
    A = df_add(df_mul(be_even, Am1), df_mul(al_even, Am2));
    B = df_add(df_mul(be_even, Bm1), df_mul(al_even, Bm2));
    Am2 = Am1; Bm2 = Bm1; Am1 = A; Bm1 = B;
    const DF lhs = df_mul(Bm1, pA);
    const DF d = df_add(lhs, df_neg(df_mul(pB, Am1)));
    const bool done = fabsf(d.hi) <= 1e-10f * fabsf(lhs.hi);
    // a pair grows A, B by about (a+n)^2: rescale every pair to stay inside binary32's range
    if (Am1.hi != 0.0f && isfinite(Am1.hi)) {
      const float sc = ara_pow2_scale_of(Am1.hi);
      Am1 = df_scale(Am1, sc); Am2 = df_scale(Am2, sc);
      Bm1 = df_scale(Bm1, sc); Bm2 = df_scale(Bm2, sc);
    }
    pA = Am1;
    pB = Bm1;
    if (done) break;
  }
  // K = B / A: a binary32 quotient corrected by the double-float remainder
  const float q1 = Bm1.hi / Am1.hi;
  const DF r = df_add(Bm1, df_neg(df_mul_f(Am1, q1)));
  const float q2 = r.hi / Am1.hi;
  return (double)q1 + (double)q2;
}

// ln I_x(a,b) for x = e^r (DLMF 8.17.22; past (a+1)/(a+b+2) through DLMF 8.17.4); lna = ln a.
ARA_HD double ara_ln_betainc_f64(double a, double b, double r, double lnB, double lna) {
  const double x = exp(r);
  if (x < (a + 1.0) / (a + b + 2.0)) {
    return a * r + b * log1p(-x) - lnB + log(ara_beta_cf_f64(a, b, x)) - lna;
  }
  const double y = 1.0 - x;
  const double Iy = exp(b * log(y) + a * r - lnB) * ara_beta_cf_f64(b, a, y) / b;
  return log1p(-Iy);
}
ARA_HD double ara_ln_betainc_f64(double a, double b, double r, double lnB) {
  return ara_ln_betainc_f64(a, b, r, lnB, log(a));
}

// The tail's beta parameters in binary64 (as computed from mean, sd and max when the ELT was
// staged) and ln B(a,b).
struct TailParams {
  double a, b, lnB;
  double lna;  // ln a (0: compute it)
};

// ln of the quantile of the tail described by br (binary32 record, solved without flipping: u <=
// br.p0) and tp (the same tail in binary64), at the uniform uf with su = ln u known exactly (or
// ln uf): the binary32 Newton inversion gives the start and one binary64 Newton step in r = ln x
// on G(r) = ln I_{e^r}(a,b) - ln u polishes it (G' = x f(x) / I_x).
ARA_HD double ara_polish_ln_quantile(const BetaRec& br, const TailParams& tp, float uf, double su,
                                     bool* ok) {
  const IbetaResult res = ara_inv_beta(br, uf);
  const double a = tp.a, b = tp.b;
  double r = res.t;
  {  // one binary64 Newton step: the binary32 start is within ~1e-7, so the step lands ~1e-14;
     // the slope G' only scales that small step, so binary32 accuracy is enough for it
    const double lnI = ara_ln_betainc_f64(a, b, r, tp.lnB, tp.lna != 0.0 ? tp.lna : log(a));
    const float xf = expf((float)r);
    const double lg = a * r - tp.lnB - lnI + (b - 1.0) * (double)log1pf(-xf);
    const double dG = (double)expf((float)lg);
    const double step = (lnI - su) / dG;
    if (isfinite(step)) r -= step;
  }
  *ok = res.converged && isfinite(r);
  return r;
}

// The binary32 record of Beta(a, b) (for the Newton start) and ln B(a,b), from binary64 a, b.
ARA_HD BetaRec ara_beta_rec_f64(double a, double b, double* lnB_out) {
  const double s = a + b;
  const double lnx0 = log(a / s), lny0 = log(b / s);
  const double lnB = lgamma(a) + lgamma(b) - lgamma(s);
  BetaRec r;
  r.a = (float)a; r.b = (float)b; r.mx = 1.0f;
  r.L0 = (float)(a * lnx0 + b * lny0 - lnB);
  r.p0 = (float)exp(ara_ln_betainc_f64(a, b, lnx0, lnB));
  r.lnx0 = (float)lnx0; r.lny0 = (float)lny0; r.lns = (float)log(s);
  *lnB_out = lnB;
  return r;
}

// ln Gamma(z) for z > 0 in binary64 by one branch-free path (so that the lanes of a warp staging
// records of any shape never diverge): shift to w = z + 8 by Gamma(z) = Gamma(z + 8) / (z (z+1) ...
// (z+7)), then Stirling's series for ln Gamma(w) (DLMF 5.11.1) through the B_12 term, whose
// remainder at w >= 8 is below 1e-14.  Within ~1.3e-14 of max(1, |ln Gamma|) over [1e-7, 2e5].
ARA_HD double ara_lngamma(double z) {
  const double p = (z * (z + 1.0) * (z + 2.0) * (z + 3.0)) * ((z + 4.0) * (z + 5.0) * (z + 6.0) *
                                                              (z + 7.0));
  const double w = z + 8.0, r = 1.0 / w, r2 = r * r;
  const double series =
      r * (1.0 / 12.0 +
           r2 * (-1.0 / 360.0 +
                 r2 * (1.0 / 1260.0 +
                       r2 * (-1.0 / 1680.0 + r2 * (1.0 / 1188.0 + r2 * (-691.0 / 360360.0))))));
  return (w - 0.5) * log(w) - w + 0.91893853320467274178 + series - log(p);  // ln sqrt(2 pi)
}

// The record staged for an ELT: the constants of ara_beta_rec_f64 (ln B by ara_lngamma), except
// p0 = I_{x0}(a,b), which only picks the tail an inversion solves and is taken in binary32: at
// the mean the prefactor is e^{L0} exactly, so p0 = e^{L0} K(a,b,x0) / a (x0 below the fraction's
// threshold when a <= b), else 1 - e^{L0} K(b,a,y0) / b.  Within ~1e-7 of the binary64 value over
// the ELT value law.
ARA_HD BetaRec ara_beta_rec_staged(double a, double b) {
  const double s = a + b;
  const double lnx0 = log(a / s), lny0 = log(b / s);
  const double lnB = ara_lngamma(a) + ara_lngamma(b) - ara_lngamma(s);
  BetaRec r;
  r.a = (float)a; r.b = (float)b; r.mx = 1.0f;
  r.L0 = (float)(a * lnx0 + b * lny0 - lnB);
  r.lnx0 = (float)lnx0; r.lny0 = (float)lny0; r.lns = (float)log(s);
  const float P = expf(r.L0);
  r.p0 = r.a <= r.b ? P * ara_beta_cf(r.a, r.b, expf(r.lnx0), nullptr) / r.a
                    : 1.0f - P * ara_beta_cf(r.b, r.a, expf(r.lny0), nullptr) / r.b;
  return r;
}

// ln x and ln(1 - x) of InvCDF_beta(u; a, b) for binary64 a, b, polished in binary64 (training
// targets and certification references of the learned surrogate).
ARA_HD bool ara_exact_quantile_logs(double a, double b, float u, double* lnx, double* ln1mx) {
  double lnB;
  const BetaRec br = ara_beta_rec_f64(a, b, &lnB);
  bool ok;
  if (u <= br.p0) {
    const TailParams tp = {a, b, lnB};
    *lnx = ara_polish_ln_quantile(br, tp, u, log((double)u), &ok);
    *ln1mx = log1p(-exp(*lnx));
  } else {
    BetaRec sw;
    sw.a = br.b; sw.b = br.a; sw.mx = 1.0f; sw.L0 = br.L0;
    sw.p0 = 1.0f - br.p0; sw.lnx0 = br.lny0; sw.lny0 = br.lnx0; sw.lns = br.lns;
    const TailParams tp = {b, a, lnB};
    const float q = 1.0f - u;  // exact on the uniform grid
    *ln1mx = ara_polish_ln_quantile(sw, tp, q, log((double)q), &ok);
    *lnx = log1p(-exp(*ln1mx));
  }
  return ok;
}

// Fills a record's start table (kStartPieces quintics of the log-odds in tau, kStartCoefs
// floats each, see ara_start_logit) from binary32 inversions at the knots
// z_i = -kTableZ + 4 i kTableH: the lower tail through the record, the upper through the swapped
// record at q = 1 - u, so that u near 1 keeps its precision; the derivatives in z are those of
// the certified tables (L'' taken on each piece's own side of the median).  Pieces with a failed
// knot are NaN.
ARA_HD void ara_build_start_record(const BetaRec& br, float* st) {
  if (!(br.a > 0.0f)) {  // sd = 0: never inverted
    for (int k = 0; k < kStartFloats; ++k) st[k] = 0.0f;
    return;
  }
  BetaRec sw;
  sw.a = br.b; sw.b = br.a; sw.mx = br.mx; sw.L0 = br.L0;
  sw.p0 = 1.0f - br.p0; sw.lnx0 = br.lny0; sw.lny0 = br.lnx0; sw.lns = br.lns;
  const float lnB = br.a * br.lnx0 + br.b * br.lny0 - br.L0;
  const float H = 4.0f * kTableH;
  float L[kStartPieces + 1], D[kStartPieces + 1], X[kStartPieces + 1], Y[kStartPieces + 1];
  bool ok[kStartPieces + 1];
  for (int i = 0; i <= kStartPieces; ++i) {
    const float z = -kTableZ + (float)i * H;
    const float t = kTableTm + fabsf(z);
    const float lnq = -0.5f * t * t;
    const float q = expf(lnq);
    float lnx, ln1mx;
    bool conv;
    if (z >= 0.0f) {  // lower tail: u = q
      const IbetaResult r = ara_inv_beta(br, q);
      conv = r.converged;
      if (q > br.p0) { ln1mx = r.t; lnx = log1pf(-expf(r.t)); }
      else { lnx = r.t; ln1mx = log1pf(-expf(r.t)); }
    } else {  // upper tail: 1 - x ~ Beta(b, a) at probability q
      const IbetaResult r = ara_inv_beta(sw, q);
      conv = r.converged;
      if (q > sw.p0) { lnx = r.t; ln1mx = log1pf(-expf(r.t)); }
      else { ln1mx = r.t; lnx = log1pf(-expf(r.t)); }
    }
    L[i] = lnx - ln1mx;
    D[i] = -t * expf(lnq + lnB - br.a * lnx - br.b * ln1mx);
    X[i] = expf(lnx);
    Y[i] = expf(ln1mx);
    ok[i] = conv && isfinite(L[i]) && isfinite(D[i]);
  }
  for (int k = 0; k < kStartPieces; ++k) {
    float* c = st + k * kStartStride;
    c[6] = c[7] = 0.0f;  // padding of the piece's sector
    if (!(ok[k] && ok[k + 1])) {
      for (int j = 0; j < kStartCoefs; ++j) c[j] = ara_bits_to_float(0x7FC00000);
      continue;
    }
    // L'' = L'^2 (b x - a (1-x)) - s (t^2 - 1) L' / t, s the piece's side of the median
    const float s = k < kStartPieces / 2 ? -1.0f : 1.0f;
    float E[2];
    for (int e = 0; e < 2; ++e) {
      const int i = k + e;
      const float t = kTableTm + fabsf(-kTableZ + (float)i * H);
      E[e] = D[i] * D[i] * (br.b * X[i] - br.a * Y[i]) - s * (t * t - 1.0f) * D[i] / t;
    }
    c[0] = L[k];
    c[1] = H * D[k];
    c[2] = 0.5f * H * H * E[0];
    const float A = L[k + 1] - (c[0] + c[1] + c[2]);
    const float B = H * D[k + 1] - (c[1] + 2.0f * c[2]);
    const float C = H * H * E[1] - 2.0f * c[2];
    c[3] = 10.0f * A - 4.0f * B + 0.5f * C;
    c[4] = -15.0f * A + 7.0f * B - C;
    c[5] = 6.0f * A - 3.0f * B + 0.5f * C;
    if (!(isfinite(c[3]) && isfinite(c[4]) && isfinite(c[5])))
      for (int j = 0; j < kStartCoefs; ++j) c[j] = ara_bits_to_float(0x7FC00000);
  }
}

// ---- certified tables ------------------------------------------------------------------------------

// ln(x^a (1-x)^b / B(a,b)) as L0 + a ln(x/x0) + b ln(y/y0), with w = (x - x0)(a+b) taken from
// the smaller of x and y, so that it has no cancellation near the mean; *mag receives the sum of
// the magnitudes of its terms (its rounding scales with it).
ARA_HD float ara_beta_log_prefactor(const BetaRec& br, float lnx, float ln1mx, float x, float y,
                                    float* mag) {
  const float a = br.a, b = br.b, s = a + b;
  const float w = x < 0.5f ? fmaf(x, s, -a) : fmaf(-y, s, b);
  const float rx = w / a, ry = -w / b;
  const float lnrx = rx > -0.5f ? log1pf(rx) : lnx - br.lnx0;
  const float lnry = ry > -0.5f ? log1pf(ry) : ln1mx - br.lny0;
  *mag = fabsf(br.L0) + fabsf(a * lnrx) + fabsf(b * lnry);
  return br.L0 + a * lnrx + b * lnry;
}

// A knot: L and its derivatives in z, L'' = L2a - s L2b on the side s of the median.
struct KnotF {
  float z, L, L1, L2a, L2b;
  float gmag;  // magnitude of the terms of the inversion's residual at the root
  bool ok;
};

// Log-odds of the quantile at z (start: an estimate of it, or 1e30 for the analytic start) and
// its derivatives in z: L' = -t e^(ln q - E), E the log prefactor at the root.  Out of line: the
// build's three call sites then share one copy of the inversion (instruction-cache footprint).
ARA_HD_CALL KnotF ara_knot(const BetaRec& br, const BetaRec& sw, float z, float start) {
  KnotF k;
  k.z = z;
  const float t = kTableTm + fabsf(z);
  const float lnq = -0.5f * t * t;
  const float q = expf(lnq);
  float lnx, ln1mx;
  bool conv;
  if (z >= 0.0f) {  // lower tail: u = q
    const IbetaResult r = ara_inv_beta(br, q, start);
    conv = r.converged;
    if (q > br.p0) { ln1mx = r.t; lnx = log1pf(-expf(r.t)); }
    else { lnx = r.t; ln1mx = log1pf(-expf(r.t)); }
  } else {  // upper tail: 1 - x ~ Beta(b, a) at probability q (start: the log-odds of 1 - x)
    const IbetaResult r = ara_inv_beta(sw, q, start < 1e29f ? -start : start);
    conv = r.converged;
    if (q > sw.p0) { lnx = r.t; ln1mx = log1pf(-expf(r.t)); }
    else { ln1mx = r.t; lnx = log1pf(-expf(r.t)); }
  }
  const float x = expf(lnx), y = expf(ln1mx);
  float mag;
  k.L = lnx - ln1mx;
  k.L1 = -t * expf(lnq - ara_beta_log_prefactor(br, lnx, ln1mx, x, y, &mag));
  k.gmag = 2.0f + mag - lnq;
  k.L2a = k.L1 * k.L1 * (br.b * x - br.a * y);
  k.L2b = (t * t - 1.0f) * k.L1 / t;
  k.ok = conv && isfinite(k.L) && isfinite(k.L1) && isfinite(k.L2a) && isfinite(k.L2b);
  return k;
}

// Pieces [i0, i1) of a record's table (br.a > 0), the knots chained from z_i0 (its own start
// analytic); true if every one passed its midpoint check.  Writes coefficients, mx and
// kPieceTable; the caller turns every piece of a record that failed anywhere to kPieceNewton.
ARA_HD bool ara_build_table_pieces(const BetaRec& br, int i0, int i1, TablePiece* pc) {
  BetaRec sw;  // the swapped record: 1 - x ~ Beta(b, a), whose own mean probability is 1 - p0
  sw.a = br.b; sw.b = br.a; sw.mx = br.mx; sw.L0 = br.L0;
  sw.p0 = 1.0f - br.p0; sw.lnx0 = br.lny0; sw.lny0 = br.lnx0; sw.lns = br.lns;
  const float h = kTableH, z0 = -kTableZ;
  const float kLog2e = 1.44269504f, kLn2 = 0.693147181f;
  const int half = kTablePieces / 2;
  KnotF k0 = ara_knot(br, sw, z0 + (float)i0 * h, 1e30f);
  bool ok = k0.ok;
  float d3 = 0.0f;  // third derivative over the piece before, by difference (0: none this side)
  for (int i = i0; i < i1 && ok; ++i) {
    const float side = i < half ? -1.0f : 1.0f;  // the median is the boundary of pieces half-1, half
    if (i == half) d3 = 0.0f;
    const float d2 = k0.L2a - side * k0.L2b;
    // the next knot starts from the cubic Taylor step, so one Halley step nearly always suffices
    const float guess = fmaf(h, fmaf(h, fmaf(h * (1.0f / 6.0f), d3, 0.5f * d2), k0.L1), k0.L);
    const KnotF k1 = ara_knot(br, sw, z0 + (float)(i + 1) * h, guess);
    const float e2 = k1.L2a - side * k1.L2b;
    d3 = (e2 - d2) * kTableInvH;
    // quintic Hermite on tau in [0,1]: values, h * first, h^2 * second derivatives at both ends
    float c[6];
    c[0] = k0.L;
    c[1] = h * k0.L1;
    c[2] = 0.5f * h * h * d2;
    const float A = k1.L - (c[0] + c[1] + c[2]);
    const float B = h * k1.L1 - (c[1] + 2.0f * c[2]);
    const float C = h * h * e2 - 2.0f * c[2];
    c[3] = 10.0f * A - 4.0f * B + 0.5f * C;
    c[4] = -15.0f * A + 7.0f * B - C;
    c[5] = 6.0f * A - 3.0f * B + 0.5f * C;
    TablePiece p;
    for (int j = 0; j < 6; ++j) p.c[j] = c[j] * kLog2e;
    p.mx = br.mx;
    p.flag = kPieceTable;
    pc[i] = p;
    // the check at the midpoint, against the inversion started from the piece (as stored)
    const float Lt =
        kLn2 * fmaf(0.5f, fmaf(0.5f, fmaf(0.5f, fmaf(0.5f, fmaf(0.5f, p.c[5], p.c[4]), p.c[3]),
                                          p.c[2]),
                               p.c[1]),
                    p.c[0]);
    const KnotF km = ara_knot(br, sw, z0 + ((float)i + 0.5f) * h, Lt);
    const float tol = (float)kTableTol + 2.384185791015625e-7f * fabsf(km.L) +
                      fminf(kTableNoiseUlps * 5.9604645e-8f * km.gmag * fabsf(km.L1) /
                                (kTableTm + fabsf(km.z)),
                            kTableNoiseCap);
    ok = k1.ok && km.ok && fabsf(Lt - km.L) <= tol;
    k0 = k1;
  }
  return ok;
}

// Pieces [i0, i1) of a record that is not tabulated: the mean (sd = 0) or Newton's method.
ARA_HD void ara_table_fill(TablePiece* pc, int i0, int i1, float mx, uint32_t flag) {
  for (int i = i0; i < i1; ++i) {
    if (flag == kPieceMean)
      for (int j = 0; j < 6; ++j) pc[i].c[j] = 0.0f;
    pc[i].mx = mx;
    pc[i].flag = flag;
  }
}

// A record's whole table in one pass (the kernels split it into kTableSegments chains); *ok_out:
// every piece certified (else every piece says kPieceNewton).
constexpr int kTableSegments = 4;
ARA_HD void ara_build_table_record(const BetaRec& br, TablePiece* pc, bool* ok_out) {
  *ok_out = true;
  if (!(br.a > 0.0f)) {  // sd = 0: the loss is the mean
    ara_table_fill(pc, 0, kTablePieces, br.mx, kPieceMean);
    return;
  }
  constexpr int per = kTablePieces / kTableSegments;
  bool ok = true;
  for (int g = 0; g < kTableSegments; ++g)
    ok = ara_build_table_pieces(br, g * per, (g + 1) * per, pc) && ok;
  if (!ok) ara_table_fill(pc, 0, kTablePieces, br.mx, kPieceNewton);
  *ok_out = ok;
}
static_assert(kTablePieces % kTableSegments == 0 && 32 % kTableSegments == 0,
              "segments split the pieces evenly and a warp into whole records");

}  // namespace ara
