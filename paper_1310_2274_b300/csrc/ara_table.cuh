// ara_table.cuh -- construction of the certified per-record quantile tables (host and device).
//
// Knots are placed at z_i = -kTableZ + i kTableH (i = 0..kTablePieces), z the signed distance
// from the median in t = sqrt(-2 ln q), q = min(u, 1 - u).  The quantile at a knot comes from
// the binary32 Newton inversion on the record's own tail (u <= p0: x itself; u > p0: 1 - x of
// the swapped record, so x near 1 keeps its precision), polished by one binary64 Newton step;
// the log-odds L = ln x - ln(1-x) and its first two derivatives in z follow from the beta density;
// each piece's quintic Hermite coefficients are formed in binary64.  Each piece is then checked at
// its midpoint against a polished inversion; a record keeps its table only if every midpoint
// agrees to kTableTol in L (so in x/(1-x) relatively) plus the binary32 rounding of L.
//
// Derivatives (g = dL/du = B(a,b) / (x^a (1-x)^b), t = t_m + |z|, u(z) with du/dz = -t q):
//   L'  = -t q g,
//   L'' = L'^2 (b x - a (1 - x)) - s (t^2 - 1) L' / t,   s = +1 for z > 0, -1 for z < 0;
// L'' jumps at the median (z = 0), which is a piece boundary: each side uses its own value.
#pragma once

#include "ara_ibeta.cuh"

namespace ara {

constexpr double kTableTol = 1e-6;

// ---- double-float arithmetic -------------------------------------------------------------------
// A value hi + lo of two binary32 numbers (|lo| <= ulp(hi)/2, ~48 significant bits): the FP64 pipe
// of this part is 1/64 of the FP32 one, so the build's continued fraction runs in pairs of
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
// (pA, pB: the previous pair at the same scale).  The knots need L to ~1e-9 (pieces fit to ~1e-8,
// certified to 1e-6).
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

ARA_HD double piece_eval(const double* c, double tau) {
  return c[0] + tau * (c[1] + tau * (c[2] + tau * (c[3] + tau * (c[4] + tau * c[5]))));
}

// Log-odds of the quantile at z and its first two derivatives in z (the second from the side s).
struct LogitKnot {
  double L, L1, L2;
  bool ok;
};

ARA_HD LogitKnot logit_knot(const BetaRec& br, const BetaRec& sw, const TailParams& lo,
                            const TailParams& up, double z, double s) {
  LogitKnot k;
  const double t = (double)kTableTm + fabs(z);
  const double lnq = -0.5 * t * t;
  const float qf = expf((float)lnq);
  // u = q below the median, 1 - q above it; ln u or ln(1 - u) (whichever the solve needs) in
  // binary64 without cancellation.  The complement ln(1 - v) of the solved v = x or 1 - x is
  // well conditioned in binary32 while v <= 1/2 (it enters L at the 1e-7 level); above that it
  // takes binary64
  const bool below = z >= 0.0 ? (double)qf <= (double)br.p0 : (1.0 - (double)qf) <= (double)br.p0;
  bool ok;
  double lnx, ln1mx;
  if (below) {
    const double lnu = z >= 0.0 ? lnq : log1p(-exp(lnq));
    float uf = (float)exp(lnu);
    if (!(uf <= br.p0)) uf = br.p0;
    if (!(uf > 0.0f)) uf = 1.17549435e-38f;
    lnx = ara_polish_ln_quantile(br, lo, uf, lnu, &ok);
    ln1mx = lnx < -0.6931471805599453 ? (double)log1pf(-expf((float)lnx)) : log1p(-exp(lnx));
  } else {
    const double ln1mu = z >= 0.0 ? log1p(-exp(lnq)) : lnq;
    float vf = (float)exp(ln1mu);
    if (!(vf <= sw.p0)) vf = sw.p0;
    if (!(vf > 0.0f)) vf = 1.17549435e-38f;
    ln1mx = ara_polish_ln_quantile(sw, up, vf, ln1mu, &ok);
    lnx = ln1mx < -0.6931471805599453 ? (double)log1pf(-expf((float)ln1mx)) : log1p(-exp(ln1mx));
  }
  const double a = lo.a, b = lo.b;
  // the derivatives need ~1e-7 relative accuracy only (they enter the pieces multiplied by h and
  // h^2): exponents in binary64, exponentials in binary32
  const double x = (double)expf((float)lnx), y = (double)expf((float)ln1mx);
  k.L = lnx - ln1mx;
  k.L1 = -t * (double)expf((float)(lnq + lo.lnB - a * lnx - b * ln1mx));
  k.L2 = k.L1 * k.L1 * (b * x - a * y) - s * (t * t - 1.0) * k.L1 / t;
  k.ok = ok && isfinite(k.L) && isfinite(k.L1) && isfinite(k.L2);
  return k;
}

// Fills a record's kTablePieces pieces (pc) and reports whether every piece was certified.
// br: the record in binary32; a64, b64: its beta parameters in binary64.
ARA_HD void ara_build_table_record(const BetaRec& br, double a64, double b64, TablePiece* pc,
                                   bool* ok_out) {
  *ok_out = true;
  if (!(br.a > 0.0f)) {  // sd = 0: the loss is the mean
    for (int i = 0; i < kTablePieces; ++i) {
      for (int j = 0; j < 6; ++j) pc[i].c[j] = 0.0f;
      pc[i].mx = br.mx;
      pc[i].flag = kPieceMean;
    }
    return;
  }
  const double lnB = lgamma(a64) + lgamma(b64) - lgamma(a64 + b64);
  const TailParams lo = {a64, b64, lnB, log(a64)}, up = {b64, a64, lnB, log(b64)};
  BetaRec sw;  // the swapped record: 1 - x ~ Beta(b, a), whose own mean probability is 1 - p0
  sw.a = br.b; sw.b = br.a; sw.mx = br.mx; sw.L0 = br.L0;
  sw.p0 = 1.0f - br.p0; sw.lnx0 = br.lny0; sw.lny0 = br.lnx0; sw.lns = br.lns;
  const double h = (double)kTableH, z0 = -(double)kTableZ;
  const double kLog2e = 1.4426950408889634;
  bool ok = true;
  const int half = kTablePieces / 2;
  LogitKnot k0 = logit_knot(br, sw, lo, up, z0, -1.0);
  ok = ok && k0.ok;
  for (int i = 0; i < kTablePieces && ok; ++i) {
    const double side = i < half ? -1.0 : 1.0;  // the median is the boundary of pieces half-1, half
    if (i == half) k0 = logit_knot(br, sw, lo, up, 0.0, 1.0);
    const LogitKnot k1 = logit_knot(br, sw, lo, up, z0 + (i + 1) * h, side);
    ok = ok && k0.ok && k1.ok;
    // quintic Hermite on tau in [0,1]: values, h * first, h^2 * second derivatives at both ends
    double c[6];
    c[0] = k0.L;
    c[1] = h * k0.L1;
    c[2] = 0.5 * h * h * k0.L2;
    const double A = k1.L - (c[0] + c[1] + c[2]);
    const double B = h * k1.L1 - (c[1] + 2.0 * c[2]);
    const double C = h * h * k1.L2 - 2.0 * c[2];
    c[3] = 10.0 * A - 4.0 * B + 0.5 * C;
    c[4] = -15.0 * A + 7.0 * B - C;
    c[5] = 6.0 * A - 3.0 * B + 0.5 * C;
    double cf[6];  // the stored log2-odds coefficients, back in natural units
    for (int j = 0; j < 6; ++j) {
      pc[i].c[j] = (float)(c[j] * kLog2e);
      cf[j] = (double)pc[i].c[j] / kLog2e;
    }
    pc[i].mx = br.mx;
    pc[i].flag = kPieceTable;
    // certify at the midpoint against a polished inversion (coefficients as stored)
    const LogitKnot km = logit_knot(br, sw, lo, up, z0 + (i + 0.5) * h, side);
    const double err = fabs(piece_eval(cf, 0.5) - km.L);
    // allowed: kTableTol plus the binary32 rounding of L (4 ulp of |L|), which dominates only for
    // x or 1 - x below ~1e-12, far below any loss that reaches a year loss
    const double tol = kTableTol + 2.384185791015625e-7 * fabs(km.L);
    if (!(err <= tol) || !km.ok) ok = false;
    k0 = k1;
  }
  if (!ok) {
    for (int i = 0; i < kTablePieces; ++i) {
      pc[i].mx = br.mx;
      pc[i].flag = kPieceNewton;
    }
  }
  *ok_out = ok;
}

// Fills a record's start table (kStartPieces quintics of the log-odds in tau, kStartCoefs
// floats each, see ara_start_logit) from binary32 inversions at the knots
// z_i = -kTableZ + 4 i kTableH: the lower tail through the record, the upper through the swapped
// record at q = 1 - u, so that u near 1 keeps its precision; the derivatives in z are those of
// logit_knot (L'' taken on each piece's own side of the median).  Pieces with a failed knot are
// NaN.
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

}  // namespace ara
