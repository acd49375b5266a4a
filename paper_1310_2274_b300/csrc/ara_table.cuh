// ara_table.cuh -- construction of the certified per-record quantile tables (host and device).
//
// For each tail, kTableIntervals + 1 knots are placed uniformly in t = sqrt(-2 ln q) between the
// mean (q = p0, or 1 - p0 for the upper tail) and the smallest uniform 2^-24.  The quantile at a
// knot comes from the binary32 Newton inversion (which works in ln x, so tails that underflow
// binary32 are still tabulated); r = ln x and its first two derivatives in t follow from the beta
// density; each piece's quintic Hermite coefficients are formed in binary64.  Each piece is then
// checked at its midpoint against the polished inversion; a record keeps its table only if every
// midpoint agrees to kTableTol in x plus the binary32 rounding of ln x (where x > 1e-30).
//
// Derivatives (s = ln u = -t^2/2, r = ln x, f the beta density):
//   dr/ds = u / (x f(x)),  x f(x) = x^a y^b / (y B(a,b)) = exp(E) / y,
//   d2r/ds2 = r_s (1 - r_s (a - (b-1) x / y)),
//   dr/dt = -t r_s,  d2r/dt2 = t^2 r_ss - r_s.
#pragma once

#include "ara_ibeta.cuh"

namespace ara {

constexpr double kTableTol = 1e-6;

// K = 1/(1 + d1/(1 + ...)) of DLMF 8.17.22 in binary64 by the Wallis recurrence of the
// division-free equivalent fraction (numerators -(a+b)x, -(a+m)(a+b+m)x, m(b-m)x; denominators
// a+n), rescaled by powers of two every step pair.
ARA_HD double ara_beta_cf_f64(double a, double b, double x) {
  const double apb = a + b;
  double Am2 = 1.0, Am1 = 1.0, Bm2 = 0.0, Bm1 = 1.0, prev = 1.0, res = 1.0;
  for (int n = 1; n < 4000; n += 2) {
    const double m = 0.5 * (double)(n - 1);
    const double al_odd = (n == 1) ? -apb * x : -(a + m) * (apb + m) * x;
    const double be_odd = a + (double)n;
    double A = be_odd * Am1 + al_odd * Am2;
    double B = be_odd * Bm1 + al_odd * Bm2;
    Am2 = Am1; Bm2 = Bm1; Am1 = A; Bm1 = B;
    const double m2 = m + 1.0;
    const double al_even = m2 * (b - m2) * x;
    const double be_even = a + (double)(n + 1);
    A = be_even * Am1 + al_even * Am2;
    B = be_even * Bm1 + al_even * Bm2;
    Am2 = Am1; Bm2 = Bm1; Am1 = A; Bm1 = B;
    int e;
    frexp(Am1, &e);
    Am1 = ldexp(Am1, -e); Am2 = ldexp(Am2, -e); Bm1 = ldexp(Bm1, -e); Bm2 = ldexp(Bm2, -e);
    res = Bm1 / Am1;
    if (fabs(res - prev) <= 1e-15 * fabs(res)) break;
    prev = res;
  }
  return res;
}

// ln I_x(a,b) for x = e^r (DLMF 8.17.22; past (a+1)/(a+b+2) through DLMF 8.17.4).
ARA_HD double ara_ln_betainc_f64(double a, double b, double r, double lnB) {
  const double x = exp(r);
  if (x < (a + 1.0) / (a + b + 2.0)) {
    return a * r + b * log1p(-x) - lnB + log(ara_beta_cf_f64(a, b, x)) - log(a);
  }
  const double y = 1.0 - x;
  const double Iy = exp(b * log(y) + a * r - lnB) * ara_beta_cf_f64(b, a, y) / b;
  return log1p(-Iy);
}

// The tail's beta parameters in binary64 (as computed from mean, sd and max when the ELT was
// staged) and ln B(a,b).
struct TailParams {
  double a, b, lnB;
};

struct Knot {
  double r, rt, rtt;  // ln x and its derivatives in t at the knot
  bool ok;
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
  {  // one binary64 Newton step: the binary32 start is within ~1e-7, so the step lands ~1e-14
    const double lnI = ara_ln_betainc_f64(a, b, r, tp.lnB);
    const double x = exp(r);
    const double dG = exp(a * r + (b - 1.0) * log1p(-x) - tp.lnB - lnI);
    const double step = (lnI - su) / dG;
    if (isfinite(step)) r -= step;
  }
  *ok = res.converged && isfinite(r);
  return r;
}

// Quantile data at table coordinate t: r = ln x and its derivatives in t, in binary64.
ARA_HD Knot knot_at(const BetaRec& br, const TailParams& tp, double t) {
  Knot k;
  const double su = -0.5 * t * t;  // ln u at the knot, exactly
  float uf = (float)exp(su);
  if (!(uf <= br.p0)) uf = br.p0;  // start on this tail
  if (!(uf > 0.0f)) uf = 1.17549435e-38f;
  bool ok;
  const double r = ara_polish_ln_quantile(br, tp, uf, su, &ok);
  const double a = tp.a, b = tp.b;
  const double x = exp(r);
  const double lny = log1p(-x);
  // x f(x) = x^a y^b / (y B(a,b))
  const double lnxf = a * r + (b - 1.0) * lny - tp.lnB;
  const double rs = exp(su - lnxf);
  const double rss = rs * (1.0 - rs * (a - (b - 1.0) * x / (1.0 - x)));
  k.r = r;
  k.rt = -t * rs;
  k.rtt = t * t * rss - rs;
  k.ok = ok && isfinite(k.rt) && isfinite(k.rtt);
  return k;
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

// Builds one tail: writes kTableIntervals pieces to iv and the span to *tlo_out, *ih_out;
// returns false if certification fails.  Pieces hold log2 x (the evaluation's exponential is
// base 2).
ARA_HD bool build_tail(const BetaRec& br, const TailParams& tp, float p_end, float4* iv,
                       float* tlo_out, float* ih_out) {
  float tlo_f, invh_f;
  ara_table_span(p_end, &tlo_f, &invh_f);
  *tlo_out = tlo_f;
  *ih_out = invh_f;
  const double kLog2e = 1.4426950408889634;
  const double tlo = tlo_f;
  const double h = 1.0 / (double)invh_f;  // the evaluation's own piece width
  bool ok = h > 0.0 && isfinite(h);
  Knot k0 = knot_at(br, tp, tlo);
  ok = ok && k0.ok;
  for (int i = 0; i < kTableIntervals; ++i) {
    const Knot k1 = knot_at(br, tp, tlo + (i + 1) * h);
    ok = ok && k1.ok;
    // quintic Hermite on tau in [0,1]: values, h * first, h^2 * second derivatives at both ends
    double c[6];
    c[0] = k0.r;
    c[1] = h * k0.rt;
    c[2] = 0.5 * h * h * k0.rtt;
    const double A = k1.r - (c[0] + c[1] + c[2]);
    const double B = h * k1.rt - (c[1] + 2.0 * c[2]);
    const double C = h * h * k1.rtt - 2.0 * c[2];
    c[3] = 10.0 * A - 4.0 * B + 0.5 * C;
    c[4] = -15.0 * A + 7.0 * B - C;
    c[5] = 6.0 * A - 3.0 * B + 0.5 * C;
    float c2[6];  // log2 x coefficients as stored
    for (int j = 0; j < 6; ++j) c2[j] = (float)(c[j] * kLog2e);
    iv[2 * i] = ara_make_float4(c2[0], c2[1], c2[2], c2[3]);
    iv[2 * i + 1] = ara_make_float4(c2[4], c2[5], 0.0f, 0.0f);
    // certify at the midpoint against the Newton inversion (binary32 coefficients as stored)
    const Knot km = knot_at(br, tp, tlo + (i + 0.5) * h);
    double cf[6];
    for (int j = 0; j < 6; ++j) cf[j] = (double)c2[j] / kLog2e;
    const double rp = piece_eval(cf, 0.5);
    if (km.r > -69.0) {
      // allowed: kTableTol plus the binary32 rounding of r itself (4 ulp of |r|), which
      // dominates only for x < ~1e-12, far below any loss that reaches a year loss
      const double err = fabs(expm1(rp - km.r));
      const double tol = kTableTol + 2.384185791015625e-7 * fabs(km.r);
      if (!(err <= tol) || !km.ok) ok = false;
    }
    k0 = k1;
  }
  return ok;
}


// br: the record in binary32; a64, b64: its beta parameters in binary64; p0 = I_{x0}(a,b).
ARA_HD void ara_build_table_record(const BetaRec& br, double a64, double b64, float4* iv,
                                   TableRec* out, bool* ok_out) {
  TableRec tr;
  tr.mx = br.mx;
  tr.iv = nullptr;
  tr.tlo[0] = tr.tlo[1] = tr.ih[0] = tr.ih[1] = 0.0f;
  *ok_out = true;
  if (!(br.a > 0.0f)) {  // sd = 0: the loss is the mean
    tr.p0 = -1.0f;
    *out = tr;
    return;
  }
  tr.p0 = br.p0;
  const double lnB = lgamma(a64) + lgamma(b64) - lgamma(a64 + b64);
  const TailParams lo = {a64, b64, lnB}, up = {b64, a64, lnB};
  bool ok = build_tail(br, lo, br.p0, iv, &tr.tlo[0], &tr.ih[0]);
  // upper tail: y = 1 - x solves I_y(b, a) = 1 - u, whose own mean probability is 1 - p0
  BetaRec sw;
  sw.a = br.b; sw.b = br.a; sw.mx = br.mx; sw.L0 = br.L0;
  sw.p0 = 1.0f - br.p0; sw.lnx0 = br.lny0; sw.lny0 = br.lnx0; sw.lns = br.lns;
  ok = ok && build_tail(sw, up, 1.0f - br.p0, iv + 2 * kTableIntervals, &tr.tlo[1], &tr.ih[1]);
  if (ok) tr.iv = iv;
  *ok_out = ok;
  *out = tr;
}

}  // namespace ara
