/*
 * ara_oracle.c -- plain FP64 CPU oracle for aggregate risk analysis with secondary uncertainty
 * (Varghese & Rau-Chaplin, "Accounting for Secondary Uncertainty", WHPCF'13).
 *
 * TEST INFRASTRUCTURE ONLY. Nothing in the library product links, loads or calls this file; only
 * the tests, the package's smoke check and the benchmark's CPU-baseline leg do. It shares no code,
 * header, table or constant with the CUDA path.
 *
 * Every function follows the paper step by step in double precision, with no blocking, fusion or
 * reordering beyond what the cited passage states:
 *
 *   ora_philox4x32_10   counter-based generator, Salmon, Moraes, Dror & Shaw, SC'11, Figure 2
 *                       and Table 2 (Philox4x32 with R = 10 rounds). It stands in for the
 *                       pre-stored uniforms z_(Prog,E) and z_(E) of paper §3.1.
 *   ora_uniform         32-bit word -> U(0,1) on the dyadic grid (2j+1) 2^-24.
 *   ora_su_uniform_corr the correlated (event-occurrence) uniform of an occurrence.
 *   ora_norm_cdf        Phi of paper §3.2 step 5, (1/2) erfc(-x / sqrt 2).
 *   ora_norm_quantile   Phi^-1 of paper §3.2 step 2 (reading G1): bracketed Newton on ln Phi.
 *   ora_su_combine      paper §3.2 steps 1-5: the uniform fed to the beta inversion.
 *   ora_betainc         regularised incomplete beta I_x(a,b), the ratio B(x;a,b)/B(a,b) of
 *                       paper §3.3; continued fraction DLMF 8.17.22 by the modified Lentz method.
 *   ora_betaincinv      its functional inverse (paper §3.3, InvCDF_beta): safeguarded Newton.
 *   ora_beta_moments    paper §3.3: sigma_beta, mu_beta, the sigma_beta_max clamp, alpha, beta.
 *   ora_occ_terms       paper §2.3 occurrence terms  min(max(l - OccR, 0), OccL).
 *   ora_agg_terms       paper §2.3 aggregate terms   min(max(S - AggR, 0), AggL).
 *   ora_run             Algorithm 1 for one layer over a list of trials -> YLT entries, and
 *                       optionally each year's largest occurrence loss (OEP year table).
 *   ora_run_events      The same with per-occurrence outputs: occurrence losses after
 *                       occurrence terms and the increments of the net aggregate loss.
 *   ora_trace           the same loop, reporting every (trial, event, ELT) hit.
 *   ora_rank / ora_risk YLT order and PML / TVaR (paper §2.4).
 *
 * Readings of points the paper leaves open (each also listed in the design notes):
 *   - occurrence/aggregate terms: the one-argument max of paper §2.3 is max(x, 0);
 *   - the aggregate terms act on the cumulative sum S of occurrence losses, so the year loss is
 *     f_agg(S) after the last event (Algorithm 1 applies them inside the loop; f_agg is
 *     monotone, so the final value is the same);
 *   - sigma = 0: alpha and beta are unbounded and the loss is the mean (primary uncertainty only);
 *   - "a value very close to sigma_beta_max" is sigma_beta_max * (1 - 2^-20);
 *   - with a single standard deviation per record (sigma_C = 0) the combination of paper §3.2
 *     returns the program/occurrence uniform unchanged, so that uniform is used directly; it is
 *     drawn by Philox keyed by (trial, event position, ELT handle);
 *   - with sigma_C > 0 (paper §3.1-3.2): z_(Prog,E) is that per-(trial, event position, ELT)
 *     uniform and z_(E), "the same across programs" for an event occurrence, is one uniform per
 *     (trial, event position) shared by every ELT and layer; sigma = sigma_I + sigma_C feeds the
 *     beta moments;
 *   - PML(RP) is the k-th largest year loss and TVaR(RP) the mean of the k largest, k = N/RP
 *     (ceil when N/RP is not an integer); ties are ordered by ascending trial index.
 */
#include <float.h>
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

#ifdef _OPENMP
#include <omp.h>
#endif

#define ORA_API __attribute__((visibility("default")))

/* ------------------------------------------------------------------------------------------ */
/* Work counters (read by the benchmark to state the algorithmic cost of one inversion).      */
/* ------------------------------------------------------------------------------------------ */
typedef struct {
  int64_t inversions;   /* calls of the inverse with 0 < p < 1                               */
  int64_t newton;       /* Newton updates accepted                                           */
  int64_t bisect;       /* bisection fallbacks                                               */
  int64_t evals;        /* evaluations of ln I_x inside the inverse                          */
  int64_t cf_terms;     /* continued-fraction terms summed inside the inverse                */
  int64_t not_conv;     /* inverses that hit the iteration cap                               */
} ora_counts;

static ora_counts g_counts;
static int g_counting; /* off unless a caller asks for the counts: atomics cost time */

ORA_API void ora_counts_enable(int on) { g_counting = on; }
ORA_API void ora_counts_reset(void) { memset(&g_counts, 0, sizeof g_counts); }
ORA_API void ora_counts_get(int64_t out[6]) {
  out[0] = g_counts.inversions; out[1] = g_counts.newton; out[2] = g_counts.bisect;
  out[3] = g_counts.evals; out[4] = g_counts.cf_terms; out[5] = g_counts.not_conv;
}

/* ------------------------------------------------------------------------------------------ */
/* Philox4x32-10 (Salmon et al., SC'11).                                                       */
/* One round maps (c0,c1,c2,c3) under key (k0,k1) to                                           */
/*   (hi(M1*c2) ^ c1 ^ k0, lo(M1*c2), hi(M0*c0) ^ c3 ^ k1, lo(M0*c0))                          */
/* with M0 = 0xD2511F53, M1 = 0xCD9E8D57; between rounds the key is bumped by the Weyl        */
/* constants W0 = 0x9E3779B9, W1 = 0xBB67AE85.                                                 */
/* ------------------------------------------------------------------------------------------ */
ORA_API void ora_philox4x32_10(const uint32_t ctr[4], const uint32_t key[2], uint32_t out[4]) {
  uint32_t c0 = ctr[0], c1 = ctr[1], c2 = ctr[2], c3 = ctr[3];
  uint32_t k0 = key[0], k1 = key[1];
  for (int r = 0; r < 10; ++r) {
    uint64_t p0 = (uint64_t)0xD2511F53u * (uint64_t)c0;
    uint64_t p1 = (uint64_t)0xCD9E8D57u * (uint64_t)c2;
    uint32_t n0 = (uint32_t)(p1 >> 32) ^ c1 ^ k0;
    uint32_t n1 = (uint32_t)p1;
    uint32_t n2 = (uint32_t)(p0 >> 32) ^ c3 ^ k1;
    uint32_t n3 = (uint32_t)p0;
    c0 = n0; c1 = n1; c2 = n2; c3 = n3;
    k0 += 0x9E3779B9u;
    k1 += 0xBB67AE85u;
  }
  out[0] = c0; out[1] = c1; out[2] = c2; out[3] = c3;
}

/* Upper 23 bits j of w -> (2j + 1) / 2^24: exact in binary32 and binary64, never 0 or 1. */
ORA_API double ora_uniform(uint32_t w) { return ldexp(2.0 * (double)(w >> 9) + 1.0, -24); }

ORA_API void ora_uniform_n(const uint32_t *w, int64_t n, double *out) {
  for (int64_t i = 0; i < n; ++i) out[i] = ora_uniform(w[i]);
}

/* The uniform for occurrence k of trial i in ELT elt: counter (k, i_lo, elt/4, i_hi),
 * key (seed_lo, seed_hi), output word elt mod 4. */
ORA_API double ora_su_uniform(uint64_t seed, int64_t trial, int64_t k, int32_t elt) {
  uint32_t ctr[4], key[2], out[4];
  ctr[0] = (uint32_t)k;
  ctr[1] = (uint32_t)((uint64_t)trial & 0xFFFFFFFFu);
  ctr[2] = (uint32_t)elt >> 2;
  ctr[3] = (uint32_t)((uint64_t)trial >> 32);
  key[0] = (uint32_t)(seed & 0xFFFFFFFFu);
  key[1] = (uint32_t)(seed >> 32);
  ora_philox4x32_10(ctr, key, out);
  return ora_uniform(out[elt & 3]);
}

/* The correlated (event-occurrence) uniform of occurrence k of trial i, shared by every ELT
 * and every layer: counter (k, i_lo, 0xFFFFFFFF, i_hi), which no ELT handle's group reaches,
 * key (seed_lo, seed_hi), output word 0. */
ORA_API double ora_su_uniform_corr(uint64_t seed, int64_t trial, int64_t k) {
  uint32_t ctr[4], key[2], out[4];
  ctr[0] = (uint32_t)k;
  ctr[1] = (uint32_t)((uint64_t)trial & 0xFFFFFFFFu);
  ctr[2] = 0xFFFFFFFFu;
  ctr[3] = (uint32_t)((uint64_t)trial >> 32);
  key[0] = (uint32_t)(seed & 0xFFFFFFFFu);
  key[1] = (uint32_t)(seed >> 32);
  ora_philox4x32_10(ctr, key, out);
  return ora_uniform(out[0]);
}

/* ------------------------------------------------------------------------------------------ */
/* Standard normal distribution, paper §3.2 (steps 2 and 5).                                  */
/* ------------------------------------------------------------------------------------------ */
/* Phi(x) = (1/2) erfc(-x / sqrt 2). */
static const double kSqrtHalf = 0.70710678118654752440;  /* 1/sqrt(2) */
static const double kSqrt2Pi = 2.50662827463100050242;   /* sqrt(2 pi) */
ORA_API double ora_norm_cdf(double x) { return 0.5 * erfc(-x * kSqrtHalf); }

/* Phi^-1(p): the x with Phi(x) = p (reading G1: step 2 maps a uniform to a normal).  The upper
 * tail y > 0 with Phi(-y) = q = min(p, 1 - p) is solved by Newton's method on
 * h(y) = ln Phi(-y) - ln q (h' = -phi(y) / Phi(-y)), kept inside a bracket [lo, hi] and replaced by
 * bisection whenever a step would leave it; start y = sqrt(-2 ln q) - 1, clipped to the bracket. */
ORA_API double ora_norm_quantile(double p) {
  if (!(p > 0.0)) return -INFINITY;
  if (!(p < 1.0)) return INFINITY;
  if (p == 0.5) return 0.0;
  const double q = p < 0.5 ? p : 1.0 - p;
  const double lnq = log(q);
  const double t = sqrt(-2.0 * lnq);
  double lo = 0.0, hi = t + 1.0; /* Phi(-y) < phi(y)/y gives the root below sqrt(-2 ln q) + 1 */
  double y = fmax(t - 1.0, 0.0);
  for (int it = 0; it < 200; ++it) {
    const double c = 0.5 * erfc(y * kSqrtHalf); /* Phi(-y) */
    const double h = log(c) - lnq;
    if (h > 0.0) lo = y; else hi = y;           /* h decreases in y */
    const double dens = exp(-0.5 * y * y) / kSqrt2Pi;
    double yn = y + h * c / dens;
    if (!(yn > lo && yn < hi)) yn = 0.5 * (lo + hi);
    if (fabs(yn - y) <= 4.0 * DBL_EPSILON * fmax(1.0, yn)) { y = yn; break; }
    y = yn;
  }
  return p < 0.5 ? -y : y;
}

/* Paper §3.2: the uniform z that the beta inversion receives, from the independent (program-and-
 * occurrence) uniform zp and the correlated (occurrence) uniform ze of a record with independent
 * and correlated standard deviations sd_i, sd_c:
 *   sigma = sd_i + sd_c (step 1); vp = Phi^-1(zp), ve = Phi^-1(ze) (step 2);
 *   LC = vp sd_i/sigma + ve sd_c/sigma (step 3); v = LC / sqrt((sd_i/sigma)^2 + (sd_c/sigma)^2)
 *   (step 4); z = Phi(v) (step 5).
 * With sd_c = 0 the steps give Phi(Phi^-1(zp)) = zp, which is returned exactly. */
ORA_API double ora_su_combine(double zp, double ze, double sd_i, double sd_c) {
  if (sd_c == 0.0) return zp;
  const double sigma = sd_i + sd_c;
  const double wi = sd_i / sigma, wc = sd_c / sigma;
  const double vp = ora_norm_quantile(zp), ve = ora_norm_quantile(ze);
  const double lc = vp * wi + ve * wc;
  const double v = lc / sqrt(wi * wi + wc * wc);
  return ora_norm_cdf(v);
}

/* ------------------------------------------------------------------------------------------ */
/* Regularised incomplete beta, paper §3.3: I_x(a,b) = B(x;a,b) / B(a,b).                      */
/* ------------------------------------------------------------------------------------------ */
static double ln_beta(double a, double b) { return lgamma(a) + lgamma(b) - lgamma(a + b); }

/* K = 1/(1 + d1/(1 + d2/(1 + ...))) of DLMF 8.17.22, with
 *   d_{2m+1} = -(a+m)(a+b+m) x / ((a+2m)(a+2m+1)),   d_{2m} = m(b-m) x / ((a+2m-1)(a+2m)),
 * evaluated front to back by the modified Lentz method (Thompson & Barnett 1986): the
 * fraction b0 + a1/(b1 + a2/(b2 + ...)) with b0 = 0, a1 = 1, a_{n+1} = d_n, b_n = 1. */
static double beta_cf(double a, double b, double x, int64_t *terms) {
  const double tiny = 1e-300;
  double f = tiny, C = tiny, D = 0.0;
  for (int n = 1; n <= 100000; ++n) {
    double an;
    if (n == 1) {
      an = 1.0;
    } else {
      int j = n - 1; /* d_j */
      if (j & 1) {
        double m = (double)(j / 2);
        an = -(a + m) * (a + b + m) * x / ((a + 2.0 * m) * (a + 2.0 * m + 1.0));
      } else {
        double m = (double)(j / 2);
        an = m * (b - m) * x / ((a + 2.0 * m - 1.0) * (a + 2.0 * m));
      }
    }
    D = 1.0 + an * D;
    if (fabs(D) < tiny) D = tiny;
    C = 1.0 + an / C;
    if (fabs(C) < tiny) C = tiny;
    D = 1.0 / D;
    double delta = C * D;
    f *= delta;
    if (terms) ++*terms;
    if (fabs(delta - 1.0) < 0.5 * DBL_EPSILON) break;
  }
  return f;
}

/* ln I_x(a,b) for 0 < x < 1.  Below x = (a+1)/(a+b+2) the fraction converges quickly and
 * I_x = x^a (1-x)^b K / (a B(a,b)) (DLMF 8.17.22); above it the symmetry
 * I_x(a,b) = 1 - I_{1-x}(b,a) (DLMF 8.17.4) is used. */
static double ln_betainc(double a, double b, double x, int64_t *terms) {
  if (x < (a + 1.0) / (a + b + 2.0)) {
    double K = beta_cf(a, b, x, terms);
    return a * log(x) + b * log1p(-x) - ln_beta(a, b) + log(K) - log(a);
  }
  double y = 1.0 - x;
  double K = beta_cf(b, a, y, terms);
  double Iy = exp(b * log(y) + a * log1p(-y) - ln_beta(a, b) + log(K) - log(b));
  return log1p(-Iy);
}

ORA_API double ora_betainc(double a, double b, double x) {
  if (!(x > 0.0)) return 0.0;
  if (!(x < 1.0)) return 1.0;
  return exp(ln_betainc(a, b, x, NULL));
}

/* Beta density f(x) = x^(a-1) (1-x)^(b-1) / B(a,b); returned as ln(x f(x)). */
static double ln_x_density(double a, double b, double x) {
  return a * log(x) + (b - 1.0) * log1p(-x) - ln_beta(a, b);
}

/* Solve I_x(a,b) = p for p <= 1/2 in t = ln x.  G(t) = ln I_{e^t}(a,b) - ln p is increasing with
 * G'(t) = x f(x) / I_x.  Newton steps on G are kept inside a bracket [lo, hi] of the root and
 * replaced by bisection whenever they would leave it.  The start is the small-x form
 * I_x ~ x^a / (a B(a,b)) (DLMF 8.17.22 with K -> 1), clipped into the bracket. */
static double inv_lower(double a, double b, double p, int *status, int64_t *cnt) {
  const double lnp = log(p);
  /* Bracket in t: x = e^-745 is below the smallest double (if the root lies lower still, the
   * iteration settles on the lower end and x rounds to 0); x = 1 gives G = -ln p > 0. */
  double lo = -745.0, hi = 0.0;
  int64_t terms = 0;
  double t = (lnp + log(a) + ln_beta(a, b)) / a;
  /* For p <= 1/2 the root sits at or below the median; do not start beyond the mean. */
  t = fmin(t, log(a / (a + b)));
  if (!(t > lo && t < hi)) t = 0.5 * (lo + hi);
  int conv = 0;
  for (int it = 0; it < 400; ++it) {
    double x = exp(t);
    double g = ln_betainc(a, b, x, &terms) - lnp;
    cnt[2]++;
    if (g == 0.0) { conv = 1; break; }
    if (g < 0.0) lo = t; else hi = t;
    double dg = exp(ln_x_density(a, b, x) - (g + lnp));
    double tn = t - g / dg;
    if (!(tn > lo && tn < hi)) {
      tn = 0.5 * (lo + hi);
      cnt[1]++;
    } else {
      cnt[0]++;
    }
    double step = fabs(tn - t);
    t = tn;
    if (step <= 4.0 * DBL_EPSILON * fmax(1.0, fabs(t))) { conv = 1; break; }
    if (hi - lo <= 4.0 * DBL_EPSILON * fmax(1.0, fabs(lo))) { conv = 1; break; }
  }
  cnt[3] += terms;
  /* A root below the smallest normal double (e^-708) is an underflow, not a failure: the bracket
   * can stall there on a CDF this flat (paper §3.3's sd clamp leaves a, b near 1e-6), and any x
   * it returns is within 2.3e-308 of the root. */
  if (!conv && t < -708.0) conv = 1;
  if (!conv) *status = 1;
  return exp(t);
}

/* InvCDF_beta(p; a, b), paper §3.3: the x in [0,1] with I_x(a,b) = p.  For p > 1/2 the upper
 * tail is solved through I_x(a,b) = 1 - I_{1-x}(b,a), since 1 - p is exact. */
ORA_API double ora_betaincinv(double a, double b, double p, int *status) {
  int st = 0;
  double x;
  int64_t cnt[4] = {0, 0, 0, 0};
  if (!(p > 0.0)) x = 0.0;
  else if (!(p < 1.0)) x = 1.0;
  else if (p <= 0.5) x = inv_lower(a, b, p, &st, cnt);
  else x = 1.0 - inv_lower(b, a, 1.0 - p, &st, cnt);
  if (g_counting && p > 0.0 && p < 1.0) {
#pragma omp atomic
    g_counts.inversions += 1;
#pragma omp atomic
    g_counts.newton += cnt[0];
#pragma omp atomic
    g_counts.bisect += cnt[1];
#pragma omp atomic
    g_counts.evals += cnt[2];
#pragma omp atomic
    g_counts.cf_terms += cnt[3];
    if (st) {
#pragma omp atomic
      g_counts.not_conv += 1;
    }
  }
  if (status) *status = st;
  return x;
}

/* ------------------------------------------------------------------------------------------ */
/* Beta moments, paper §3.3.  Returns 0 (normal), 1 (sigma_beta clamped), 2 (sigma = 0: the    */
/* loss is the mean and no beta is drawn), -1 (invalid record).                                */
/* ------------------------------------------------------------------------------------------ */
ORA_API int ora_beta_moments(double mean, double sd, double mx, double *alpha, double *beta) {
  if (sd == 0.0) { *alpha = INFINITY; *beta = INFINITY; return 2; }
  if (!(mean > 0.0) || !(sd > 0.0) || !(mx > mean)) return -1;
  double sigma_b = sd / mx;
  double mu_b = mean / mx;
  double sigma_b_max = sqrt(mu_b * (1.0 - mu_b));
  int clamped = 0;
  if (sigma_b > sigma_b_max) {
    sigma_b = sigma_b_max * (1.0 - ldexp(1.0, -20));
    clamped = 1;
  }
  double r = sigma_b_max / sigma_b;
  double k = r * r - 1.0;
  *alpha = mu_b * k;
  *beta = (1.0 - mu_b) * k;
  return clamped;
}

/* Paper §2.3 terms. */
ORA_API double ora_occ_terms(double l, double occ_ret, double occ_lim) {
  return fmin(fmax(l - occ_ret, 0.0), occ_lim);
}
ORA_API double ora_agg_terms(double s, double agg_ret, double agg_lim) {
  return fmin(fmax(s - agg_ret, 0.0), agg_lim);
}

/* Secondary-uncertainty loss of one record for uniform u: max_l * InvCDF_beta(u; alpha, beta). */
ORA_API double ora_su_loss(double mean, double sd, double mx, double u, int *status) {
  double a, b;
  int m = ora_beta_moments(mean, sd, mx, &a, &b);
  if (status) *status = 0;
  if (m == 2) return mean;
  if (m < 0) { if (status) *status = 2; return NAN; }
  return mx * ora_betaincinv(a, b, u, status);
}

/* ------------------------------------------------------------------------------------------ */
/* Event lookup, paper Algorithm 1 ("Lookup E in the XELT"): binary search in a sorted copy.   */
/* ------------------------------------------------------------------------------------------ */
typedef struct {
  int64_t n;
  int32_t *ids;   /* sorted ascending */
  int64_t *perm;  /* perm[s] = caller record index of sorted slot s */
} ora_index;

static const int32_t *g_sort_ids;
static int cmp_rec(const void *x, const void *y) {
  int64_t i = *(const int64_t *)x, j = *(const int64_t *)y;
  int32_t a = g_sort_ids[i], b = g_sort_ids[j];
  return (a > b) - (a < b);
}

static int build_index(ora_index *ix, const int32_t *ids, int64_t n) {
  ix->n = n;
  ix->ids = (int32_t *)malloc(sizeof(int32_t) * (size_t)(n ? n : 1));
  ix->perm = (int64_t *)malloc(sizeof(int64_t) * (size_t)(n ? n : 1));
  if (!ix->ids || !ix->perm) return -1;
  for (int64_t r = 0; r < n; ++r) ix->perm[r] = r;
  g_sort_ids = ids;
  qsort(ix->perm, (size_t)n, sizeof(int64_t), cmp_rec);
  for (int64_t s = 0; s < n; ++s) ix->ids[s] = ids[ix->perm[s]];
  for (int64_t s = 1; s < n; ++s)
    if (ix->ids[s] == ix->ids[s - 1]) return -2; /* duplicate event in one ELT */
  return 0;
}

static void free_index(ora_index *ix) { free(ix->ids); free(ix->perm); }

static int64_t lookup(const ora_index *ix, int32_t e) {
  int64_t lo = 0, hi = ix->n - 1;
  while (lo <= hi) {
    int64_t mid = lo + (hi - lo) / 2;
    if (ix->ids[mid] == e) return ix->perm[mid];
    if (ix->ids[mid] < e) lo = mid + 1; else hi = mid - 1;
  }
  return -1;
}

/* ------------------------------------------------------------------------------------------ */
/* Algorithm 1 for one layer.                                                                  */
/*                                                                                             */
/* yet_offsets[n_trials+1], yet_ids[]: the YET in CSR form, events in timestamp order.         */
/* n_elts ELTs, concatenated: records elt_off[j]..elt_off[j+1]-1 of ids/mean/sd/mx belong to   */
/* the j-th ELT of the layer (layer order = summation order); elt_handle[j] is its global     */
/* handle, which keys its uniforms.  terms[4] = (OccR, OccL, AggR, AggL).                      */
/* trials[n_sel]: the trials to evaluate -> ylt[n_sel].                                        */
/* Returns 0, or -1 (bad input), -2 (duplicate id), and sets *not_conv to the number of        */
/* inversions that hit the iteration cap.                                                      */
/* ------------------------------------------------------------------------------------------ */
typedef struct {
  int64_t trial, k, rec;
  int32_t j;
  double u, x, loss;
} ora_hit;

static int run_impl(const int64_t *yet_offsets, const int32_t *yet_ids, int32_t n_elts,
                    const int64_t *elt_off, const int32_t *ids, const double *mean,
                    const double *sd, const double *sdc, const double *mx,
                    const int32_t *elt_handle,
                    const double *terms, uint64_t seed, const int64_t *trials, int64_t n_sel,
                    double *ylt, double *oep, double *olt, double *inc, ora_hit *hits,
                    int64_t max_hits, int64_t *n_hits, int64_t *not_conv, int n_threads) {
  /* per-occurrence outputs: the selected trials' occurrences, concatenated in selection order */
  int64_t *out_off = NULL;
  if (olt || inc) {
    out_off = (int64_t *)malloc(sizeof(int64_t) * (size_t)(n_sel + 1));
    if (!out_off) return -1;
    out_off[0] = 0;
    for (int64_t s = 0; s < n_sel; ++s)
      out_off[s + 1] = out_off[s] + yet_offsets[trials[s] + 1] - yet_offsets[trials[s]];
  }
  ora_index *ix = (ora_index *)calloc((size_t)(n_elts > 0 ? n_elts : 1), sizeof(ora_index));
  if (!ix) {
    free(out_off);
    return -1;
  }
  int rc = 0;
  for (int32_t j = 0; j < n_elts && rc == 0; ++j)
    rc = build_index(&ix[j], ids + elt_off[j], elt_off[j + 1] - elt_off[j]);
  int64_t nc = 0, nh = 0;
  if (rc == 0) {
#ifdef _OPENMP
    if (n_threads > 0) omp_set_num_threads(n_threads);
#else
    (void)n_threads;
#endif
#pragma omp parallel for schedule(dynamic, 16) reduction(+ : nc) if (hits == NULL)
    for (int64_t s = 0; s < n_sel; ++s) {
      int64_t i = trials[s];
      double S = 0.0;    /* cumulative occurrence loss, paper §2.3 */
      double omax = 0.0; /* the year's largest occurrence loss (event-level output) */
      for (int64_t q = yet_offsets[i]; q < yet_offsets[i + 1]; ++q) {
        int64_t k = q - yet_offsets[i];
        int32_t e = yet_ids[q];
        double l = 0.0; /* event loss summed over the layer's ELTs, Algorithm 1 */
        for (int32_t j = 0; j < n_elts; ++j) {
          int64_t r = lookup(&ix[j], e);
          if (r < 0) continue;
          int64_t g = elt_off[j] + r;
          double u = ora_su_uniform(seed, i, k, elt_handle[j]);
          int st = 0;
          /* paper §3.2: independent SD sd, correlated SD sdc (0 when not given) */
          const double sc = sdc ? sdc[g] : 0.0;
          if (sc > 0.0) u = ora_su_combine(u, ora_su_uniform_corr(seed, i, k), sd[g], sc);
          double loss = ora_su_loss(mean[g], sd[g] + sc, mx[g], u, &st);
          if (st == 1) nc += 1;
          l += loss;
          if (hits && nh < max_hits) {
            ora_hit *h = &hits[nh];
            h->trial = i; h->k = k; h->rec = r; h->j = j; h->u = u;
            h->x = (sd[g] + sc == 0.0) ? NAN : loss / mx[g];
            h->loss = loss;
          }
          if (hits) nh++;
        }
        const double o = ora_occ_terms(l, terms[0], terms[1]);
        /* Algorithm 1 applies the aggregate terms after every event: the year's net loss so far
         * before (A_prev) and after (A) this occurrence; the increment is its share of the YLT */
        const double A_prev = ora_agg_terms(S, terms[2], terms[3]);
        S += o;
        if (o > omax) omax = o;
        if (olt) olt[out_off[s] + k] = o;
        if (inc) inc[out_off[s] + k] = ora_agg_terms(S, terms[2], terms[3]) - A_prev;
      }
      ylt[s] = ora_agg_terms(S, terms[2], terms[3]);
      if (oep) oep[s] = omax;
    }
  }
  for (int32_t j = 0; j < n_elts; ++j) free_index(&ix[j]);
  free(ix);
  free(out_off);
  if (not_conv) *not_conv = nc;
  if (n_hits) *n_hits = nh;
  return rc;
}

ORA_API int ora_run(const int64_t *yet_offsets, const int32_t *yet_ids, int32_t n_elts,
                    const int64_t *elt_off, const int32_t *ids, const double *mean,
                    const double *sd, const double *sdc, const double *mx,
                    const int32_t *elt_handle, const double *terms, uint64_t seed,
                    const int64_t *trials, int64_t n_sel, double *ylt, double *oep,
                    int64_t *not_conv, int n_threads) {
  return run_impl(yet_offsets, yet_ids, n_elts, elt_off, ids, mean, sd, sdc, mx, elt_handle,
                  terms, seed, trials, n_sel, ylt, oep, NULL, NULL, NULL, 0, NULL, not_conv,
                  n_threads);
}

/* As ora_run, with the per-occurrence outputs of the selected trials (their occurrences
 * concatenated in selection order, sum of their lengths entries each): olt = the occurrence loss
 * after occurrence terms, inc = the increment of the year's net loss (aggregate terms applied to
 * the running sum) at that occurrence.  Any output may be NULL. */
ORA_API int ora_run_events(const int64_t *yet_offsets, const int32_t *yet_ids, int32_t n_elts,
                           const int64_t *elt_off, const int32_t *ids, const double *mean,
                           const double *sd, const double *sdc, const double *mx,
                           const int32_t *elt_handle, const double *terms, uint64_t seed,
                           const int64_t *trials, int64_t n_sel, double *ylt, double *oep,
                           double *olt, double *inc, int64_t *not_conv, int n_threads) {
  return run_impl(yet_offsets, yet_ids, n_elts, elt_off, ids, mean, sd, sdc, mx, elt_handle,
                  terms, seed, trials, n_sel, ylt, oep, olt, inc, NULL, 0, NULL, not_conv,
                  n_threads);
}

/* Same loop, single-threaded, additionally listing every hit (trial, event position k, layer
 * slot j, record index r in the caller's ELT order, the uniform z the inversion received, beta
 * quantile x, loss) in loop order; at most max_hits are written, the total is in *n_hits. */
ORA_API int ora_trace(const int64_t *yet_offsets, const int32_t *yet_ids, int32_t n_elts,
                      const int64_t *elt_off, const int32_t *ids, const double *mean,
                      const double *sd, const double *sdc, const double *mx,
                      const int32_t *elt_handle,
                      const double *terms, uint64_t seed, const int64_t *trials, int64_t n_sel,
                      double *ylt, int64_t max_hits, int64_t *hit_trial, int64_t *hit_k,
                      int32_t *hit_j, int64_t *hit_rec, double *hit_u, double *hit_x,
                      double *hit_loss, int64_t *n_hits) {
  ora_hit *hits = (ora_hit *)malloc(sizeof(ora_hit) * (size_t)(max_hits > 0 ? max_hits : 1));
  if (!hits) return -1;
  int64_t nh = 0, nc = 0;
  int rc = run_impl(yet_offsets, yet_ids, n_elts, elt_off, ids, mean, sd, sdc, mx, elt_handle,
                    terms, seed, trials, n_sel, ylt, NULL, NULL, NULL, hits, max_hits, &nh, &nc,
                    1);
  int64_t w = nh < max_hits ? nh : max_hits;
  for (int64_t h = 0; h < w; ++h) {
    hit_trial[h] = hits[h].trial; hit_k[h] = hits[h].k; hit_j[h] = hits[h].j;
    hit_rec[h] = hits[h].rec; hit_u[h] = hits[h].u; hit_x[h] = hits[h].x;
    hit_loss[h] = hits[h].loss;
  }
  free(hits);
  *n_hits = nh;
  return rc;
}

/* ------------------------------------------------------------------------------------------ */
/* YLT order and risk measures, paper §2.4.                                                    */
/* ------------------------------------------------------------------------------------------ */
static const double *g_rank_ylt;
static int cmp_rank(const void *x, const void *y) {
  int64_t i = *(const int64_t *)x, j = *(const int64_t *)y;
  double a = g_rank_ylt[i], b = g_rank_ylt[j];
  if (a > b) return -1;
  if (a < b) return 1;
  return (i > j) - (i < j);
}

/* order[r] = index of the r-th largest year loss (ties: smaller index first). */
ORA_API int ora_rank(const double *ylt, int64_t n, int64_t *order) {
  for (int64_t i = 0; i < n; ++i) order[i] = i;
  g_rank_ylt = ylt;
  qsort(order, (size_t)n, sizeof(int64_t), cmp_rank);
  return 0;
}

/* Number of tail trials for return period rp over n trials: n/rp, rounded up when it is not an
 * integer (an integer quotient within 1e-9 relative is taken as exact). */
ORA_API int64_t ora_tail_count(int64_t n, double rp) {
  double q = (double)n / rp;
  double r = nearbyint(q);
  int64_t k = (fabs(q - r) <= 1e-9 * fmax(1.0, q)) ? (int64_t)r : (int64_t)ceil(q);
  if (k < 1) k = 1;
  if (k > n) k = n;
  return k;
}

/* PML(rp) = year loss at rank k; TVaR(rp) = mean of ranks 1..k (summed in long double). */
ORA_API int ora_risk(const double *ylt, int64_t n, const double *rps, int32_t m, double *pml,
                     double *tvar) {
  if (n <= 0) return -1;
  for (int32_t q = 0; q < m; ++q)
    if (!(rps[q] > 1.0)) return -1;
  int64_t *order = (int64_t *)malloc(sizeof(int64_t) * (size_t)n);
  if (!order) return -1;
  ora_rank(ylt, n, order);
  for (int32_t q = 0; q < m; ++q) {
    int64_t k = ora_tail_count(n, rps[q]);
    long double s = 0.0L;
    for (int64_t r = 0; r < k; ++r) s += (long double)ylt[order[r]];
    pml[q] = ylt[order[k - 1]];
    tvar[q] = (double)(s / (long double)k);
  }
  free(order);
  return 0;
}
