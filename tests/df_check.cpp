// Host check of the table build's double-float arithmetic (the device code compiled for the host,
// where the same binary32 operations run): error-free sum and product, and the continued fraction
// of DLMF 8.17.22 against a long-double evaluation of the same recurrence.
#include <cmath>
#include <cstdio>
#include <random>

#include "ara_table.cuh"

int main() {
  using namespace ara;
  std::mt19937_64 rng(12345);
  std::uniform_real_distribution<double> U(-1.0, 1.0);
  double worst_add = 0, worst_mul = 0;
  for (int i = 0; i < 200000; ++i) {
    const double x = U(rng) * std::ldexp(1.0, (int)(U(rng) * 20)), y = U(rng) * std::ldexp(1.0, (int)(U(rng) * 20));
    const DF a = df_from(x), b = df_from(y);
    const long double ea = (long double)a.hi + a.lo, eb = (long double)b.hi + b.lo;
    const DF s = df_add(a, b), p = df_mul(a, b);
    const long double rs = ea + eb, rp = ea * eb;
    // the sum's error is bounded relative to the operands (cancellation is exact but leaves
    // the operands' own rounding)
    worst_add = std::fmax(worst_add, (double)(std::fabs(((long double)s.hi + s.lo) - rs) /
                                              (std::fabs(ea) + std::fabs(eb))));
    worst_mul = std::fmax(worst_mul, (double)(std::fabs(((long double)p.hi + p.lo) - rp) / std::fabs(rp)));
  }
  double worst_cf = 0;
  for (int i = 0; i < 3000; ++i) {
    const double a = 0.1 + std::fabs(U(rng)) * 50, b = 0.1 + std::fabs(U(rng)) * 100;
    const double x = (0.001 + 0.998 * std::fabs(U(rng))) * (a + 1) / (a + b + 2);
    long double ap = (long double)a + b, Am2 = 1, Am1 = 1, Bm2 = 0, Bm1 = 1;
    for (int n = 1; n < 4000; n += 2) {
      const long double m = 0.5L * (n - 1);
      const long double al = (n == 1) ? -ap * x : -((long double)a + m) * (ap + m) * x;
      const long double be = (long double)a + n;
      long double A = be * Am1 + al * Am2, B = be * Bm1 + al * Bm2;
      Am2 = Am1; Bm2 = Bm1; Am1 = A; Bm1 = B;
      const long double m2 = m + 1, ale = m2 * ((long double)b - m2) * x, bee = (long double)a + n + 1;
      A = bee * Am1 + ale * Am2;
      B = bee * Bm1 + ale * Bm2;
      Am2 = Am1; Bm2 = Bm1; Am1 = A; Bm1 = B;
      const long double sc = 1.0L / std::fabs(Am1);
      Am1 *= sc; Am2 *= sc; Bm1 *= sc; Bm2 *= sc;
    }
    const double ref = (double)(Bm1 / Am1), got = ara_beta_cf_f64(a, b, x);
    worst_cf = std::fmax(worst_cf, std::fabs(got - ref) / std::fabs(ref));
  }
  std::printf("%.6e %.6e %.6e\n", worst_add, worst_mul, worst_cf);
  return 0;
}
