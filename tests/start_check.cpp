// Host check of the start tables of the Newton-Halley inversion (the device code compiled for the
// host): over records drawn from the ELT value law, the table's estimate of ln x (of the tail the
// inversion solves) against the binary64-polished quantile.
#include <cmath>
#include <cstdio>
#include <random>

#include "ara_table.cuh"

int main() {
  using namespace ara;
  std::mt19937_64 rng(5);
  std::uniform_real_distribution<double> U(0.0, 1.0);
  double worst = 0.0, sum = 0.0;
  long n = 0, nan = 0;
  for (int rr = 0; rr < 300; ++rr) {
    const double s = 0.3 + 0.9 * U(rng), m = 3.0 + 7.0 * U(rng);  // sd/mean, max/mean
    const double k = (m - 1.0) / (s * s) - 1.0, a = k / m, b = (1.0 - 1.0 / m) * k;
    double lnB;
    const BetaRec br = ara_beta_rec_f64(a, b, &lnB);
    float st[kStartFloats];
    ara_build_start_record(br, st);
    for (int j = 0; j < 200; ++j) {
      const float u = (float)((std::floor(U(rng) * 16777216.0) + 0.5) / 16777216.0);
      double lnx, ln1mx;
      ara_exact_quantile_logs(a, b, u, &lnx, &ln1mx);
      const float L = ara_start_logit(st, u);
      if (!(L == L)) {
        ++nan;
        continue;
      }
      const bool flip = u > br.p0;
      const double exact = flip ? ln1mx : lnx;
      const double est = flip ? -std::log1p(std::exp((double)L)) : -std::log1p(std::exp(-(double)L));
      const double e = std::fabs(est - exact);
      if (std::isfinite(e)) {
        worst = std::fmax(worst, e);
        sum += e;
        ++n;
      }
    }
  }
  std::printf("%.6e %.6e %ld %ld\n", worst, sum / (double)n, n, nan);
  return 0;
}
