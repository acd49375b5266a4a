// Host check of the staging's ln Gamma (the device code compiled for the host) against the C
// library's lgamma over z in [1e-7, 2e5], log-uniform, and of ln B(a,b) over the ELT value law.
// Prints the worst |difference| / max(1, |lgamma(z)|), then the worst |difference| of ln B.
#include <cmath>
#include <cstdio>
#include <random>

#include "ara_table.cuh"

int main() {
  std::mt19937_64 rng(3);
  std::uniform_real_distribution<double> U(std::log(1e-7), std::log(2e5)), V(0.0, 1.0);
  double worst = 0.0, worst_b = 0.0;
  for (int i = 0; i < 1000000; ++i) {
    const double z = std::exp(U(rng));
    const double ref = std::lgamma(z);
    worst = std::fmax(worst, std::fabs(ara::ara_lngamma(z) - ref) / std::fmax(1.0, std::fabs(ref)));
  }
  for (int i = 0; i < 200000; ++i) {
    const double s = 0.3 + 0.9 * V(rng), m = 3.0 + 7.0 * V(rng);  // sd/mean, max/mean
    const double k = (m - 1.0) / (s * s) - 1.0, a = k / m, b = (1.0 - 1.0 / m) * k;
    const double mine = ara::ara_lngamma(a) + ara::ara_lngamma(b) - ara::ara_lngamma(a + b);
    const double ref = std::lgamma(a) + std::lgamma(b) - std::lgamma(a + b);
    worst_b = std::fmax(worst_b, std::fabs(mine - ref));
  }
  std::printf("%.6e %.6e\n", worst, worst_b);
  return 0;
}
