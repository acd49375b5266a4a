// Host check of the certified quantile tables as staging builds them (the device code compiled
// for the host): over records drawn from the ELT value law, staged as ara_add_elt stages them,
// each table's x at uniforms of the grid against the binary64-polished quantile, beside the
// binary32 Newton-Halley inversion the tables are checked against.  Prints: records, records
// certified, then for the tables and for Newton-Halley the worst and the mean relative error of x
// (the loss is max_l x), over x >= 1e-12, then the worst of each over x >= 1e-4.
#include <cmath>
#include <cstdio>
#include <random>

#include "ara_table.cuh"

int main() {
  using namespace ara;
  std::mt19937_64 rng(11);
  std::uniform_real_distribution<double> U(0.0, 1.0);
  const int n_rec = 1500, n_u = 100;
  int certified = 0;
  double worst_t = 0.0, sum_t = 0.0, worst_n = 0.0, sum_n = 0.0, worst_t4 = 0.0, worst_n4 = 0.0;
  long n = 0;
  static TablePiece pc[kTablePieces];
  for (int rr = 0; rr < n_rec; ++rr) {
    const double s = 0.3 + 0.9 * U(rng), m = 3.0 + 7.0 * U(rng);  // sd/mean, max/mean
    const double k = (m - 1.0) / (s * s) - 1.0, a = k / m, b = (1.0 - 1.0 / m) * k;
    BetaRec br = ara_beta_rec_staged(a, b);
    bool ok;
    ara_build_table_record(br, pc, &ok);
    if (!ok) continue;
    ++certified;
    for (int j = 0; j < n_u; ++j) {
      const float u = (float)((2.0 * std::floor(U(rng) * 8388608.0) + 1.0) * 0x1p-24);
      double lnx, ln1mx;
      ara_exact_quantile_logs(a, b, u, &lnx, &ln1mx);
      if (!(lnx >= std::log(1e-12))) continue;
      float tau;
      const int kp = ara_table_piece(u, &tau);
      const double xt = ara_piece_x(pc[kp], tau);
      const double xn = ara_inv_beta(br, u).x;
      const double x = std::exp(lnx);
      const double et = std::fabs(xt - x) / x, en = std::fabs(xn - x) / x;
      worst_t = std::fmax(worst_t, et);
      worst_n = std::fmax(worst_n, en);
      if (x >= 1e-4) {
        worst_t4 = std::fmax(worst_t4, et);
        worst_n4 = std::fmax(worst_n4, en);
      }
      sum_t += et;
      sum_n += en;
      ++n;
    }
  }
  std::printf("%d %d %.6e %.6e %.6e %.6e %.6e %.6e\n", n_rec, certified, worst_t, sum_t / (double)n,
              worst_n, sum_n / (double)n, worst_t4, worst_n4);
  return 0;
}
