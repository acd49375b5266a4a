// Host check of the binary32 inversion (the device code compiled for the host) on records whose
// SD exceeds the largest a beta distribution with their mean allows: paper §3.3 clamps sigma_beta
// just below sigma_beta_max, which leaves alpha and beta near 1e-6.  Arguments: mean sd max step.
// Prints alpha, beta, whether the record's certified table was accepted, then one line per
// uniform of the grid u = (2i + 1) 2^-24, i = 0, step, 2 step, ..., and of a dense window around
// the jump of the quantile: u, x from the analytic start, x from the record's start table, and
// whether each converged.
#include <cmath>
#include <cstdio>
#include <cstdlib>

#include "ara_table.cuh"

int main(int argc, char** argv) {
  using namespace ara;
  if (argc != 5) return 2;
  const double mean = atof(argv[1]), sd = atof(argv[2]), mx = atof(argv[3]);
  const long step = atol(argv[4]);
  const double mu_b = mean / mx, sig_max = std::sqrt(mu_b * (1.0 - mu_b));
  double sig_b = sd / mx;
  if (sig_b > sig_max) sig_b = sig_max * (1.0 - 0x1p-20);
  const double r = sig_max / sig_b, k = r * r - 1.0, a = mu_b * k, b = (1.0 - mu_b) * k;
  double lnB;
  BetaRec br = ara_beta_rec_f64(a, b, &lnB);
  br.mx = (float)mx;
  static TablePiece pc[kTablePieces];
  bool ok;
  ara_build_table_record(br, pc, &ok);
  float st[kStartFloats];
  ara_build_start_record(br, st);
  std::printf("%.17g %.17g %d\n", a, b, (int)ok);
  // the grid, then every uniform within 3,000 grid points of p0 = I_{x0}, where the quantile
  // climbs from near 0 to near 1
  const long i0 = (long)((double)br.p0 * 0x1p23);
  for (long i = 0, j = 0; i < (1L << 23) || j <= 6000; i < (1L << 23) ? (i += step) : ++j) {
    const long g = i < (1L << 23) ? i : i0 - 3000 + j;
    const float u = (float)((2.0 * (double)g + 1.0) * 0x1p-24);
    const IbetaResult rn = ara_inv_beta<true>(br, u);
    const IbetaResult rs = ara_inv_beta<true>(br, u, ara_start_logit(st, u));
    std::printf("%.9g %.9g %.9g %d %d\n", u, rn.x, rs.x, (int)rn.converged, (int)rs.converged);
  }
  return 0;
}
