// ara_tscheck.cu -- the host-side check of a host-resident YET's timestamps (§2.1: each trial's
// occurrences in nondecreasing time order), run on host threads while the event ids cross PCIe.
// It reads every timestamp once; on a CPU with AVX2 eight at a time (compared with their
// predecessors through an overlapping load), else (or on other CPUs) with the scalar loop.
#include <stdint.h>
#if defined(__x86_64__)
#include <immintrin.h>
#endif

#include <algorithm>
#include <thread>
#include <vector>

namespace ara {
namespace {

// Flags of trials [a, b): 4 if a timestamp is NaN, 2 if one is below its predecessor in the same
// trial.
unsigned int check_trials_scalar(const int64_t* off, const float* ts, int64_t a, int64_t b) {
  unsigned int f = 0;
  for (int64_t i = a; i < b; ++i) {
    const int64_t s = off[i], e = off[i + 1];
    int nan = 0, dec = 0;
    for (int64_t q = s; q < e; ++q) nan |= (ts[q] != ts[q]);
    for (int64_t q = s + 1; q < e; ++q) dec |= (ts[q] < ts[q - 1]);
    f |= (nan ? 4u : 0u) | (dec ? 2u : 0u);
  }
  return f;
}

#if defined(__x86_64__)
__attribute__((target("avx2"))) unsigned int check_trials_avx2(const int64_t* off,
                                                               const float* ts, int64_t a,
                                                               int64_t b) {
  __m256 nan = _mm256_setzero_ps(), dec = _mm256_setzero_ps();
  int nan_s = 0, dec_s = 0;
  for (int64_t i = a; i < b; ++i) {
    const int64_t s = off[i], e = off[i + 1];
    if (s >= e) continue;
    nan_s |= (ts[s] != ts[s]);
    int64_t q = s + 1;
    for (; q + 8 <= e; q += 8) {
      const __m256 x = _mm256_loadu_ps(ts + q), prev = _mm256_loadu_ps(ts + q - 1);
      nan = _mm256_or_ps(nan, _mm256_cmp_ps(x, x, _CMP_UNORD_Q));
      dec = _mm256_or_ps(dec, _mm256_cmp_ps(x, prev, _CMP_LT_OQ));
    }
    for (; q < e; ++q) {
      nan_s |= (ts[q] != ts[q]);
      dec_s |= (ts[q] < ts[q - 1]);
    }
  }
  const bool any_nan = nan_s || _mm256_movemask_ps(nan) != 0;
  const bool any_dec = dec_s || _mm256_movemask_ps(dec) != 0;
  return (any_nan ? 4u : 0u) | (any_dec ? 2u : 0u);
}

#endif

}  // namespace

unsigned int validate_timestamps_host(const int64_t* off, const float* ts, int64_t n_trials);

unsigned int validate_timestamps_host(const int64_t* off, const float* ts, int64_t n_trials) {
  const int64_t n_occ = off[n_trials];
  // parts of at least 4M occurrences, cut at trial boundaries, one host thread each; one core is
  // left to the thread that waits on the GPU meanwhile
  const int64_t hw = std::max<int64_t>(1, (int64_t)std::thread::hardware_concurrency() - 1);
  const int64_t parts = std::max<int64_t>(1, std::min<int64_t>(hw, n_occ >> 22));
  std::vector<int64_t> cut((size_t)parts + 1, n_trials);
  cut[0] = 0;
  for (int64_t k = 1; k < parts; ++k) {
    const int64_t target = n_occ / parts * k;
    cut[(size_t)k] = std::upper_bound(off, off + n_trials + 1, target) - off - 1;
  }
#if defined(__x86_64__)
  static const bool avx2 = __builtin_cpu_supports("avx2");
#endif
  std::vector<unsigned int> flags((size_t)parts, 0u);
  auto check = [&](int64_t k) {
    const int64_t a = cut[(size_t)k], b = cut[(size_t)k + 1];
#if defined(__x86_64__)
    if (avx2) {
      flags[(size_t)k] = check_trials_avx2(off, ts, a, b);
      return;
    }
#endif
    flags[(size_t)k] = check_trials_scalar(off, ts, a, b);
  };
  std::vector<std::thread> pool;
  for (int64_t k = 1; k < parts; ++k) pool.emplace_back(check, k);
  check(0);
  for (auto& th : pool) th.join();
  unsigned int f = 0;
  for (unsigned int x : flags) f |= x;
  return f;
}

}  // namespace ara
