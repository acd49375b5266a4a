// Host check of the host-resident YET's timestamp validation (the library's source compiled for
// the host): its flags against the plain definition (4: a NaN anywhere; 2: a timestamp below its
// predecessor in the same trial; a trial may start below the previous trial's end) on seeded
// YETs with a NaN or a decrease planted at random places, lengths that leave vector tails, empty
// trials, and YETs large enough to be cut across several threads.
#include <cmath>
#include <cstdint>
#include <cstdio>
#include <random>
#include <vector>

namespace ara {
unsigned int validate_timestamps_host(const int64_t* off, const float* ts, int64_t n_trials);
}

static unsigned int plain(const std::vector<int64_t>& off, const std::vector<float>& ts) {
  unsigned int f = 0;
  for (size_t i = 0; i + 1 < off.size(); ++i)
    for (int64_t q = off[i]; q < off[i + 1]; ++q) {
      if (std::isnan(ts[q])) f |= 4u;
      if (q > off[i] && ts[q] < ts[q - 1]) f |= 2u;
    }
  return f;
}

int main() {
  std::mt19937_64 rng(2024);
  int cases = 0, wrong = 0, flagged = 0;
  for (int c = 0; c < 400; ++c) {
    const bool big = c % 100 == 99;  // > 2^23 occurrences: several parts
    const int64_t n_trials = big ? 40000 : 1 + (int64_t)(rng() % 300);
    const int max_len = big ? 420 : (c % 3 == 0 ? 9 : 40);
    std::vector<int64_t> off(1, 0);
    for (int64_t i = 0; i < n_trials; ++i) off.push_back(off.back() + (int64_t)(rng() % (max_len + 1)));
    std::vector<float> ts((size_t)off.back());
    std::uniform_real_distribution<float> U(0.0f, 365.0f);
    for (int64_t i = 0; i < n_trials; ++i) {
      float t = U(rng) * 0.1f;  // each trial starts low: below the previous trial's end
      for (int64_t q = off[i]; q < off[i + 1]; ++q) {
        if (rng() % 4) t += U(rng) * 0.01f;  // else an equal timestamp (allowed)
        ts[q] = t;
      }
    }
    const int kind = c % 4;  // 0 clean, 1 a NaN, 2 a decrease, 3 both
    if (!ts.empty()) {
      if (kind & 1) ts[rng() % ts.size()] = NAN;
      if (kind & 2) {
        // a position that has a predecessor in its trial
        for (int tries = 0; tries < 1000; ++tries) {
          const int64_t i = (int64_t)(rng() % n_trials);
          if (off[i + 1] - off[i] < 2) continue;
          const int64_t q = off[i] + 1 + (int64_t)(rng() % (off[i + 1] - off[i] - 1));
          if (std::isnan(ts[q]) || std::isnan(ts[q - 1])) continue;
          ts[q] = ts[q - 1] - 0.5f;
          break;
        }
      }
    }
    const unsigned int want = plain(off, ts);
    const unsigned int got = ara::validate_timestamps_host(off.data(), ts.data(), n_trials);
    ++cases;
    wrong += got != want;
    flagged += want != 0;
  }
  printf("%d %d %d\n", cases, wrong, flagged);
  return 0;
}
