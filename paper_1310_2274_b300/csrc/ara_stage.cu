// ara_stage.cu -- staging kernels: YET validation, ELT record preparation, layer lookup build.
//
// The paper's preprocessing stage (§2.2) loads YET, XELTs and portfolio into memory; its §4.1
// chooses a direct-access table over compact forms for lookup speed.  A dense direct-access
// table of 16 ELTs over a 2,000,000-event catalogue would be 16x larger than the L2 cache, so
// here each layer gets one compact direct-access entry per catalogue event (record base + ELT bit
// mask, 8 or 16 bytes) and the event's records packed contiguously in layer order: one random
// read per occurrence plus one 32-byte sector per hit, all L2-resident at paper scale.
#include <cuda_runtime.h>
#include <math.h>
#include <stdint.h>

#include <algorithm>
#include <atomic>

#include "ara_internal.h"
#include "ara_table.cuh"

namespace ara {

namespace {

constexpr int kThreads = 256;

inline unsigned grid_for(int64_t n, int per_block = kThreads) {
  int64_t g = (n + per_block - 1) / per_block;
  if (g < 1) g = 1;
  if (g > 0x7FFFFFFF) g = 0x7FFFFFFF;
  return (unsigned)g;
}

// ---- YET validation (warp per trial) ----------------------------------------------------------
// flags bit 0: id out of range; bit 1: timestamp decreases within a trial; bit 2: NaN timestamp.
// Trials [t_begin, t_begin + n_trials); ids/ts hold occurrences from occ_base on (ts may be null).
__global__ void validate_yet_kernel(const int32_t* __restrict__ ids, const float* __restrict__ ts,
                                    int64_t occ_base, const int64_t* __restrict__ off,
                                    int64_t t_begin, int64_t n_trials, int32_t catalog,
                                    unsigned int* flags, int32_t* __restrict__ ids_out) {
  const int lane = threadIdx.x & 31;
  const int64_t warp = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  const int64_t nwarps = ((int64_t)gridDim.x * blockDim.x) >> 5;
  unsigned int f = 0;
  for (int64_t i = t_begin + warp; i < t_begin + n_trials; i += nwarps) {
    const int64_t beg = off[i] - occ_base, end = off[i + 1] - occ_base;
    // unrolled by 4: a lane keeps four groups of loads in flight (a memory-bound pass)
#pragma unroll 4
    for (int64_t q = beg + lane; q < end; q += 32) {
      const int32_t e = ids[q];
      if (ids_out != nullptr) ids_out[q] = e;  // the YET's device copy, made in the same pass
      if (e < 0 || e >= catalog) f |= 1u;
      if (ts != nullptr) {  // null: the timestamps are checked on the host
        const float t = ts[q];
        if (t != t) f |= 4u;
        if (q > beg && t < ts[q - 1]) f |= 2u;
      }
    }
  }
  f = __reduce_or_sync(0xFFFFFFFFu, f);
  if (lane == 0 && f) atomicOr(flags, f);
}

// Offsets: the longest trial by a maximum, the first decrease by a minimum over trial indices
// (both as 64-bit integer atomics on fields set by check_offsets_init).
__global__ void check_offsets_init(const int64_t* __restrict__ off, int64_t n_trials,
                                   OffsetCheck* out) {
  out->first = off[0];
  out->first_decrease = INT64_MAX;
  out->max_len = 0;
  out->last = off[n_trials];
}

__global__ void check_offsets_kernel(const int64_t* __restrict__ off, int64_t n_trials,
                                     OffsetCheck* out) {
  int64_t len_max = 0, dec = INT64_MAX;
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n_trials;
       i += (int64_t)gridDim.x * blockDim.x) {
    const int64_t len = off[i + 1] - off[i];
    if (len > len_max) len_max = len;
    if (len < 0 && i < dec) dec = i;
  }
  // lengths and indices are non-negative here, so unsigned maxima and minima order them
  unsigned long long lm = (unsigned long long)len_max, dm = (unsigned long long)dec;
#pragma unroll
  for (int d = 16; d >= 1; d >>= 1) {
    lm = max(lm, __shfl_xor_sync(0xFFFFFFFFu, lm, d));
    dm = min(dm, __shfl_xor_sync(0xFFFFFFFFu, dm, d));
  }
  if ((threadIdx.x & 31) == 0) {
    if (lm) atomicMax(reinterpret_cast<unsigned long long*>(&out->max_len), lm);
    if (dm != (unsigned long long)INT64_MAX)
      atomicMin(reinterpret_cast<unsigned long long*>(&out->first_decrease), dm);
  }
}

__global__ void check_offsets_fini(OffsetCheck* out) {
  if (out->first_decrease == INT64_MAX) out->first_decrease = -1;
}

// ---- ELT record preparation (FP64, once per record) --------------------------------------------

// One record of an ELT (job j of a launch): flags bit 3: id out of range; bit 4: mean <= 0 or an
// SD < 0 or non-finite; bit 5: max <= mean with sd > 0; bit 6: a duplicate event id (bit j of
// dup[e] marks event e as met in job j).  sdc (NULL: zero) is the correlated SD of paper §3.1:
// sigma = sd + sdc feeds the moments and corr[r] receives the normalised correlated weight of
// §3.2, (sdc/sigma) / |(sd, sdc)/sigma|.
__device__ __forceinline__ unsigned int prepare_record(const PrepJobs& J, int j, int64_t r,
                                                       int32_t catalog, unsigned int* dup) {
  unsigned int f = 0;
  const int32_t e = J.ids[j][r];
  if (J.ids_out[j]) J.ids_out[j][r] = e;
  const unsigned int bit = 1u << j;
  if (e < 0 || e >= catalog) {
    f |= 8u;
  } else if (atomicOr(&dup[e], bit) & bit) {
    f |= 64u;
  }
  const double* sdc = J.sdc[j];
  const double sd_i = J.sd[j][r], sd_c = sdc ? sdc[r] : 0.0;
  const double mu = J.mean[j][r], sigma = sd_i + sd_c, m = J.mx[j][r];
  if (J.corr[j]) {  // paper §3.2 steps 3-4: weights sd_i/sigma, sd_c/sigma, normalised
    const double wi = sigma > 0.0 ? sd_i / sigma : 1.0, wc = sigma > 0.0 ? sd_c / sigma : 0.0;
    J.corr[j][r] = (float)(wc / sqrt(wi * wi + wc * wc));
  }
  if (!(sd_i >= 0.0) || !(sd_c >= 0.0)) f |= 16u;
  BetaRec rec;
  rec.a = 0.f; rec.b = 0.f; rec.mx = (float)mu; rec.L0 = 0.f;
  rec.p0 = 0.5f; rec.lnx0 = 0.f; rec.lny0 = 0.f; rec.lns = 0.f;
  if (!(mu > 0.0) || !(sigma >= 0.0) || !isfinite(mu) || !isfinite(sigma)) {
    f |= 16u;
  } else if (sigma > 0.0) {
    if (!(m > mu) || !isfinite(m)) {
      f |= 32u;
    } else {
      // paper §3.3: sigma_beta = sigma/max, mu_beta = mu/max, clamp, alpha, beta
      const double mu_b = mu / m;
      double sig_b = sigma / m;
      const double sig_max = sqrt(mu_b * (1.0 - mu_b));
      if (sig_b > sig_max) sig_b = sig_max * (1.0 - 0x1p-20);
      const double rr = sig_max / sig_b;
      const double k = rr * rr - 1.0;
      const double a = mu_b * k, b = (1.0 - mu_b) * k;
      rec = ara_beta_rec_staged(a, b);
      rec.mx = (float)m;
      if (!(rec.a > 0.f) || !(rec.b > 0.f)) f |= 16u;  // alpha or beta outside binary32 range
    }
  }
  J.recs[j][r] = rec;
  return f;
}

// The records of up to kMaxPrepJobs ELTs in one launch (thread per record); flags[j] collects
// job j's flags.
__global__ void prepare_elts_kernel(const __grid_constant__ PrepJobs J, int32_t catalog,
                                    unsigned int* dup, unsigned int* flags) {
  const int64_t g = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (g >= J.first[J.n]) return;
  int lo = 0, hi = J.n - 1;
  while (lo < hi) {  // the job holding record g: the last whose first record is <= g
    const int mid = (lo + hi + 1) >> 1;
    if (J.first[mid] <= g) lo = mid; else hi = mid - 1;
  }
  const unsigned int f = prepare_record(J, lo, g - J.first[lo], catalog, dup);
  if (f) atomicOr(flags + lo, f);
}

// ---- layer lookup structure ----------------------------------------------------------------------
__global__ void layer_mask_kernel(int64_t n, const int32_t* __restrict__ ids, int slot,
                                  int mask_words, uint32_t* mask) {
  const int64_t r = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (r >= n) return;
  const int32_t e = ids[r];
  atomicOr(&mask[(int64_t)e * mask_words + (slot >> 5)], 1u << (slot & 31));
}

__global__ void layer_counts_kernel(const uint32_t* __restrict__ mask, int mask_words,
                                    int64_t catalog, uint32_t* cnt) {
  const int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (e >= catalog) return;
  uint32_t c = __popc(mask[e * mask_words]);
  if (mask_words == 2) c += __popc(mask[e * mask_words + 1]);
  cnt[e] = c;
}

// Entry layout: mask_words == 1 -> (base, mask) 8 bytes; == 2 -> (base, mask_lo, mask_hi, 0).
__global__ void layer_index_kernel(const uint32_t* __restrict__ mask,
                                   const uint32_t* __restrict__ base, int mask_words,
                                   int64_t catalog, uint32_t* evt) {
  const int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (e >= catalog) return;
  if (mask_words == 1) {
    reinterpret_cast<uint2*>(evt)[e] = make_uint2(base[e], mask[e]);
  } else {
    reinterpret_cast<uint4*>(evt)[e] = make_uint4(base[e], mask[2 * e], mask[2 * e + 1], 0u);
  }
}

__global__ void layer_scatter_kernel(int64_t n, const int32_t* __restrict__ ids,
                                     const BetaRec* __restrict__ recs,
                                     const TablePiece* __restrict__ tables, int slot,
                                     int mask_words, const uint32_t* __restrict__ evt,
                                     BetaRec* packed, const TablePiece** table_src,
                                     uint32_t* packed_rec, const float* __restrict__ corr,
                                     float* packed_corr, const float* __restrict__ starts,
                                     const float** start_src) {
  const int64_t r = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (r >= n) return;
  const int64_t e = ids[r];
  uint32_t base, rank;
  if (mask_words == 1) {
    const uint2 v = reinterpret_cast<const uint2*>(evt)[e];
    base = v.x;
    rank = __popc(v.y & ((1u << slot) - 1u));
  } else {
    const uint4 v = reinterpret_cast<const uint4*>(evt)[e];
    base = v.x;
    const uint64_t m = ((uint64_t)v.z << 32) | v.y;
    rank = __popcll(m & ((1ull << slot) - 1ull));
  }
  packed[base + rank] = recs[r];
  table_src[base + rank] = tables + r * kTablePieces;
  if (packed_corr) packed_corr[base + rank] = corr ? corr[r] : 0.0f;
  packed_rec[base + rank] = (uint32_t)r;
  if (start_src) start_src[base + rank] = starts + r * kStartFloats;  // copied by gather_starts
}

// The largest loss an event of the layer can bring before occurrence terms: over catalogue events,
// the sum of the event's records' loss bounds (the support bound max_l with sd > 0, the mean with
// sd = 0: packed[].mx holds exactly that), summed in binary64 and rounded up to binary32; the
// warp's maximum goes to *bound as an integer maximum of non-negative binary32 patterns.  It sizes
// the grid of the exact year sums (paper §2.3: o <= min(OccL, max(l - OccR, 0))).
__global__ void layer_event_bound_kernel(const uint32_t* __restrict__ evt, int mask_words,
                                         int64_t catalog, const BetaRec* __restrict__ packed,
                                         unsigned int* bound) {
  const int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  unsigned int b = 0u;
  if (e < catalog) {
    uint32_t base, cnt;
    if (mask_words == 1) {
      const uint2 v = reinterpret_cast<const uint2*>(evt)[e];
      base = v.x;
      cnt = __popc(v.y);
    } else {
      const uint4 v = reinterpret_cast<const uint4*>(evt)[e];
      base = v.x;
      cnt = __popc(v.y) + __popc(v.z);
    }
    double s = 0.0;
    for (uint32_t r = 0; r < cnt; ++r) s += (double)packed[base + r].mx;
    b = __float_as_uint(__double2float_ru(s));
  }
  b = __reduce_max_sync(0xFFFFFFFFu, b);
  if ((threadIdx.x & 31) == 0 && b != 0u) atomicMax(bound, b);
}

// ---- exclusive scan of uint32 (three passes: block sums, scan of sums, block scans) ----------
constexpr int kScanBlock = 1024;
constexpr int kScanItems = 8;  // per thread
constexpr int kScanTile = kScanBlock * kScanItems;

__device__ __forceinline__ uint32_t warp_incl_scan(uint32_t v) {
  const int lane = threadIdx.x & 31;
#pragma unroll
  for (int d = 1; d < 32; d <<= 1) {
    const uint32_t t = __shfl_up_sync(0xFFFFFFFFu, v, d);
    if (lane >= d) v += t;
  }
  return v;
}

// Block-wide exclusive scan of one value per thread; returns the exclusive prefix, *total = sum.
__device__ uint32_t block_excl_scan(uint32_t v, uint32_t* total) {
  __shared__ uint32_t warp_sums[32];
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const uint32_t incl = warp_incl_scan(v);
  if (lane == 31) warp_sums[warp] = incl;
  __syncthreads();
  if (warp == 0) {
    const int nw = blockDim.x >> 5;
    uint32_t s = lane < nw ? warp_sums[lane] : 0u;
    s = warp_incl_scan(s);
    if (lane < nw) warp_sums[lane] = s;
  }
  __syncthreads();
  const uint32_t warp_excl = warp == 0 ? 0u : warp_sums[warp - 1];
  *total = warp_sums[(blockDim.x >> 5) - 1];
  __syncthreads();
  return warp_excl + incl - v;
}

__global__ void scan_tile_sums_kernel(const uint32_t* __restrict__ in, int64_t n,
                                      uint32_t* sums) {
  const int64_t base = (int64_t)blockIdx.x * kScanTile;
  uint32_t s = 0;
#pragma unroll
  for (int k = 0; k < kScanItems; ++k) {
    const int64_t q = base + (int64_t)k * kScanBlock + threadIdx.x;
    if (q < n) s += in[q];
  }
  uint32_t total;
  block_excl_scan(s, &total);
  if (threadIdx.x == 0) sums[blockIdx.x] = total;
}

__global__ void scan_sums_kernel(uint32_t* sums, int64_t n_tiles) {
  // one block: exclusive scan of the tile sums in chunks of blockDim
  uint32_t carry = 0;
  for (int64_t c = 0; c < n_tiles; c += blockDim.x) {
    const int64_t q = c + threadIdx.x;
    const uint32_t v = q < n_tiles ? sums[q] : 0u;
    uint32_t total;
    const uint32_t ex = block_excl_scan(v, &total);
    if (q < n_tiles) sums[q] = carry + ex;
    carry += total;
  }
}

__global__ void scan_tiles_kernel(const uint32_t* __restrict__ in, int64_t n,
                                  const uint32_t* __restrict__ sums, uint32_t* out) {
  // each thread owns kScanItems consecutive elements of the tile
  const int64_t base = (int64_t)blockIdx.x * kScanTile + (int64_t)threadIdx.x * kScanItems;
  uint32_t v[kScanItems];
  uint32_t s = 0;
#pragma unroll
  for (int k = 0; k < kScanItems; ++k) {
    const int64_t q = base + k;
    v[k] = q < n ? in[q] : 0u;
    s += v[k];
  }
  uint32_t total;
  uint32_t ex = block_excl_scan(s, &total) + sums[blockIdx.x];
#pragma unroll
  for (int k = 0; k < kScanItems; ++k) {
    const int64_t q = base + k;
    if (q < n) out[q] = ex;
    ex += v[k];
  }
}

}  // namespace

namespace {
std::atomic<int64_t> g_launches{0};
}
void count_launches(int64_t n) { g_launches.fetch_add(n, std::memory_order_relaxed); }
int64_t launches_so_far() { return g_launches.load(std::memory_order_relaxed); }

cudaError_t launch_validate_yet_range(const int32_t* ids, const float* ts, int64_t occ_base,
                                      const int64_t* offsets, int64_t t_begin, int64_t n,
                                      int32_t catalog, unsigned int* d_flags, cudaStream_t st,
                                      int32_t* ids_out) {
  if (n == 0) return cudaSuccess;
  int64_t blocks = (n * 32 + kThreads - 1) / kThreads;
  if (blocks > 148 * 64) blocks = 148 * 64;
  validate_yet_kernel<<<(unsigned)blocks, kThreads, 0, st>>>(ids, ts, occ_base, offsets, t_begin,
                                                              n, catalog, d_flags, ids_out);
  count_launches(1);
  return cudaGetLastError();
}

cudaError_t launch_check_offsets(const int64_t* off, int64_t n_trials, OffsetCheck* out,
                                 cudaStream_t st) {
  check_offsets_init<<<1, 1, 0, st>>>(off, n_trials, out);
  if (n_trials > 0) {
    const int64_t blocks = std::min<int64_t>((n_trials + kThreads - 1) / kThreads, 148 * 8);
    check_offsets_kernel<<<(unsigned)blocks, kThreads, 0, st>>>(off, n_trials, out);
  }
  check_offsets_fini<<<1, 1, 0, st>>>(out);
  count_launches(n_trials > 0 ? 3 : 2);
  return cudaGetLastError();
}

cudaError_t launch_prepare_elts(const PrepJobs& jobs, int32_t catalog, unsigned int* d_dup,
                               unsigned int* d_flags, cudaStream_t st) {
  const int64_t n = jobs.first[jobs.n];
  if (n == 0) return cudaSuccess;
  prepare_elts_kernel<<<grid_for(n), kThreads, 0, st>>>(jobs, catalog, d_dup, d_flags);
  count_launches(1);
  return cudaGetLastError();
}

cudaError_t launch_layer_mask(const EltDev& e, int slot, int mask_words, uint32_t* d_mask,
                              cudaStream_t st) {
  if (e.n == 0) return cudaSuccess;
  layer_mask_kernel<<<grid_for(e.n), kThreads, 0, st>>>(e.n, e.ids, slot, mask_words, d_mask);
  count_launches(1);
  return cudaGetLastError();
}

cudaError_t launch_layer_counts(const uint32_t* d_mask, int mask_words, int64_t catalog,
                                uint32_t* d_cnt, cudaStream_t st) {
  layer_counts_kernel<<<grid_for(catalog), kThreads, 0, st>>>(d_mask, mask_words, catalog, d_cnt);
  count_launches(1);
  return cudaGetLastError();
}

int64_t scan_tmp_words(int64_t n) { return (n + kScanTile - 1) / kScanTile + 1; }

cudaError_t launch_exclusive_scan_u32(const uint32_t* in, uint32_t* out, int64_t n,
                                      uint32_t* d_tmp, int64_t tmp_words, cudaStream_t st) {
  if (n == 0) return cudaSuccess;
  const int64_t tiles = (n + kScanTile - 1) / kScanTile;
  if (tiles > tmp_words) return cudaErrorInvalidValue;
  scan_tile_sums_kernel<<<(unsigned)tiles, kScanBlock, 0, st>>>(in, n, d_tmp);
  scan_sums_kernel<<<1, kScanBlock, 0, st>>>(d_tmp, tiles);
  scan_tiles_kernel<<<(unsigned)tiles, kScanBlock, 0, st>>>(in, n, d_tmp, out);
  count_launches(3);
  return cudaGetLastError();
}

cudaError_t launch_layer_index(const uint32_t* d_mask, const uint32_t* d_base, int mask_words,
                               int64_t catalog, uint32_t* d_evt, cudaStream_t st) {
  layer_index_kernel<<<grid_for(catalog), kThreads, 0, st>>>(d_mask, d_base, mask_words, catalog,
                                                             d_evt);
  count_launches(1);
  return cudaGetLastError();
}

cudaError_t launch_layer_scatter(const EltDev& e, int slot, int mask_words,
                                 const uint32_t* d_evt, BetaRec* packed,
                                 const TablePiece** table_src, uint32_t* packed_rec,
                                 float* packed_corr, const float** start_src, cudaStream_t st) {
  if (e.n == 0) return cudaSuccess;
  layer_scatter_kernel<<<grid_for(e.n), kThreads, 0, st>>>(e.n, e.ids, e.recs, e.tables, slot,
                                                           mask_words, d_evt, packed, table_src,
                                                           packed_rec, e.corr, packed_corr,
                                                           e.starts, start_src);
  count_launches(1);
  return cudaGetLastError();
}

cudaError_t launch_layer_event_bound(const uint32_t* d_evt, int mask_words, int64_t catalog,
                                     const BetaRec* packed, unsigned int* d_bound,
                                     cudaStream_t st) {
  cudaError_t e = cudaMemsetAsync(d_bound, 0, sizeof(unsigned int), st);
  if (e != cudaSuccess || catalog == 0) return e;
  layer_event_bound_kernel<<<grid_for(catalog), kThreads, 0, st>>>(d_evt, mask_words, catalog,
                                                                   packed, d_bound);
  count_launches(1);
  return cudaGetLastError();
}

}  // namespace ara
