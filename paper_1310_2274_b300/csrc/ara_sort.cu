// ara_sort.cu -- ordering of the Year Loss Table and the PML / TVaR tail sums (paper §2.4).
//
// The trials are ordered by year loss descending, ties by ascending trial index.  Each loss is
// mapped to a 64-bit key whose unsigned order is the descending order of the loss
// (order-preserving bit pattern of the binary64 value, complemented), and the (key, index) pairs
// are sorted by a stable least-significant-digit radix sort, 8 bits per pass: stability keeps
// equal losses in index order, which is the tie rule.  Passes whose digit is the same for every
// key are skipped (found in one pre-pass).
//
// One pass = per-warp-tile digit histograms -> exclusive scan in (digit, tile) order -> stable
// scatter, where each warp walks its tile in order, 32 keys at a time, ranking equal digits with
// __match_any_sync against per-warp running counters.
#include <cuda_runtime.h>
#include <stdint.h>

#include "ara_internal.h"

namespace ara {

namespace {

constexpr int kSortWarps = 8;
constexpr int kSortItems = 16;                 // rounds of 32 keys per warp tile
constexpr int kTile = 32 * kSortItems;         // keys per warp tile

__device__ __forceinline__ uint64_t desc_key(double y) {
  if (y == 0.0) y = 0.0;  // one zero: -0 and +0 are the same loss
  const uint64_t u = (uint64_t)__double_as_longlong(y);
  const uint64_t ord = (u >> 63) ? ~u : (u | 0x8000000000000000ull);  // increasing in y
  return ~ord;                                                         // increasing in -y
}

__global__ void make_keys_kernel(const double* __restrict__ ylt, int64_t n, uint64_t* keys,
                                 uint32_t* vals, unsigned long long* varying,
                                 unsigned int* nan_flag) {
  __shared__ unsigned long long s_var;
  if (threadIdx.x == 0) s_var = 0ull;
  __syncthreads();
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  unsigned long long v = 0ull;
  if (i < n) {
    const double y = ylt[i];
    if (y != y) atomicOr(nan_flag, 1u);
    const uint64_t k = desc_key(y);
    keys[i] = k;
    vals[i] = (uint32_t)i;
    v = k ^ desc_key(ylt[0]);
  }
  v = __reduce_or_sync(0xFFFFFFFFu, (unsigned)(v & 0xFFFFFFFFull)) |
      ((unsigned long long)__reduce_or_sync(0xFFFFFFFFu, (unsigned)(v >> 32)) << 32);
  if ((threadIdx.x & 31) == 0 && v) atomicOr(&s_var, v);
  __syncthreads();
  if (threadIdx.x == 0 && s_var) atomicOr(varying, s_var);
}

__global__ void __launch_bounds__(kSortWarps * 32)
    hist_kernel(const uint64_t* __restrict__ keys, int64_t n, int shift, int64_t n_tiles,
                uint32_t* hist) {
  __shared__ uint32_t cnt[kSortWarps][256];
  const int lane = threadIdx.x & 31, wib = threadIdx.x >> 5;
  for (int d = lane; d < 256; d += 32) cnt[wib][d] = 0u;
  __syncwarp();
  const int64_t tile = (int64_t)blockIdx.x * kSortWarps + wib;
  if (tile >= n_tiles) return;
  const int64_t base = tile * kTile;
#pragma unroll 4
  for (int r = 0; r < kSortItems; ++r) {
    const int64_t i = base + r * 32 + lane;
    if (i < n) atomicAdd(&cnt[wib][(keys[i] >> shift) & 255u], 1u);
  }
  __syncwarp();
  for (int d = lane; d < 256; d += 32) hist[(int64_t)d * n_tiles + tile] = cnt[wib][d];
}

__global__ void __launch_bounds__(kSortWarps * 32)
    scatter_kernel(const uint64_t* __restrict__ kin, const uint32_t* __restrict__ vin, int64_t n,
                   int shift, int64_t n_tiles, const uint32_t* __restrict__ offs, uint64_t* kout,
                   uint32_t* vout) {
  __shared__ uint32_t run[kSortWarps][256];
  const int lane = threadIdx.x & 31, wib = threadIdx.x >> 5;
  const int64_t tile = (int64_t)blockIdx.x * kSortWarps + wib;
  if (tile >= n_tiles) return;
  for (int d = lane; d < 256; d += 32) run[wib][d] = offs[(int64_t)d * n_tiles + tile];
  __syncwarp();
  const uint32_t lt = (1u << lane) - 1u;
  const int64_t base = tile * kTile;
  for (int r = 0; r < kSortItems; ++r) {
    const int64_t i = base + r * 32 + lane;
    const bool valid = i < n;
    uint64_t k = 0;
    uint32_t v = 0;
    unsigned d = 256u;  // invalid lanes form their own group
    if (valid) {
      k = kin[i];
      v = vin[i];
      d = (unsigned)((k >> shift) & 255u);
    }
    const unsigned peers = __match_any_sync(0xFFFFFFFFu, d);
    const unsigned rank = __popc(peers & lt);
    if (valid) {
      const uint32_t dst = run[wib][d] + rank;
      kout[dst] = k;
      vout[dst] = v;
    }
    __syncwarp();
    if (valid && rank == 0) run[wib][d] += __popc(peers);
    __syncwarp();
  }
}

// One block per return period: pml = loss at rank k, tvar = mean of ranks 1..k (binary64; each
// thread sums a fixed strided subset, then a fixed tree: deterministic).
__global__ void tail_kernel(const double* __restrict__ ylt, const uint32_t* __restrict__ order,
                            const int64_t* __restrict__ ks, double* pml, double* tvar) {
  __shared__ double part[256];
  const int q = blockIdx.x;
  const int64_t k = ks[q];
  double s = 0.0;
  for (int64_t r = threadIdx.x; r < k; r += blockDim.x) s += ylt[order[r]];
  part[threadIdx.x] = s;
  __syncthreads();
  for (int h = blockDim.x / 2; h >= 1; h >>= 1) {
    if ((int)threadIdx.x < h) part[threadIdx.x] += part[threadIdx.x + h];
    __syncthreads();
  }
  if (threadIdx.x == 0) {
    pml[q] = ylt[order[k - 1]];
    tvar[q] = part[0] / (double)k;
  }
}

// As tail_kernel, with the tail counts passed by value and a NaN flag raised by the key pass:
// when it is set every output is NaN (the ordering of a YLT holding NaN is undefined).
__global__ void tail_kernel_flagged(const double* __restrict__ ylt,
                                   const uint32_t* __restrict__ order, const TailCounts ks,
                                   const unsigned int* __restrict__ nan_flag, double* pml,
                                   double* tvar) {
  __shared__ double part[256];
  const int q = blockIdx.x;
  const int64_t k = ks.k[q];
  double s = 0.0;
  for (int64_t r = threadIdx.x; r < k; r += blockDim.x) s += ylt[order[r]];
  part[threadIdx.x] = s;
  __syncthreads();
  for (int h = blockDim.x / 2; h >= 1; h >>= 1) {
    if ((int)threadIdx.x < h) part[threadIdx.x] += part[threadIdx.x + h];
    __syncthreads();
  }
  if (threadIdx.x == 0) {
    const bool bad = *nan_flag != 0u;
    pml[q] = bad ? __longlong_as_double(0x7FF8000000000000ll) : ylt[order[k - 1]];
    tvar[q] = bad ? __longlong_as_double(0x7FF8000000000000ll) : part[0] / (double)k;
  }
}

__global__ void order_to_i64_kernel(const uint32_t* __restrict__ o, int64_t n, int64_t* out) {
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i < n) out[i] = (int64_t)o[i];
}

// flags[order[r]] = 1 for the first k ranks (flags zeroed before).
__global__ void mark_top_kernel(const uint32_t* __restrict__ order, int64_t k, uint32_t* flags) {
  const int64_t r = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (r < k) flags[order[r]] = 1u;
}

// The marked entries in index order: out[pos[i]] = y[i] where flags[i] is set.
__global__ void compact_marked_kernel(const double* __restrict__ y, const uint32_t* __restrict__ flags,
                                      const uint32_t* __restrict__ pos, int64_t n, double* out) {
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i < n && flags[i]) out[pos[i]] = y[i];
}

}  // namespace

int64_t sort_tiles(int64_t n) { return (n + kTile - 1) / kTile; }

cudaError_t sort_ylt_desc(const double* d_ylt, int64_t n, SortScratch& s, int* which,
                          cudaStream_t st) {
  // s.digit_flags: [0..1] = varying-bit mask (64-bit), [2] = NaN flag
  unsigned long long* varying = reinterpret_cast<unsigned long long*>(s.digit_flags);
  unsigned int* nan_flag = s.digit_flags + 2;
  cudaError_t e = cudaMemsetAsync(s.digit_flags, 0, 4 * sizeof(uint32_t), st);
  if (e != cudaSuccess) return e;
  const unsigned blocks = (unsigned)((n + 255) / 256);
  make_keys_kernel<<<blocks, 256, 0, st>>>(d_ylt, n, s.keys[0], s.vals[0], varying, nan_flag);
  count_launches(1);
  if ((e = cudaGetLastError()) != cudaSuccess) return e;
  uint32_t flags[4];
  if ((e = cudaMemcpyAsync(flags, s.digit_flags, sizeof flags, cudaMemcpyDeviceToHost, st)) !=
      cudaSuccess)
    return e;
  if ((e = cudaStreamSynchronize(st)) != cudaSuccess) return e;
  if (flags[2]) return cudaErrorInvalidValue;  // NaN in the YLT
  const uint64_t var = (uint64_t)flags[0] | ((uint64_t)flags[1] << 32);
  const int64_t n_tiles = sort_tiles(n);
  const int64_t hist_n = 256 * n_tiles;
  const unsigned grid = (unsigned)((n_tiles + kSortWarps - 1) / kSortWarps);
  int cur = 0;
  for (int pass = 0; pass < 8; ++pass) {
    const int shift = 8 * pass;
    if (((var >> shift) & 255ull) == 0ull) continue;  // the same digit everywhere
    hist_kernel<<<grid, kSortWarps * 32, 0, st>>>(s.keys[cur], n, shift, n_tiles, s.hist);
    count_launches(1);
    if ((e = cudaGetLastError()) != cudaSuccess) return e;
    e = launch_exclusive_scan_u32(s.hist, s.hist, hist_n, s.scan_tmp, s.scan_cap, st);
    if (e != cudaSuccess) return e;
    scatter_kernel<<<grid, kSortWarps * 32, 0, st>>>(s.keys[cur], s.vals[cur], n, shift, n_tiles,
                                                     s.hist, s.keys[1 - cur], s.vals[1 - cur]);
    count_launches(1);
    if ((e = cudaGetLastError()) != cudaSuccess) return e;
    cur = 1 - cur;
  }
  *which = cur;
  return cudaSuccess;
}

cudaError_t launch_tail_sums(const double* d_ylt, const uint32_t* d_order, int64_t n,
                             const int64_t* d_k, int32_t m, double* d_pml, double* d_tvar,
                             cudaStream_t st) {
  (void)n;
  if (m == 0) return cudaSuccess;
  tail_kernel<<<m, 256, 0, st>>>(d_ylt, d_order, d_k, d_pml, d_tvar);
  count_launches(1);
  return cudaGetLastError();
}

cudaError_t sort_ylt_desc_no_sync(const double* d_ylt, int64_t n, uint64_t* keys0,
                                  uint64_t* keys1, uint32_t* vals0, uint32_t* vals1,
                                  uint32_t* hist, uint32_t* scan_tmp, int64_t scan_cap,
                                  uint32_t* flags4, const uint32_t** order, cudaStream_t st) {
  // flags4: [0..1] varying-bit mask (unused here), [2] NaN flag; all cleared first
  cudaError_t e = cudaMemsetAsync(flags4, 0, 4 * sizeof(uint32_t), st);
  if (e != cudaSuccess) return e;
  uint64_t* keys[2] = {keys0, keys1};
  uint32_t* vals[2] = {vals0, vals1};
  make_keys_kernel<<<(unsigned)((n + 255) / 256), 256, 0, st>>>(
      d_ylt, n, keys[0], vals[0], reinterpret_cast<unsigned long long*>(flags4), flags4 + 2);
  count_launches(1);
  if ((e = cudaGetLastError()) != cudaSuccess) return e;
  const int64_t n_tiles = sort_tiles(n);
  const int64_t hist_n = 256 * n_tiles;
  const unsigned grid = (unsigned)((n_tiles + kSortWarps - 1) / kSortWarps);
  int cur = 0;
  for (int pass = 0; pass < 8; ++pass) {  // every pass: no host round trip to skip any
    const int shift = 8 * pass;
    hist_kernel<<<grid, kSortWarps * 32, 0, st>>>(keys[cur], n, shift, n_tiles, hist);
    count_launches(1);
    if ((e = cudaGetLastError()) != cudaSuccess) return e;
    e = launch_exclusive_scan_u32(hist, hist, hist_n, scan_tmp, scan_cap, st);
    if (e != cudaSuccess) return e;
    scatter_kernel<<<grid, kSortWarps * 32, 0, st>>>(keys[cur], vals[cur], n, shift, n_tiles,
                                                     hist, keys[1 - cur], vals[1 - cur]);
    count_launches(1);
    if ((e = cudaGetLastError()) != cudaSuccess) return e;
    cur = 1 - cur;
  }
  *order = vals[cur];
  return cudaSuccess;
}

cudaError_t launch_tail_sums_flagged(const double* d_ylt, const uint32_t* d_order,
                                     const TailCounts& ks, int32_t m,
                                     const unsigned int* d_nan_flag, double* d_pml,
                                     double* d_tvar, cudaStream_t st) {
  if (m == 0) return cudaSuccess;
  tail_kernel_flagged<<<m, 256, 0, st>>>(d_ylt, d_order, ks, d_nan_flag, d_pml, d_tvar);
  count_launches(1);
  return cudaGetLastError();
}

cudaError_t launch_order_to_i64(const uint32_t* d_order, int64_t n, int64_t* d_out,
                                cudaStream_t st) {
  order_to_i64_kernel<<<(unsigned)((n + 255) / 256), 256, 0, st>>>(d_order, n, d_out);
  count_launches(1);
  return cudaGetLastError();
}

cudaError_t launch_top_k_in_index_order(const double* d_y, const uint32_t* d_order, int64_t n,
                                       int64_t k, uint32_t* flags, uint32_t* pos, uint32_t* tmp,
                                       int64_t tmp_words, double* d_out, cudaStream_t st) {
  cudaError_t e = cudaMemsetAsync(flags, 0, sizeof(uint32_t) * (size_t)n, st);
  if (e != cudaSuccess) return e;
  if (k > 0) {
    mark_top_kernel<<<(unsigned)((k + 255) / 256), 256, 0, st>>>(d_order, k, flags);
    count_launches(1);
    if ((e = cudaGetLastError()) != cudaSuccess) return e;
  }
  if ((e = launch_exclusive_scan_u32(flags, pos, n, tmp, tmp_words, st)) != cudaSuccess) return e;
  compact_marked_kernel<<<(unsigned)((n + 255) / 256), 256, 0, st>>>(d_y, flags, pos, n, d_out);
  count_launches(1);
  return cudaGetLastError();
}

}  // namespace ara
