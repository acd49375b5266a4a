// ara_table.cu -- builds and certifies the per-record quantile tables (kTableSegments threads per
// record), builds the start tables, and gathers both into a layer's packed order; the
// construction itself is in ara_table.cuh.
#include <cuda_runtime.h>
#include <math.h>
#include <stdint.h>

#include "ara_internal.h"
#include "ara_table.cuh"

namespace ara {

namespace {

// Tables of the records of several ELTs in one launch.  A block takes 32 records; its warp w
// builds segment w (kTablePieces / kTableSegments pieces, a chain from its own first knot) of
// each of them, so a warp's lanes solve at nearby uniforms of 32 records (similar work) and a
// record's 129 inversions run as kTableSegments short chains.  A record keeps its table only if
// all its segments passed their checks (combined in shared memory); uncert[j] counts the
// records of job j that did not.
__global__ void __launch_bounds__(32 * kTableSegments) build_tables_kernel(
    const __grid_constant__ TableJobs J, unsigned long long* uncert) {
  constexpr int per = kTablePieces / kTableSegments;
  __shared__ unsigned int s_ok[kTableSegments];
  const int lane = threadIdx.x & 31, seg = threadIdx.x >> 5;
  const int64_t g = (int64_t)blockIdx.x * 32 + lane;
  const bool valid = g < J.first[J.n];
  int j = 0;
  if (valid) {  // the job holding record g: the last whose first record is <= g
    int lo = 0, hi = J.n - 1;
    while (lo < hi) {
      const int mid = (lo + hi + 1) >> 1;
      if (J.first[mid] <= g) lo = mid; else hi = mid - 1;
    }
    j = lo;
  }
  bool ok = true;
  BetaRec br{};
  TablePiece* pc = nullptr;
  if (valid) {
    const int64_t r = g - J.first[j];
    br = J.recs[j][r];
    pc = J.tables[j] + r * kTablePieces;
    if (!(br.a > 0.0f))
      ara_table_fill(pc, seg * per, (seg + 1) * per, br.mx, kPieceMean);
    else
      ok = ara_build_table_pieces(br, seg * per, (seg + 1) * per, pc);
  }
  const unsigned failed = __ballot_sync(0xFFFFFFFFu, !ok);  // lanes of this segment that failed
  if (lane == 0) s_ok[seg] = failed;
  __syncthreads();
  unsigned any = 0u;
#pragma unroll
  for (int w = 0; w < kTableSegments; ++w) any |= s_ok[w];
  if (valid && (any >> lane & 1u)) {
    ara_table_fill(pc, seg * per, (seg + 1) * per, br.mx, kPieceNewton);
    if (seg == 0) atomicAdd(uncert + j, 1ull);
  }
}

__global__ void build_starts_kernel(int64_t n, const BetaRec* __restrict__ recs, float* starts) {
  const int64_t r = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (r >= n) return;
  ara_build_start_record(recs[r], starts + r * kStartFloats);
}

// Layer copy of the tables in packed order: one warp per packed record, 2 KB each.
__global__ void gather_tables_kernel(int64_t n, const TablePiece* const* __restrict__ src,
                                     TablePiece* __restrict__ dst) {
  const int64_t w = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  const int lane = threadIdx.x & 31;
  if (w >= n) return;
  const uint4* s = reinterpret_cast<const uint4*>(src[w]);
  uint4* d = reinterpret_cast<uint4*>(dst + w * kTablePieces);
#pragma unroll
  for (int i = 0; i < (int)(kTablePieces * sizeof(TablePiece) / 16 / 32); ++i)
    d[i * 32 + lane] = s[i * 32 + lane];
}

// Layer copy of the start tables in packed order: one thread per 16 bytes, 24 per record, so the
// warp's stores are contiguous.
__global__ void gather_starts_kernel(int64_t n, const float* const* __restrict__ src,
                                     float* __restrict__ dst) {
  constexpr int kParts = kStartFloats * (int)sizeof(float) / 16;
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n * kParts) return;
  const int64_t w = i / kParts;
  const int part = (int)(i - w * kParts);
  reinterpret_cast<uint4*>(dst)[i] = reinterpret_cast<const uint4*>(src[w])[part];
}
static_assert(kStartFloats * sizeof(float) % 16 == 0, "start tables copy in 16-byte parts");

// An ELT's tables copied out of a layer whose tables were built in its packed order: record r of
// the ELT in slot `slot` sits at packed position base(e) + (rank of the slot among e's mask bits),
// e its event.  One thread per 16 bytes, kParts per record; uncert counts the ELT's records whose
// table failed certification.
__global__ void unpack_tables_kernel(int64_t n, const int32_t* __restrict__ ids, int slot,
                                     int mask_words, const uint32_t* __restrict__ evt,
                                     const TablePiece* __restrict__ layer_tables,
                                     TablePiece* __restrict__ elt_tables,
                                     unsigned long long* uncert) {
  constexpr int kParts = kTablePieces * (int)sizeof(TablePiece) / 16;
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n * kParts) return;
  const int64_t r = i / kParts;
  const int part = (int)(i - r * kParts);
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
  const uint4* src =
      reinterpret_cast<const uint4*>(layer_tables + (int64_t)(base + rank) * kTablePieces);
  const uint4 v = src[part];
  reinterpret_cast<uint4*>(elt_tables + r * kTablePieces)[part] = v;
  if (part == kParts - 1 && v.w == kPieceNewton) atomicAdd(uncert, 1ull);  // piece 63's flag
}

}  // namespace

cudaError_t launch_gather_starts(int64_t n, const float* const* d_src, float* dst,
                                 cudaStream_t st) {
  if (n == 0) return cudaSuccess;
  const int threads = 256;
  const int64_t total = n * (kStartFloats * (int64_t)sizeof(float) / 16);
  gather_starts_kernel<<<(unsigned)((total + threads - 1) / threads), threads, 0, st>>>(n, d_src,
                                                                                       dst);
  count_launches(1);
  return cudaGetLastError();
}

cudaError_t launch_build_tables(const TableJobs& jobs, unsigned long long* d_uncert,
                                cudaStream_t st) {
  const int64_t n = jobs.first[jobs.n];
  if (n == 0) return cudaSuccess;
  build_tables_kernel<<<(unsigned)((n + 31) / 32), 32 * kTableSegments, 0, st>>>(jobs, d_uncert);
  count_launches(1);
  return cudaGetLastError();
}

cudaError_t launch_build_starts(int64_t n, const BetaRec* recs, float* starts, cudaStream_t st) {
  if (n == 0) return cudaSuccess;
  const int threads = 128;
  build_starts_kernel<<<(unsigned)((n + threads - 1) / threads), threads, 0, st>>>(n, recs,
                                                                                  starts);
  count_launches(1);
  return cudaGetLastError();
}

cudaError_t launch_unpack_tables(int64_t n, const int32_t* ids, int slot, int mask_words,
                                 const uint32_t* evt, const TablePiece* layer_tables,
                                 TablePiece* elt_tables, unsigned long long* d_uncertified,
                                 cudaStream_t st) {
  if (n == 0) return cudaSuccess;
  const int threads = 256;
  const int64_t total = n * (kTablePieces * (int64_t)sizeof(TablePiece) / 16);
  unpack_tables_kernel<<<(unsigned)((total + threads - 1) / threads), threads, 0, st>>>(
      n, ids, slot, mask_words, evt, layer_tables, elt_tables, d_uncertified);
  count_launches(1);
  return cudaGetLastError();
}

cudaError_t launch_gather_tables(int64_t n, const TablePiece* const* d_src, TablePiece* dst,
                                 cudaStream_t st) {
  if (n == 0) return cudaSuccess;
  const int threads = 256;
  gather_tables_kernel<<<(unsigned)((n * 32 + threads - 1) / threads), threads, 0, st>>>(
      n, d_src, dst);
  count_launches(1);
  return cudaGetLastError();
}

}  // namespace ara
