// ara_table.cu -- builds and certifies the per-record quantile tables when an ELT is staged
// (one thread per record; the construction itself is in ara_table.cuh).
#include <cuda_runtime.h>
#include <math.h>
#include <stdint.h>

#include "ara_internal.h"
#include "ara_table.cuh"

namespace ara {

namespace {

__global__ void build_tables_kernel(int64_t n, const BetaRec* __restrict__ recs,
                                    const double2* __restrict__ ab64, TablePiece* tables,
                                    unsigned long long* n_uncertified) {
  const int64_t r = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (r >= n) return;
  const BetaRec br = recs[r];
  const double2 ab = ab64[r];
  bool ok;
  ara_build_table_record(br, ab.x, ab.y, tables + r * kTablePieces, &ok);
  if (!ok) atomicAdd(n_uncertified, 1ull);
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

cudaError_t launch_build_tables(int64_t n, const BetaRec* recs, const double2* ab64,
                                TablePiece* tables, unsigned long long* d_uncertified,
                                cudaStream_t st) {
  if (n == 0) return cudaSuccess;
  const int threads = 128;
  build_tables_kernel<<<(unsigned)((n + threads - 1) / threads), threads, 0, st>>>(
      n, recs, ab64, tables, d_uncertified);
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
