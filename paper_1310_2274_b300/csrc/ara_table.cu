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
                                    const double2* __restrict__ ab64, TableRec* trecs,
                                    float4* ivals, unsigned long long* n_uncertified) {
  const int64_t r = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (r >= n) return;
  const BetaRec br = recs[r];
  const double2 ab = ab64[r];
  TableRec tr;
  bool ok;
  ara_build_table_record(br, ab.x, ab.y, ivals + (int64_t)r * 4 * kTableIntervals, &tr, &ok);
  if (!ok) atomicAdd(n_uncertified, 1ull);
  trecs[r] = tr;
}

}  // namespace

cudaError_t launch_build_tables(int64_t n, const BetaRec* recs, const double2* ab64,
                                TableRec* trecs, float4* ivals,
                                unsigned long long* d_uncertified, cudaStream_t st) {
  if (n == 0) return cudaSuccess;
  const int threads = 128;
  build_tables_kernel<<<(unsigned)((n + threads - 1) / threads), threads, 0, st>>>(
      n, recs, ab64, trecs, ivals, d_uncertified);
  count_launches(1);
  return cudaGetLastError();
}

}  // namespace ara
