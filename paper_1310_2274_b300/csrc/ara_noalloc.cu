// ara_noalloc.cu -- PML / TVaR for callers that must not allocate device memory.
//
// ara_risk_measures() keeps its sort buffers in the context and grows them with cudaMalloc when
// a longer YLT arrives.  Some callers cannot allow that: code that runs inside a pre-sized
// memory pool or under another allocator that owns all device memory, real-time pricing loops
// that must not hit cudaMalloc's implicit device synchronisation or its failure under memory
// pressure, and callers that hold no ara_ctx at all.  ara_risk_measures_noalloc() serves them:
// it runs the same radix-sort and tail kernels on scratch that lives in a fixed file-scope
// device array, and takes its inputs and outputs from the caller.
//
// The scratch array is part of this module's device image, so every GPU that loads the library
// holds it (about 29 MB) until the process exits.  Calls share it and it keeps the last call's
// contents; everything that must start at zero is cleared at the start of each call.  Calls
// whose work overlaps on the GPU (on different streams, or from different host threads without
// ordering) race on the array and must not be made.
#include <cuda_runtime.h>
#include <math.h>
#include <stdint.h>

#include "../../include/ara.h"
#include "ara_internal.h"

namespace {

constexpr int64_t kMaxTrials = ARA_NOALLOC_MAX_TRIALS;
// sort buffers: two key and two index buffers, a digit histogram per 256 keys (at least as many
// as the sort's tiles need), the scan's tile sums, and four flag words
constexpr int64_t kHistWords = 256 * ((kMaxTrials + 255) / 256);
constexpr int64_t kScanWords = 4096;
constexpr size_t kKeysBytes = sizeof(uint64_t) * kMaxTrials;
constexpr size_t kValsBytes = sizeof(uint32_t) * kMaxTrials;
constexpr size_t kOffKeys0 = 0;
constexpr size_t kOffKeys1 = kOffKeys0 + kKeysBytes;
constexpr size_t kOffVals0 = kOffKeys1 + kKeysBytes;
constexpr size_t kOffVals1 = kOffVals0 + kValsBytes;
constexpr size_t kOffHist = kOffVals1 + kValsBytes;
constexpr size_t kOffScan = kOffHist + sizeof(uint32_t) * kHistWords;
constexpr size_t kOffFlags = kOffScan + sizeof(uint32_t) * kScanWords;
constexpr size_t kScratchBytes = kOffFlags + 256;

static __device__ __align__(256) unsigned char g_risk_scratch[kScratchBytes];

// Device address of g_risk_scratch on the current device.  In host code the array's name is only
// a host-side stand-in, never a device address.  The address is looked up on every call, not
// cached: a cudaDeviceReset (or any other teardown of the device's primary context) reloads the
// module, and an address kept from before it would point at freed memory.
cudaError_t scratch_for_current_device(unsigned char** out) {
  void* p = nullptr;
  const cudaError_t e = cudaGetSymbolAddress(&p, g_risk_scratch);
  if (e != cudaSuccess) return e;
  *out = static_cast<unsigned char*>(p);
  return cudaSuccess;
}

bool on_device(const void* p, int dev) {
  cudaPointerAttributes a;
  if (cudaPointerGetAttributes(&a, p) != cudaSuccess) {
    cudaGetLastError();
    return false;
  }
  return (a.type == cudaMemoryTypeDevice || a.type == cudaMemoryTypeManaged) && a.device == dev;
}

}  // namespace

extern "C" ara_status ara_risk_measures_noalloc(const double* ylt, int64_t n, const double* rps,
                                                int32_t m, double* pml, double* tvar,
                                                void* stream) {
  using namespace ara;
  if (n < 1 || n > kMaxTrials) return ARA_ERR_INVALID_ARG;
  if (m < 0 || m > kMaxTailCounts || (m > 0 && !rps)) return ARA_ERR_INVALID_ARG;
  if (!ylt || (m > 0 && (!pml || !tvar))) return ARA_ERR_INVALID_ARG;
  TailCounts ks{};
  for (int q = 0; q < m; ++q) {
    const double rp = rps[q];
    if (!(rp > 1.0) || !isfinite(rp)) return ARA_ERR_INVALID_ARG;
    // k = n / rp, rounded up when not an integer (an integer within 1e-9 relative is exact)
    const double x = (double)n / rp;
    const double r = nearbyint(x);
    int64_t k = (fabs(x - r) <= 1e-9 * fmax(1.0, x)) ? (int64_t)r : (int64_t)ceil(x);
    ks.k[q] = k < 1 ? 1 : (k > n ? n : k);
  }
  int dev = -1;
  if (cudaGetDevice(&dev) != cudaSuccess) {
    cudaGetLastError();
    return ARA_ERR_NO_DEVICE;
  }
  if (!on_device(ylt, dev) || (m > 0 && (!on_device(pml, dev) || !on_device(tvar, dev))))
    return ARA_ERR_INVALID_ARG;
  unsigned char* base = nullptr;
  if (scratch_for_current_device(&base) != cudaSuccess) {
    cudaGetLastError();
    return ARA_ERR_CUDA;
  }
  // the sort's own sizing must fit the fixed layout (holds for every n <= kMaxTrials)
  const int64_t hist_n = 256 * sort_tiles(n);
  if (hist_n > kHistWords || scan_tmp_words(hist_n) > kScanWords) return ARA_ERR_INVALID_ARG;
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  uint32_t* flags = reinterpret_cast<uint32_t*>(base + kOffFlags);
  const uint32_t* order = nullptr;
  cudaError_t e = sort_ylt_desc_no_sync(
      ylt, n, reinterpret_cast<uint64_t*>(base + kOffKeys0),
      reinterpret_cast<uint64_t*>(base + kOffKeys1), reinterpret_cast<uint32_t*>(base + kOffVals0),
      reinterpret_cast<uint32_t*>(base + kOffVals1), reinterpret_cast<uint32_t*>(base + kOffHist),
      reinterpret_cast<uint32_t*>(base + kOffScan), kScanWords, flags, &order, st);
  if (e == cudaSuccess)
    e = launch_tail_sums_flagged(ylt, order, ks, m, flags + 2, pml, tvar, st);
  if (e != cudaSuccess) {
    cudaGetLastError();
    return ARA_ERR_CUDA;
  }
  return ARA_OK;
}
