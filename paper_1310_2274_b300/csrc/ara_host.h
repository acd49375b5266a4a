// ara_host.h -- host-side helpers shared by the C-ABI implementation files: error detail,
// pointer kinds, plain and stream-ordered device allocation, grow-only context scratch.
#pragma once

#include <cuda_runtime.h>
#include <math.h>
#include <stdarg.h>
#include <stdio.h>

#include "../../include/ara.h"
#include "ara_ctx.h"
#include "ara_internal.h"

namespace ara {
inline ara_status fail(ara_ctx* c, ara_status s, const char* fmt, ...) {
  if (c) {
    char buf[512];
    va_list ap;
    va_start(ap, fmt);
    vsnprintf(buf, sizeof buf, fmt, ap);
    va_end(ap);
    c->detail = buf;
  }
  return s;
}

#define CUDA_TRY(ctx, call)                                                                   \
  do {                                                                                        \
    cudaError_t _e = (call);                                                                  \
    if (_e != cudaSuccess) {                                                                  \
      cudaGetLastError();                                                                     \
      return fail(ctx, _e == cudaErrorMemoryAllocation ? ARA_ERR_OOM : ARA_ERR_CUDA, "%s: %s", \
                  #call, cudaGetErrorString(_e));                                             \
    }                                                                                         \
  } while (0)

inline bool is_device_ptr(const void* p) {
  if (!p) return false;
  cudaPointerAttributes a;
  if (cudaPointerGetAttributes(&a, p) != cudaSuccess) {
    cudaGetLastError();
    return false;
  }
  return a.type == cudaMemoryTypeDevice || a.type == cudaMemoryTypeManaged;
}

// An address through which kernels can read caller memory in place: device and managed memory as
// they are, page-locked host memory mapped into the device's address space by its device alias;
// nullptr for pageable host memory (which must be copied first).
template <class T>
const T* device_readable(const T* p) {
  cudaPointerAttributes a;
  if (!p || cudaPointerGetAttributes(&a, p) != cudaSuccess) {
    cudaGetLastError();
    return nullptr;
  }
  if (a.type == cudaMemoryTypeDevice || a.type == cudaMemoryTypeManaged) return p;
  if (a.type == cudaMemoryTypeHost && a.devicePointer) return static_cast<const T*>(a.devicePointer);
  return nullptr;
}

template <class T>
cudaError_t dev_alloc(T** p, int64_t n) {
  *p = nullptr;
  if (n <= 0) n = 1;
  return cudaMalloc(reinterpret_cast<void**>(p), sizeof(T) * (size_t)n);
}

inline void dev_free(void* p) {
  if (p) cudaFree(p);
}

// Object memory: the device buffers of YETs, ELTs and layers come from the context's own
// memory pool, stream-ordered on its stream, and go back to it when freed.  The pool keeps up to
// kPoolKeepBytes of freed memory for the next staging: an analysis stages and frees ~10 GB in
// ~80 buffers, and a cudaMalloc / cudaFree pair of a multi-GB buffer costs milliseconds (cudaFree
// also waits for the whole device).  A buffer is freed only once no stream can still read it:
// the ara_free_* calls synchronise the device first, staging's own error paths free after
// synchronising the context's stream, the only one their work was on.
constexpr uint64_t kPoolKeepBytes = (uint64_t)32 << 30;

template <class T>
cudaError_t obj_alloc(ara_ctx* c, T** p, int64_t n) {
  *p = nullptr;
  if (n <= 0) n = 1;
  const size_t bytes = sizeof(T) * (size_t)n;
  cudaError_t e = cudaMallocFromPoolAsync(reinterpret_cast<void**>(p), bytes, c->pool, c->stream);
  if (e == cudaErrorMemoryAllocation) {  // hand back what the pool keeps, then try again
    cudaGetLastError();
    cudaStreamSynchronize(c->stream);
    cudaMemPoolTrimTo(c->pool, 0);
    e = cudaMallocFromPoolAsync(reinterpret_cast<void**>(p), bytes, c->pool, c->stream);
  }
  return e;
}

inline void obj_free(ara_ctx* c, const void* p) {
  if (p) cudaFreeAsync(const_cast<void*>(p), c->stream);
}

// Layer memory: object memory, or stream-ordered on st from the device's default pool (ordered:
// the serving loop builds and frees request layers while launches run, and never blocks).
template <class T>
cudaError_t mem_alloc(ara_ctx* c, T** p, int64_t n, bool ordered, cudaStream_t st) {
  if (!ordered) return obj_alloc(c, p, n);
  *p = nullptr;
  if (n <= 0) n = 1;
  return cudaMallocAsync(reinterpret_cast<void**>(p), sizeof(T) * (size_t)n, st);
}

inline void mem_free(ara_ctx* c, const void* p, bool ordered, cudaStream_t st) {
  if (!p) return;
  if (ordered) cudaFreeAsync(const_cast<void*>(p), st);
  else obj_free(c, p);
}

// A stream-ordered temporary freed when the call returns, on whichever path.
struct OrderedTemp {
  void* p;
  cudaStream_t st;
  ~OrderedTemp() {
    if (p) cudaFreeAsync(p, st);
  }
};

// Copies n elements from a host or device pointer into device memory on the stream.
template <class T>
cudaError_t copy_in(T* dst, const T* src, int64_t n, cudaStream_t st) {
  if (n <= 0) return cudaSuccess;
  return cudaMemcpyAsync(dst, src, sizeof(T) * (size_t)n, cudaMemcpyDefault, st);
}

inline void free_yet(ara_ctx* c, YetDev& y) {
  for (auto& v : y.bands) free_band_variant(v);
  obj_free(c, y.ids);
  obj_free(c, y.offsets);
  y = YetDev();
}
inline void free_elt(ara_ctx* c, EltDev& e) {
  obj_free(c, e.ids);
  obj_free(c, e.recs);
  obj_free(c, e.tables);
  obj_free(c, e.corr);
  obj_free(c, e.starts);
  e = EltDev();
}

// The table build of one ELT as a batch of one.
inline TableJobs one_job(const EltDev& e) {
  TableJobs j{};
  j.recs[0] = e.recs;
  j.tables[0] = e.tables;
  j.first[0] = 0;
  j.first[1] = e.n;
  j.n = 1;
  return j;
}

inline ara_status set_device(ara_ctx* c) {
  CUDA_TRY(c, cudaSetDevice(c->device));
  return ARA_OK;
}

inline ara_status ensure_ylt_tmp(ara_ctx* c, int64_t n) {
  if (n <= c->ylt_tmp_cap) return ARA_OK;
  dev_free(c->d_ylt_tmp);
  c->d_ylt_tmp = nullptr;
  c->ylt_tmp_cap = 0;
  CUDA_TRY(c, dev_alloc(&c->d_ylt_tmp, n));
  c->ylt_tmp_cap = n;
  return ARA_OK;
}

// Staging scratch: the temporaries of the staging calls (ELT and layer builds, table and start
// table packing) are carved from one device buffer the context keeps until ara_destroy (grown,
// never shrunk), so these calls free nothing: a cudaFree waits for the whole device, the copy
// stream included, and would hold staging back behind the ids a host-resident YET copies ahead.
// Each staging call synchronises its stream before it returns, so the buffer is idle between
// calls.  Pieces start on 256-byte boundaries.
template <class T>
constexpr size_t scratch_bytes(int64_t n) {
  return (sizeof(T) * (size_t)(n > 0 ? n : 1) + 255) / 256 * 256;
}

struct ScratchCarver {
  char* cur;
  template <class T>
  T* take(int64_t n) {
    T* p = reinterpret_cast<T*>(cur);
    cur += scratch_bytes<T>(n);
    return p;
  }
};

inline cudaError_t ensure_scratch(ara_ctx* c, size_t bytes) {
  if (bytes <= c->scratch_cap) return cudaSuccess;
  dev_free(c->d_scratch);
  c->d_scratch = nullptr;
  c->scratch_cap = 0;
  const size_t cap = bytes > ((size_t)64 << 20) ? bytes : ((size_t)64 << 20);
  const cudaError_t e = cudaMalloc(reinterpret_cast<void**>(&c->d_scratch), cap);
  if (e == cudaSuccess) c->scratch_cap = cap;
  return e;
}

inline ara_status ensure_ysum(ara_ctx* c, int64_t n) {
  if (n <= c->ysum_cap) return ARA_OK;
  dev_free(c->d_ysum);
  c->d_ysum = nullptr;
  c->ysum_cap = 0;
  CUDA_TRY(c, dev_alloc(&c->d_ysum, n));
  c->ysum_cap = n;
  return ARA_OK;
}

inline ara_status ensure_sort(ara_ctx* c, int64_t n) {
  SortScratch& s = c->sort;
  const int64_t tiles = sort_tiles(n);
  const int64_t hist_n = 256 * tiles;
  if (n > s.cap) {
    for (int b = 0; b < 2; ++b) {
      dev_free(s.keys[b]);
      dev_free(s.vals[b]);
      s.keys[b] = nullptr;
      s.vals[b] = nullptr;
    }
    s.cap = 0;
    for (int b = 0; b < 2; ++b) {
      CUDA_TRY(c, dev_alloc(&s.keys[b], n));
      CUDA_TRY(c, dev_alloc(&s.vals[b], n));
    }
    s.cap = n;
  }
  if (hist_n > s.hist_cap) {
    dev_free(s.hist);
    dev_free(s.scan_tmp);
    s.hist = nullptr;
    s.scan_tmp = nullptr;
    s.hist_cap = 0;
    CUDA_TRY(c, dev_alloc(&s.hist, hist_n));
    s.scan_cap = scan_tmp_words(hist_n);
    CUDA_TRY(c, dev_alloc(&s.scan_tmp, s.scan_cap));
    s.hist_cap = hist_n;
  }
  if (!s.digit_flags) CUDA_TRY(c, dev_alloc(&s.digit_flags, 4));
  return ARA_OK;
}

inline int64_t tail_count(int64_t n, double rp) {
  const double q = (double)n / rp;
  const double r = nearbyint(q);
  int64_t k = (fabs(q - r) <= 1e-9 * fmax(1.0, q)) ? (int64_t)r : (int64_t)ceil(q);
  if (k < 1) k = 1;
  if (k > n) k = n;
  return k;
}

// Timestamps of a host YET checked on host threads: bit 1 if they decrease within a trial, bit 2
// if one is NaN (the flags of the device check).  off: n_trials + 1 host offsets.
unsigned int validate_timestamps_host(const int64_t* off, const float* ts, int64_t n_trials);

}  // namespace ara
