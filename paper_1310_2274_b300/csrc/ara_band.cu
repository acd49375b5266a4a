// ara_band.cu -- band-major schedule of Algorithm 1 for the certified-table inversion.
//
// The work of one run is the same as in the trial-major kernel (for every trial, every event in
// order, every ELT of the layer holding it: Philox uniform, table quantile, loss; per-event sum,
// occurrence terms; year sum, aggregate terms), but it is visited band by band: the catalogue is
// cut into bands of W = 2^log2w events, the YET is stored band-major (each trial's occurrences of
// band b together), and a launch sweeps the bands in order.  While the blocks of band b run they
// touch only band b's lookup entries, record headers and table pieces, which fit in L2, so each
// table piece comes from DRAM about once per launch instead of once per hit.
//
// Summation order (paper §2.3, reading G16): an event's ELT losses are summed in binary32 by a
// segmented warp scan over a round of hits that never splits an event except at multiples of 32
// hits from its first, exactly as in the trial-major kernel, so event losses are bit-identical in
// both schedules.  Year sums are exact integer sums of grid units (see AccExact), so the order in
// which bands and occurrences reach a trial's sum does not matter: both schedules, any trial
// range and any batch give the same year losses, bit for bit.
#include <cuda_runtime.h>
#include <stdint.h>

#include <algorithm>
#include <cmath>

#include "ara_ibeta.cuh"
#include "ara_internal.h"
#include "ara_philox.cuh"
#include "ara_trial_common.cuh"

namespace ara {

namespace {

// Warps per block.  The warps of a block share nothing but its slot on the SM, which is freed
// only when the slowest of them ends; with work per trial tile uneven, 2-warp blocks (16 per SM)
// waste least of it (8-warp blocks took 14.36 ms, 4-warp 14.01, 2-warp 13.83, 1-warp 14.24).
constexpr int kBW = 2;
constexpr int kT = 32;               // trials per warp
constexpr int kV = 4;                // positions per lane per chunk
constexpr int kCh = 32 * kV;         // positions per chunk
constexpr int kTrialsPerBlock = kBW * kT;
constexpr int kHitCap = 512;         // hits per chunk mapped to their positions in shared memory

constexpr int kStageWarps = 8;       // warps per block of the bucketing kernels

// ---- staging: the band-major copy of a YET ---------------------------------------------------

// Occurrences per (band, trial): counts[b * N + i].  One warp per trial, counters in shared
// memory.
__global__ void band_count_kernel(const int32_t* __restrict__ ids,
                                  const int64_t* __restrict__ offsets, int64_t n_trials,
                                  int log2w, int n_bands, uint32_t* __restrict__ counts) {
  extern __shared__ uint32_t s_cnt[];
  const int lane = threadIdx.x & 31, wib = threadIdx.x >> 5;
  uint32_t* c = s_cnt + wib * n_bands;
  for (int b = lane; b < n_bands; b += 32) c[b] = 0u;
  __syncwarp();
  const int64_t i = (int64_t)blockIdx.x * kStageWarps + wib;
  if (i >= n_trials) return;
  const int64_t beg = offsets[i], end = offsets[i + 1];
  for (int64_t q = beg + lane; q < end; q += 32) atomicAdd(&c[ids[q] >> log2w], 1u);
  __syncwarp();
  for (int b = lane; b < n_bands; b += 32) counts[(int64_t)b * n_trials + i] = c[b];
}

// Scatter of each trial's occurrences into their bands, in occurrence order within a band.
__global__ void band_scatter_kernel(const int32_t* __restrict__ ids,
                                    const int64_t* __restrict__ offsets, int64_t n_trials,
                                    int log2w, int kbits, int n_bands,
                                    const uint32_t* __restrict__ off, uint32_t* __restrict__ occ) {
  extern __shared__ uint32_t s_cur[];
  const int lane = threadIdx.x & 31, wib = threadIdx.x >> 5;
  uint32_t* cur = s_cur + wib * n_bands;
  const int64_t i = (int64_t)blockIdx.x * kStageWarps + wib;
  if (i >= n_trials) return;
  for (int b = lane; b < n_bands; b += 32) cur[b] = off[(int64_t)b * n_trials + i];
  __syncwarp();
  const int64_t beg = offsets[i], end = offsets[i + 1];
  const uint32_t wmask = (1u << log2w) - 1u;
  const uint32_t below = (1u << lane) - 1u;
  for (int64_t q0 = beg; q0 < end; q0 += 32) {
    const int64_t q = q0 + lane;
    const bool v = q < end;
    const int32_t id = v ? ids[q] : 0;
    const int band = v ? (id >> log2w) : -1;
    const unsigned act = __ballot_sync(0xFFFFFFFFu, v);
    const unsigned peers = __match_any_sync(0xFFFFFFFFu, band) & act;
    if (v) {
      const uint32_t dst = cur[band] + (uint32_t)__popc(peers & below);
      occ[dst] = (((uint32_t)id & wmask) << kbits) | (uint32_t)(q - beg);
    }
    __syncwarp();
    if (v && (peers & below) == 0u) cur[band] += (uint32_t)__popc(peers);
    __syncwarp();
  }
}

// ---- the band kernel ---------------------------------------------------------------------------

struct BandWarpSmem {
  int32_t excl[kCh];          // hits before each position (chunk order)
  uint32_t base[kCh];         // record base of each position's event
  uint32_t mask[2][kCh];
  alignas(16) float lsum[kCh];  // the event's summed loss
  uint32_t k[kCh];            // occurrence position in its trial
  alignas(4) uint8_t t[kCh];  // warp-local trial of each position
  uint8_t hitev[kHitCap];     // position of each of the chunk's hits (when they fit)
  uint32_t off[kT + 1];       // segment starts of the warp's trials in this band
  unsigned long long ys[kT];  // year-sum units gathered by the warp
  unsigned int om[kT];        // bit patterns of the trials' largest occurrence losses in the band
};

__device__ __forceinline__ uint32_t ld_stream_u32(const uint32_t* p, unsigned long long pol) {
  uint32_t v;
  asm volatile("ld.global.nc.L1::no_allocate.L2::cache_hint.u32 %0, [%1], %2;"
               : "=r"(v) : "l"(p), "l"(pol));
  return v;
}

// Trials [i_rel0, i_rel0 + nt) of the launch item P in band `band`, by one warp: the band-major
// words of those trials are contiguous, and the warp walks them 128 at a time.
// CORR: the launch may carry correlated weights (paper §3.2; P.corr is still checked, since a
// batch mixes items); without them the draw is the hit's own uniform and the weight load and
// combination are compiled out.
// INV: 0 certified tables (Newton-Halley fallback for uncertified records), 1 Newton-Halley from
// the start tables, records and start tables kept in L2 like the table pieces.
template <int MW, bool CORR, int INV>
__device__ __forceinline__ void band_warp(const TrialParams& P, int band, int64_t i_rel0, int nt,
                                          int lane, BandWarpSmem& sm) {
  const L2Policies pol = L2Policies::make();
  const uint32_t kmask = (1u << P.kbits) - 1u;
  const int32_t ebase = band << P.log2w;
  const int64_t orow = (int64_t)band * P.yet_n + P.t0 + i_rel0;
  if (lane < nt) {
    sm.off[lane] = __ldg(P.boff + orow + lane);
    sm.ys[lane] = 0ull;
    sm.om[lane] = 0u;
  }
  if (lane == 0) sm.off[nt] = __ldg(P.boff + orow + nt);
  __syncwarp();
  const uint32_t beg = sm.off[0], end = sm.off[nt];
  const float qs = P.q_scale;
  const bool want_oep = P.omax != nullptr;
  unsigned int nc = 0, n_inv = 0, n_it = 0, n_cf = 0, n_tab = 0, n_hit = 0;

  // the band words are streamed one chunk ahead, so their DRAM latency overlaps a chunk's hits
  uint32_t wn[kV];
#pragma unroll
  for (int v = 0; v < kV; ++v) {
    const uint32_t q = beg + v * 32 + lane;
    wn[v] = q < end ? ld_stream_u32(P.bocc + q, pol.stream) : 0u;
  }
  int t_row = 0;  // trial of the next row's first position (nondecreasing along the band words)
  for (uint32_t c = beg; c < end; c += kCh) {
    // ---- look up the chunk's entries, lay out its hits ----------------------------------------
    uint32_t w[kV];
#pragma unroll
    for (int v = 0; v < kV; ++v) {
      w[v] = wn[v];
      const uint32_t q = c + kCh + v * 32 + lane;
      wn[v] = q < end ? ld_stream_u32(P.bocc + q, pol.stream) : 0u;
    }
    Entry<MW> en[kV];
#pragma unroll
    for (int v = 0; v < kV; ++v) {
      en[v].base = 0;
      en[v].m0 = 0;
      if constexpr (MW == 2) en[v].m1 = 0;
      if (c + v * 32 + lane < end)
        en[v] = Entry<MW>::load(P.evt, ebase + (int32_t)(w[v] >> P.kbits), pol.keep);
    }
    int32_t run = 0;
#pragma unroll
    for (int v = 0; v < kV; ++v) {
      const uint32_t q = c + v * 32 + lane;
      // trial of position q: the last whose segment starts at or before q, found by advancing
      // from the trial of the row's first position (segments are short, so a step or two)
      int t = t_row;
      if (q < end)
        while (t + 1 < nt && sm.off[t + 1] <= q) ++t;
      t_row = __shfl_sync(0xFFFFFFFFu, t, 31);
      {
        const uint32_t q31 = c + v * 32 + 31;  // the next row starts at the trial of lane 31
        if (q31 >= end) t_row = nt - 1;
      }
      const int cnt = en[v].count();
      int incl = cnt;
#pragma unroll
      for (int d = 1; d < 32; d <<= 1) {
        const int x = __shfl_up_sync(0xFFFFFFFFu, incl, d);
        if (lane >= d) incl += x;
      }
      const int idx = v * 32 + lane;
      const int e0 = run + incl - cnt;
      sm.excl[idx] = e0;
      sm.base[idx] = en[v].base;
      sm.mask[0][idx] = en[v].m0;
      if constexpr (MW == 2) sm.mask[1][idx] = en[v].m1;
      sm.lsum[idx] = 0.f;
      sm.k[idx] = w[v] & kmask;
      sm.t[idx] = (uint8_t)t;
      for (int j = 0; j < cnt && e0 + j < kHitCap; ++j) sm.hitev[e0 + j] = (uint8_t)idx;
      run += __shfl_sync(0xFFFFFFFFu, incl, 31);
    }
    __syncwarp();
    const bool mapped = run <= kHitCap;

    // ---- rounds of up to 32 hits that end on an event boundary -------------------------------
    for (int32_t r0 = 0; r0 < run;) {
      const int32_t g = r0 + lane;
      int ev = 0;  // event of hit g: the last position whose exclusive prefix is <= g
      if (g < run) {
        if (mapped) {
          ev = sm.hitev[g];
        } else {
#pragma unroll
          for (int step = kCh / 2; step >= 1; step >>= 1)
            if (sm.excl[ev + step] <= g) ev += step;
        }
      }
      // the round ends at r0 + 32 unless the event of hit r0 + 31 continues past it: then at that
      // event's first hit, or at r0 + 32 if it began at or before r0 (more than 32 hits left)
      int32_t r1 = min(run, r0 + 32);
      if (run > r0 + 32) {
        const int ev31 = __shfl_sync(0xFFFFFFFFu, ev, 31);
        const int32_t end31 = ev31 + 1 < kCh ? sm.excl[ev31 + 1] : run;
        if (end31 > r0 + 32) {
          const int32_t s31 = sm.excl[ev31];
          r1 = s31 > r0 ? s31 : r0 + 32;
        }
      }
      const bool has = g < r1;
      float loss = 0.f;
      int seg_start = lane;  // first lane of this hit's event in the round
      if (has) {
        const int nth = g - sm.excl[ev];
        seg_start = max(lane - nth, 0);
        int slot;
        if constexpr (MW == 1) {
          slot = nth_set_bit(sm.mask[0][ev], nth);
        } else {
          const uint32_t m0 = sm.mask[0][ev];
          const int c0 = __popc(m0);
          slot = nth < c0 ? nth_set_bit(m0, nth) : 32 + nth_set_bit(sm.mask[1][ev], nth - c0);
        }
        const uint32_t pos = sm.base[ev] + (uint32_t)nth;
        const int64_t trial = P.t0 + i_rel0 + sm.t[ev];
        const float u0 = su_uniform_rk(P.rk0, P.rk1, trial, sm.k[ev], P.handles[slot]);
        const float cc = (CORR && P.corr != nullptr) ? __ldg(P.corr + pos) : 0.0f;
        const SuDraw d =
            su_draw(u0, cc > 0.0f ? su_uniform_corr_rk(P.rk0, P.rk1, trial, sm.k[ev]) : 0.5f, cc);
        const float u = d.z;
        if constexpr (INV == 1) {
          const BetaRec rec = load_rec_policy(P.recs + pos, pol.keep);
          if (!(rec.a > 0.f)) {
            loss = rec.mx;  // sd = 0: the mean (primary uncertainty only)
          } else {
            const float sl = start_logit_policy(P.starts + (size_t)pos * kStartFloats, u, pol.keep);
            const IbetaResult ib = ara_inv_beta<true>(rec, u, sl);
            nc += ib.converged ? 0u : 1u;
            n_inv += 1u;
            n_it += (unsigned)ib.iters;
            n_cf += (unsigned)ib.cf_terms;
            loss = rec.mx * ib.x;
          }
        } else {
        float tau;
        const int kp = ara_table_piece_q(d.lower, d.q, &tau);
        const TablePiece pc = ara_load_piece<true>(P.tables + (size_t)pos * kTablePieces, kp);
        if (pc.flag == kPieceTable) {
          loss = pc.mx * ara_piece_x(pc, tau);
          n_tab += 1u;
        } else if (pc.flag == kPieceMean) {
          loss = pc.mx;  // sd = 0: the mean (primary uncertainty only)
        } else {
          const IbetaResult ib = newton_fallback<false>(P.recs + pos, u);
          nc += ib.converged ? 0u : 1u;
          n_inv += 1u;
          n_it += (unsigned)ib.iters;
          n_cf += (unsigned)ib.cf_terms;
          loss = pc.mx * ib.x;
        }
        }
      }
      // segmented inclusive scan: segments are the runs of equal ev, lanes seg_start .. lane
      const int seg = has ? ev : -1;
      float val = loss;
#pragma unroll
      for (int d = 1; d < 32; d <<= 1) {
        const float nv = __shfl_up_sync(0xFFFFFFFFu, val, d);
        if (lane - d >= seg_start) val += nv;
      }
      const int next_seg = __shfl_down_sync(0xFFFFFFFFu, seg, 1);
      if (has && (lane == 31 || next_seg != seg)) sm.lsum[ev] += val;
      __syncwarp();
      r0 = r1;
    }
    n_hit += (lane == 0) ? (unsigned)run : 0u;

    // ---- occurrence terms; exact year-sum units gathered per trial ----------------------------
    // lane l takes the chunk's positions 4l .. 4l+3, which mostly belong to one trial; their
    // event losses and trials come in one 16-byte and one 4-byte shared load
    static_assert(kV == 4, "a lane's positions are one float4 of lsum and one word of t");
    const float4 l4 = *reinterpret_cast<const float4*>(&sm.lsum[kV * lane]);
    const uint32_t t4 = *reinterpret_cast<const uint32_t*>(&sm.t[kV * lane]);
    const float lv[kV] = {l4.x, l4.y, l4.z, l4.w};
    unsigned long long acc = 0;
    float om = 0.f;
    int tc = -1;
#pragma unroll
    for (int j = 0; j < kV; ++j) {
      const int p = kV * lane + j;
      if (c + (uint32_t)p < end) {
        const int t = (int)((t4 >> (8 * j)) & 0xFFu);
        const float o = fminf(fmaxf(lv[j] - P.occ_ret, 0.f), P.occ_lim);
        if (t != tc) {
          if (tc >= 0) {
            atomicAdd(&sm.ys[tc], acc);
            if (want_oep && om > 0.f) atomicMax(&sm.om[tc], __float_as_uint(om));
          }
          acc = 0;
          om = 0.f;
          tc = t;
        }
        acc += AccExact::units(o, qs);
        om = fmaxf(om, o);
      }
    }
    if (tc >= 0) {
      atomicAdd(&sm.ys[tc], acc);
      if (want_oep && om > 0.f) atomicMax(&sm.om[tc], __float_as_uint(om));
    }
    __syncwarp();
  }

  if (lane < nt && sm.ys[lane] != 0ull) atomicAdd(P.ysum + i_rel0 + lane, sm.ys[lane]);
  // the maximum over bands: an integer maximum of non-negative binary32 patterns, order-free
  if (want_oep && lane < nt && sm.om[lane] != 0u) atomicMax(P.omax + i_rel0 + lane, sm.om[lane]);
  // work counters, one striped atomic each
  nc = __reduce_add_sync(0xFFFFFFFFu, nc);
  n_inv = __reduce_add_sync(0xFFFFFFFFu, n_inv);
  n_it = __reduce_add_sync(0xFFFFFFFFu, n_it);
  n_cf = __reduce_add_sync(0xFFFFFFFFu, n_cf);
  n_tab = __reduce_add_sync(0xFFFFFFFFu, n_tab);
  n_hit = __reduce_add_sync(0xFFFFFFFFu, n_hit);
  if (lane == 0) {
    unsigned long long* st =
        P.stats + ((blockIdx.x * kBW + (threadIdx.x >> 5)) & (kStatStripes - 1));
    if (nc) atomicAdd(P.not_conv, (unsigned long long)nc);
    if (n_inv) atomicAdd(st + 0 * kStatStripes, (unsigned long long)n_inv);
    if (n_it) atomicAdd(st + 1 * kStatStripes, (unsigned long long)n_it);
    if (n_cf) atomicAdd(st + 2 * kStatStripes, (unsigned long long)n_cf);
    if (n_hit) atomicAdd(st + 3 * kStatStripes, (unsigned long long)n_hit);
    if (n_tab) atomicAdd(st + 4 * kStatStripes, (unsigned long long)n_tab);
  }
}

template <int MW, bool CORR, int INV>
__device__ __forceinline__ void band_block(const TrialParams& P, int64_t local_block,
                                           BandWarpSmem* sms) {
  const int lane = threadIdx.x & 31, wib = threadIdx.x >> 5;
  const int band = (int)(local_block / P.tiles);
  const int64_t tile = local_block - (int64_t)band * P.tiles;
  const int64_t i_rel0 = tile * kTrialsPerBlock + (int64_t)wib * kT;
  const int64_t left = P.n - i_rel0;
  if (left <= 0) return;  // whole warp; no block-wide barrier in this kernel
  band_warp<MW, CORR, INV>(P, band, i_rel0, (int)min((int64_t)kT, left), lane, sms[wib]);
}

// 64 registers for 32 warps per SM (16 blocks of 2), as the trial-major path.
template <int INV>
constexpr int kBandBlocksPerSM = 32 / kBW;

template <int MW, bool CORR, int INV>
__global__ void __launch_bounds__(kBW * 32, kBandBlocksPerSM<INV>)
    band_kernel(const __grid_constant__ TrialParams P) {
  __shared__ BandWarpSmem s_w[kBW];
  band_block<MW, CORR, INV>(P, (int64_t)blockIdx.x, s_w);
}

template <int MW, bool CORR, int INV>
__global__ void __launch_bounds__(kBW * 32, kBandBlocksPerSM<INV>)
    band_batch_kernel(const TrialParams* __restrict__ items,
                      const int64_t* __restrict__ block_begin, int n_items) {
  __shared__ BandWarpSmem s_w[kBW];
  const int64_t b = blockIdx.x;
  int lo = 0, hi = n_items - 1;
  while (lo < hi) {  // last item whose first block is <= b
    const int mid = (lo + hi + 1) >> 1;
    if (block_begin[mid] <= b) lo = mid; else hi = mid - 1;
  }
  band_block<MW, CORR, INV>(items[lo], b - block_begin[lo], s_w);
}

// Year losses from the exact year sums: S = units x 2^e, then the aggregate terms.
__device__ __forceinline__ void finalize_one(const TrialParams& P, int64_t i) {
  const double S = (double)P.ysum[i] * P.q_unit;
  P.ylt[i] = fmin(fmax(S - P.agg_ret, 0.0), P.agg_lim);
  if (P.oep) P.oep[i] = (double)__uint_as_float(P.omax[i]);
}

__global__ void band_finalize_kernel(const __grid_constant__ TrialParams P) {
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i < P.n) finalize_one(P, i);
}

__global__ void band_finalize_batch_kernel(const TrialParams* __restrict__ items,
                                           const int64_t* __restrict__ trial_begin, int n_items,
                                           int64_t total) {
  const int64_t g = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (g >= total) return;
  int lo = 0, hi = n_items - 1;
  while (lo < hi) {
    const int mid = (lo + hi + 1) >> 1;
    if (trial_begin[mid] <= g) lo = mid; else hi = mid - 1;
  }
  finalize_one(items[lo], g - trial_begin[lo]);
}

template <int MW, int INV>
cudaError_t launch_band_t(const TrialParams& p0, cudaStream_t st) {
  TrialParams p = p0;
  p.tiles = (int32_t)band_tiles(p.n);
  const int64_t blocks = (int64_t)p.n_bands * p.tiles;
  if (blocks <= 0) return cudaSuccess;
  if (blocks > 0x7FFFFFFFll) return cudaErrorInvalidConfiguration;
  if ((p.oep == nullptr) != (p.omax == nullptr)) return cudaErrorInvalidValue;
  cudaError_t e = cudaMemsetAsync(p.ysum, 0, sizeof(unsigned long long) * (size_t)p.n, st);
  if (e != cudaSuccess) return e;
  if (p.omax) {
    e = cudaMemsetAsync(p.omax, 0, sizeof(unsigned int) * (size_t)p.n, st);
    if (e != cudaSuccess) return e;
  }
  if (p.corr != nullptr)
    band_kernel<MW, true, INV><<<(unsigned)blocks, kBW * 32, 0, st>>>(p);
  else
    band_kernel<MW, false, INV><<<(unsigned)blocks, kBW * 32, 0, st>>>(p);
  count_launches(1);
  e = cudaGetLastError();
  if (e != cudaSuccess) return e;
  band_finalize_kernel<<<(unsigned)((p.n + 255) / 256), 256, 0, st>>>(p);
  count_launches(1);
  return cudaGetLastError();
}

}  // namespace

int year_grid_exponent(double o_max, int64_t max_len) {
  // the largest possible year sum, max_len x o_max, must fit in 2^62 units, so that the 64-bit
  // integer sum (at most half a unit of rounding per occurrence on top) never wraps; the finest
  // grid is 2^-100, far below any binary32 occurrence result that matters
  const double top = o_max * (double)std::max<int64_t>(1, max_len);
  if (!(top > 0.0)) return -62;
  return std::max(-100, (int)std::ceil(std::log2(top)) - 62);
}

double occurrence_bound(float ev_bound, double occ_ret, double occ_lim) {
  // an event's binary32 loss sum exceeds the exact sum of its records' bounds by at most 64
  // roundings (2^-18 relative); OccR and OccL are rounded to binary32, and l - OccR once more
  const double l = (double)ev_bound * (1.0 + 0x1p-16);
  const double o = std::max(0.0, l - occ_ret * (1.0 - 0x1p-20)) * (1.0 + 0x1p-20);
  return std::min(o, occ_lim * (1.0 + 0x1p-20));
}

// Band width for a layer: the largest power of four (2^12 .. 2^18; even exponents only, so a YET
// needs few band-major copies) for which one band's lookup entries (16 B per event), record
// headers (16 B per record) and the part of the records' tables a band pass touches (about
// 1.25 KB of the 2 KB per record at paper-scale hit rates) stay within 80 MB of the 126 MB L2.
// (At the paper-scale layer: 2^15 events, 38 MB, took 13.86 ms; 2^16, 77 MB, 13.37 ms; 2^17,
// 154 MB, 14.15 ms.)
int choose_band_log2w(int64_t catalog, int64_t n_packed) {
  const double per_event = 16.0 + (double)n_packed / (double)catalog * (16.0 + 1280.0);
  int best = 12;
  for (int l = 12; l <= 18; l += 2)
    if ((double)((int64_t)1 << l) * per_event <= 80.0 * 1024 * 1024) best = l;
  // a band wider than the catalogue gains nothing: use the smallest width that covers it
  for (int l = 12; l <= best; l += 2)
    if (((int64_t)1 << l) >= catalog) return l;
  return best;
}

bool band_layout_fits(const YetDev& y, int log2w) {
  const int kbits = 32 - log2w;
  const int64_t bands = ((int64_t)y.catalog + ((int64_t)1 << log2w) - 1) >> log2w;
  return y.n_occ < ((int64_t)1 << 32) && y.max_len <= ((int64_t)1 << kbits) &&
         bands <= kMaxBands && bands * y.n_trials + 1 < ((int64_t)1 << 32);
}

int64_t band_tiles(int64_t n) { return (n + kTrialsPerBlock - 1) / kTrialsPerBlock; }

void free_band_variant(BandedYet& v) {
  if (v.occ) cudaFree(v.occ);
  if (v.off) cudaFree(v.off);
  v = BandedYet();
}

cudaError_t build_band_variant(const YetDev& y, int log2w, BandedYet& out, cudaStream_t st) {
  BandedYet v;
  v.log2w = log2w;
  v.kbits = 32 - log2w;
  v.n_bands = (int32_t)(((int64_t)y.catalog + ((int64_t)1 << log2w) - 1) >> log2w);
  const int64_t n_off = (int64_t)v.n_bands * y.n_trials + 1;
  uint32_t* counts = nullptr;
  uint32_t* tmp = nullptr;
  const int64_t tmp_words = scan_tmp_words(n_off);
  cudaError_t e;
  if ((e = cudaMalloc(&v.occ, sizeof(uint32_t) * (size_t)std::max<int64_t>(1, y.n_occ))) != cudaSuccess ||
      (e = cudaMalloc(&v.off, sizeof(uint32_t) * (size_t)n_off)) != cudaSuccess ||
      (e = cudaMalloc(&counts, sizeof(uint32_t) * (size_t)n_off)) != cudaSuccess ||
      (e = cudaMalloc(&tmp, sizeof(uint32_t) * (size_t)std::max<int64_t>(1, tmp_words))) != cudaSuccess) {
    cudaGetLastError();
    free_band_variant(v);
    if (counts) cudaFree(counts);
    if (tmp) cudaFree(tmp);
    return e;
  }
  const unsigned blocks = (unsigned)((y.n_trials + kStageWarps - 1) / kStageWarps);
  const size_t smem = sizeof(uint32_t) * (size_t)v.n_bands * kStageWarps;
  e = cudaMemsetAsync(counts, 0, sizeof(uint32_t) * (size_t)n_off, st);
  if (e == cudaSuccess && blocks > 0) {
    band_count_kernel<<<blocks, kStageWarps * 32, smem, st>>>(y.ids, y.offsets, y.n_trials, log2w,
                                                              v.n_bands, counts);
    count_launches(1);
    e = cudaGetLastError();
  }
  if (e == cudaSuccess) e = launch_exclusive_scan_u32(counts, v.off, n_off, tmp, tmp_words, st);
  if (e == cudaSuccess && blocks > 0) {
    band_scatter_kernel<<<blocks, kStageWarps * 32, smem, st>>>(
        y.ids, y.offsets, y.n_trials, log2w, v.kbits, v.n_bands, v.off, v.occ);
    count_launches(1);
    e = cudaGetLastError();
  }
  if (e == cudaSuccess) e = cudaStreamSynchronize(st);
  cudaFree(counts);
  cudaFree(tmp);
  if (e != cudaSuccess) {
    cudaGetLastError();
    free_band_variant(v);
    return e;
  }
  out = v;
  return cudaSuccess;
}

cudaError_t launch_band(const TrialParams& p, int mask_words, int precision, int inversion,
                        cudaStream_t st) {
  if (precision != 0) return cudaErrorInvalidValue;  // exact year sums only
  if (inversion == 1) {
    if (p.starts == nullptr) return cudaErrorInvalidValue;
    return mask_words == 1 ? launch_band_t<1, 1>(p, st) : launch_band_t<2, 1>(p, st);
  }
  if (inversion != 0) return cudaErrorInvalidValue;
  return mask_words == 1 ? launch_band_t<1, 0>(p, st) : launch_band_t<2, 0>(p, st);
}

cudaError_t launch_band_batch(const TrialParams* d_items, const int64_t* d_block_begin,
                              const int64_t* d_trial_begin, int n_items, int64_t total_blocks,
                              int64_t total_trials, int mask_words, bool corr, int precision,
                              cudaStream_t st) {
  if (precision != 0) return cudaErrorInvalidValue;
  if (total_blocks <= 0) return cudaSuccess;
  if (total_blocks > 0x7FFFFFFFll) return cudaErrorInvalidConfiguration;
  const dim3 grid((unsigned)total_blocks), block(kBW * 32);
  if (mask_words == 1) {
    if (corr)
      band_batch_kernel<1, true, 0><<<grid, block, 0, st>>>(d_items, d_block_begin, n_items);
    else
      band_batch_kernel<1, false, 0><<<grid, block, 0, st>>>(d_items, d_block_begin, n_items);
  } else {
    if (corr)
      band_batch_kernel<2, true, 0><<<grid, block, 0, st>>>(d_items, d_block_begin, n_items);
    else
      band_batch_kernel<2, false, 0><<<grid, block, 0, st>>>(d_items, d_block_begin, n_items);
  }
  count_launches(1);
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return e;
  band_finalize_batch_kernel<<<(unsigned)((total_trials + 255) / 256), 256, 0, st>>>(
      d_items, d_trial_begin, n_items, total_trials);
  count_launches(1);
  return cudaGetLastError();
}

}  // namespace ara
