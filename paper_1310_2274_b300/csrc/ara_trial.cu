// ara_trial.cu -- Algorithm 1 of the paper for one layer: one warp per trial.
//
// Per trial (paper §2.2, Algorithm 1; §2.3 terms; §3.3 secondary uncertainty):
//   for each event in timestamp order, for each ELT of the layer holding it:
//       u = Philox(trial, event position, ELT handle);  loss = max_l * InvCDF_beta(u; a, b)
//   l = sum of the event's losses (layer order), o = min(max(l - OccR, 0), OccL)
//   S = sum of o over the year;  YLT[trial] = min(max(S - AggR, 0), AggL)
//
// Schedule (designed for SIMT on sm_103a, not the paper's thread-per-trial):
//   * A warp walks its trial in chunks of 256 occurrences (128 on the surrogate path); lane l
//     reads occurrences c + 32v + l (v = 0..7, or 0..3), so each id load is one coalesced
//     128-byte line.
//   * Each occurrence reads its 8/16-byte lookup entry (record base + ELT mask); hits are counted
//     with popc and laid out in event order by a warp scan, giving the chunk's hit list.
//   * The hit list is processed in rounds of up to 32 hits, one hit per lane, so the inversion
//     (the time sink) runs with nearly every lane busy however sparse the hits are; a round ends
//     on an event boundary, so an event's ELT losses are summed the same way in every schedule.
//     A lane finds its hit's event by binary search of the chunk's hit prefix in shared memory
//     and its ELT by the n-th set bit of the mask.
//   * An event's losses (contiguous in the hit list) are summed by a segmented warp scan; the
//     tail lane adds the segment to the event's shared accumulator.  The order is fixed by the
//     data, so results do not depend on the launch configuration.
//   * Occurrence terms are applied per event in FP32; the year sum S is carried per lane exactly
//     in integer grid units (or Kahan-compensated FP32) and reduced across the warp at the end.
#include <cuda_runtime.h>
#include <stdint.h>

#include <algorithm>

#include "ara_ibeta.cuh"
#include "ara_internal.h"
#include "ara_mlp.cuh"
#include "ara_philox.cuh"
#include "ara_trial_common.cuh"

namespace ara {

namespace {

// Warps per block: 2 where a block's warps run independent trials (its slot on the SM is freed
// only when its slowest warp ends, so small blocks waste least of it), 4 for the surrogate path,
// whose blocks first load the network's weights into shared memory.
template <int INV>
constexpr int kWPB = INV == 2 ? 4 : 2;
// Occurrences per lane per chunk: 8 (the 8 index lookups a lane issues together hide each
// other's latency); 4 where the surrogate's network and segments already fill a block's shared
// memory.
template <int INV>
constexpr int kVOf = INV == 2 ? 4 : 8;
template <int INV>
constexpr int kChunkOf = 32 * kVOf<INV>;  // occurrences per chunk

// One 16-row tile of the network (tile mt of the warp's 32 rows: lane 16 mt + r holds row r's
// inputs); returns row g's output in *y0 and row g + 8's in *y8.  Out of line, so that the two
// tiles run one after the other and its registers do not add to the caller's.
__device__ __noinline__ void surrogate_tile(const MlpSmem& W, float z0, float z1, float z2,
                                            int mt, int lane, float* y0, float* y8) {
  const int g = lane >> 2, t = lane & 3;
  const float zc[3] = {z0, z1, z2};
  float zr0[3], zr8[3];
#pragma unroll
  for (int c = 0; c < 3; ++c) {
    zr0[c] = __shfl_sync(0xFFFFFFFFu, zc[c], mt * 16 + g);
    zr8[c] = __shfl_sync(0xFFFFFFFFu, zc[c], mt * 16 + g + 8);
  }
  mlp_tile_forward(W, zr0, zr8, g, t, y0, y8);
}

// Surrogate inference for 32 rows (one per lane): x from logit x = kOutScale * y; the rows are
// two 16-row MMA tiles (lane 16 m + r is row r of tile m).
__device__ __forceinline__ float surrogate_round(const MlpSmem& W, const float (&z)[3], int lane) {
  float a0, a8, b0, b8;
  surrogate_tile(W, z[0], z[1], z[2], 0, lane, &a0, &a8);
  surrogate_tile(W, z[0], z[1], z[2], 1, lane, &b0, &b8);
  // row r of tile m sits in lanes 4 (r mod 8) .. 4 (r mod 8) + 3, component r >= 8
  const int r = lane & 15, src = 4 * (r & 7);
  a0 = __shfl_sync(0xFFFFFFFFu, a0, src);
  a8 = __shfl_sync(0xFFFFFFFFu, a8, src);
  b0 = __shfl_sync(0xFFFFFFFFu, b0, src);
  b8 = __shfl_sync(0xFFFFFFFFu, b8, src);
  const float y = lane < 16 ? (r < 8 ? a0 : a8) : (r < 8 ? b0 : b8);
  return 1.0f / (1.0f + __expf(-kOutScale * y));
}

// ---- the learned surrogate's hits, a segment at a time ------------------------------------------
// Running the network in every round where any lane's hit is eligible costs a full 32-row pass
// per round (a minority of hits is eligible); instead the losses of a segment of up to kSegCap
// hits are computed ahead: pass A draws every hit and inverts the ineligible ones (Newton-Halley
// from the record's start table), listing the eligible ones; pass B runs the network over the
// list 32 rows at a time.  The rounds then read each hit's loss.
constexpr int kSegCap = 128;
struct SurrWarpSmem {
  float z[3][kSegCap];     // network inputs of the listed hits
  float mx[kSegCap];       // their loss scale
  uint8_t idx[kSegCap];    // their position in the segment
  float loss[kSegCap];     // every hit of the segment
};

// The exact inversion of a hit the network does not serve: Newton-Halley from the record's start
// table (analytic start without one), out of line so its registers do not add to the network's.
__device__ __noinline__ IbetaResult surrogate_fallback(const BetaRec* p, float u,
                                                       const float* start) {
  return ara_inv_beta<true>(load_rec(p), u, start ? ara_start_logit(start, u) : 1e30f);
}

// Losses of hits [s0, s1) of the chunk (s1 - s0 <= kSegCap) into sm.loss (and, with TRACE, x and
// u into tx, tu); hit(g) gives (packed record, slot, occurrence position) of hit g.
template <bool TRACE, bool CORR, class HitFn>
__device__ __forceinline__ void surrogate_segment(const TrialParams& P, const MlpSmem& W,
                                                  int64_t trial, int32_t s0, int32_t s1,
                                                  HitFn hit, SurrWarpSmem& sm, float* tx,
                                                  float* tu, int lane, unsigned int& nc,
                                                  unsigned int& n_inv, unsigned int& n_it,
                                                  unsigned int& n_cf, unsigned int& n_net) {
  const unsigned below = (1u << lane) - 1u;
  int n_list = 0;
  for (int32_t g0 = s0; g0 < s1; g0 += 32) {
    const int32_t g = g0 + lane;
    bool listed = false;
    float z0 = 0.f, z1 = 0.f, z2 = 0.f, mx = 0.f, u = 0.f;
    if (g < s1) {
      uint32_t pos, k;
      int slot;
      hit(g, &pos, &slot, &k);
      const BetaRec rec = load_rec(P.recs + pos);
      mx = rec.mx;
      const bool sd0 = !(rec.a > 0.f);
      if (!sd0 || TRACE) {
        const float cc = (CORR && P.corr != nullptr) ? __ldg(P.corr + pos) : 0.0f;
        u = su_draw(su_uniform_rk(P.rk0, P.rk1, trial, k, P.handles[slot]),
                    cc > 0.0f ? su_uniform_corr_rk(P.rk0, P.rk1, trial, k) : 0.5f, cc).z;
      }
      float l = mx, x = __int_as_float(0x7FC00000);
      if (!sd0) {
        // the network serves the hit if (alpha, beta) lies in its box and the certified error
        // in x of the hit's cell is within eps * mu_beta (mu_beta = alpha / (alpha + beta), the
        // record's mean over its maximum exposure): the served loss mx * x is then within eps
        // times the record's mean loss, so a year's sum of served losses is within eps of its
        // expectation whatever the hits' x
        if (rec.a >= kBoxLo && rec.a <= kBoxHi && rec.b >= kBoxLo && rec.b <= kBoxHi) {
          z0 = (logf(rec.a) - kLnCenter) / kLnHalf;
          z1 = (logf(rec.b) - kLnCenter) / kLnHalf;
          z2 = (logf(u) - log1pf(-u)) / kLogitScale;
          const int i0 = min(max((int)((z0 + 1.0f) * (0.5f * kCert0)), 0), kCert0 - 1);
          const int i1 = min(max((int)((z1 + 1.0f) * (0.5f * kCert1)), 0), kCert1 - 1);
          const int i2 = min(max((int)((z2 + 1.0f) * (0.5f * kCert2)), 0), kCert2 - 1);
          const float mu = rec.a / (rec.a + rec.b);
          listed = __ldg(P.mlp_bound + ((i0 * kCert1) + i1) * kCert2 + i2) <= P.mlp_eps * mu;
        }
        if (!listed) {
          const IbetaResult ib = surrogate_fallback(
              P.recs + pos, u, P.starts ? P.starts + (size_t)pos * kStartFloats : nullptr);
          nc += ib.converged ? 0u : 1u;
          n_inv += 1u;
          n_it += (unsigned)ib.iters;
          n_cf += (unsigned)ib.cf_terms;
          x = ib.x;
          l = mx * x;
        }
      }
      if (!listed) sm.loss[g - s0] = l;
      if constexpr (TRACE) {
        tx[g - s0] = x;
        tu[g - s0] = u;
      }
    }
    const unsigned m = __ballot_sync(0xFFFFFFFFu, listed);
    if (listed) {
      const int j = n_list + __popc(m & below);
      sm.z[0][j] = z0;
      sm.z[1][j] = z1;
      sm.z[2][j] = z2;
      sm.mx[j] = mx;
      sm.idx[j] = (uint8_t)(g - s0);
    }
    n_list += __popc(m);
  }
  __syncwarp();
  for (int j0 = 0; j0 < n_list; j0 += 32) {
    const int j = j0 + lane;
    const bool in = j < n_list;
    const float zz[3] = {in ? sm.z[0][j] : 0.f, in ? sm.z[1][j] : 0.f, in ? sm.z[2][j] : 0.f};
    const float xs = surrogate_round(W, zz, lane);
    if (in) {
      const int i = sm.idx[j];
      sm.loss[i] = sm.mx[j] * xs;
      if constexpr (TRACE) tx[i] = xs;
      n_net += 1u;
    }
  }
  __syncwarp();
}

// Per-occurrence outputs for 32 consecutive occurrences (lane l: position q), in trial order:
// the occurrence loss o after occurrence terms, and the increment of the year's net loss
// A(S) = min(max(S - AggR, 0), AggL) that o brings, Algorithm 1 applying the aggregate terms
// after every event.  S is the running year sum in exact grid units (an inclusive warp scan plus
// the carry of earlier groups), so the trial's last A is its YLT entry bit for bit.
__device__ __forceinline__ void occurrence_outputs(const TrialParams& P, int64_t q, int64_t end,
                                                   float o, int64_t q0,
                                                   unsigned long long& carry, int lane) {
  const bool in = q < end;
  if (P.olt != nullptr && in) P.olt[q - q0] = o;
  if (P.inc == nullptr) return;
  const unsigned long long un = in ? AccExact::units(o, P.q_scale) : 0ull;
  unsigned long long incl = un;
#pragma unroll
  for (int d = 1; d < 32; d <<= 1) {
    const unsigned long long t = __shfl_up_sync(0xFFFFFFFFu, incl, d);
    if (lane >= d) incl += t;
  }
  const unsigned long long s1 = carry + incl, s0 = s1 - un;
  carry += __shfl_sync(0xFFFFFFFFu, incl, 31);
  if (!in) return;
  // binary64 is slow on this part: below the retention and past the limit A is constant, so the
  // formula runs only for occurrences that cross into or lie inside the layer
  double d = 0.0;
  if (s1 > P.agg_zero_max && s0 < P.agg_full_min) {
    const double a1 = fmin(fmax((double)s1 * P.q_unit - P.agg_ret, 0.0), P.agg_lim);
    const double a0 = fmin(fmax((double)s0 * P.q_unit - P.agg_ret, 0.0), P.agg_lim);
    d = a1 - a0;
  }
  P.inc[q - q0] = d;
}

// The whole of Algorithm 1 for one trial (w-th of the launch item P), run by one warp.  CORR:
// the item may carry correlated weights (paper §3.2; P.corr is still checked); without them the
// weight load and the combination are compiled out.
template <int MW, class Acc, bool TRACE, int INV, bool CORR>
__device__ __forceinline__ void process_trial(const TrialParams& P, int64_t w, int lane, int wib,
                                              int32_t* excl, uint32_t* sbase,
                                              uint32_t (*s_maskw)[kChunkOf<INV>], float* lsum,
                                              const MlpSmem* s_mlp, SurrWarpSmem* s_surr,
                                              float* s_tx, float* s_tu) {
  constexpr bool TABLE = INV == 0;
  constexpr int kV = kVOf<INV>, kChunk = kChunkOf<INV>;
  constexpr bool SURR = INV == 2;
  const int64_t trial = P.t0 + w;
  if (P.abort_flag != nullptr && *reinterpret_cast<const volatile unsigned int*>(P.abort_flag))
    return;  // the streamed chunk holding this trial failed validation
  const int64_t beg = P.offsets[trial];
  const int64_t end = P.offsets[trial + 1];

  const L2Policies pol = L2Policies::make();
  Acc acc = Acc::make(P);
  float omax = 0.f;  // the year's largest occurrence loss (event-level output)
  // per-occurrence outputs: exact running year sum (grid units) of the occurrences before the
  // current group of 32, and the output index origin
  const bool evt = P.olt != nullptr || P.inc != nullptr;
  unsigned long long carry = 0ull;
  const int64_t q0 = evt ? P.offsets[P.t0] : 0;
  int32_t trace_n = 0;
  unsigned int nc = 0;
  unsigned int n_inv = 0, n_it = 0, n_cf = 0, n_hit = 0, n_tab = 0, n_net = 0;

  for (int64_t c = beg; c < end; c += kChunk) {
    // ---- stream ids, look up entries, lay out the chunk's hits in event order ---------------
    int32_t run = 0;
#pragma unroll
    for (int v = 0; v < kV; ++v) {
      const int64_t q = c + v * 32 + lane;
      Entry<MW> en;
      en.base = 0;
      en.m0 = 0;
      if constexpr (MW == 2) en.m1 = 0;
      if (q < end)
        en = Entry<MW>::load(P.evt, ld_stream_s32(P.ids + (q - P.occ_base), pol.stream), pol.keep);
      const int cnt = en.count();
      int incl = cnt;
#pragma unroll
      for (int d = 1; d < 32; d <<= 1) {
        const int t = __shfl_up_sync(0xFFFFFFFFu, incl, d);
        if (lane >= d) incl += t;
      }
      const int idx = v * 32 + lane;
      excl[idx] = run + incl - cnt;
      sbase[idx] = en.base;
      s_maskw[0][idx] = en.m0;
      if constexpr (MW == 2) s_maskw[1][idx] = en.m1;
      lsum[idx] = 0.f;
      run += __shfl_sync(0xFFFFFFFFu, incl, 31);
    }
    __syncwarp();

    // ---- rounds of up to 32 hits ending on an event boundary (an event with more than 32
    // hits left is split 32 hits from its first): uniform draw, inverse beta, per-event
    // segmented sum.  Rounds depend on the event's hits alone, so the FP32 event sums do too.
    int32_t seg0 = 0, seg1 = 0;  // surrogate: hits whose losses are computed ahead
    for (int32_t r0 = 0; r0 < run;) {
      if constexpr (SURR) {
        if (r0 + 32 > seg1 && seg1 < run) {  // the next round may need hits past the segment
          seg0 = r0;
          seg1 = min(run, r0 + kSegCap);
          const uint32_t kc = (uint32_t)(c - beg);
          auto hit = [&](int32_t gg, uint32_t* pos, int* slot, uint32_t* k) {
            int e = 0;
#pragma unroll
            for (int step = kChunk / 2; step >= 1; step >>= 1)
              if (excl[e + step] <= gg) e += step;
            const int nth = gg - excl[e];
            if constexpr (MW == 1) {
              *slot = nth_set_bit(s_maskw[0][e], nth);
            } else {
              const uint32_t m0 = s_maskw[0][e];
              const int c0 = __popc(m0);
              *slot = nth < c0 ? nth_set_bit(m0, nth) : 32 + nth_set_bit(s_maskw[1][e], nth - c0);
            }
            *pos = sbase[e] + (uint32_t)nth;
            *k = kc + (uint32_t)e;
          };
          surrogate_segment<TRACE, CORR>(P, *s_mlp, trial, seg0, seg1, hit, *s_surr, s_tx, s_tu,
                                         lane, nc, n_inv, n_it, n_cf, n_net);
        }
      }
      const int32_t g = r0 + lane;
      int ev = 0;  // event of hit g: the last position whose exclusive prefix is <= g
      if (g < run) {
#pragma unroll
        for (int step = kChunk / 2; step >= 1; step >>= 1)
          if (excl[ev + step] <= g) ev += step;
      }
      // the round ends at r0 + 32 unless the event of hit r0 + 31 continues past it: then at that
      // event's first hit, or at r0 + 32 if it began at or before r0 (more than 32 hits left)
      int32_t r1 = min(run, r0 + 32);
      if (run > r0 + 32) {
        const int ev31 = __shfl_sync(0xFFFFFFFFu, ev, 31);
        const int32_t end31 = ev31 + 1 < kChunk ? excl[ev31 + 1] : run;
        if (end31 > r0 + 32) {
          const int32_t s31 = excl[ev31];
          r1 = s31 > r0 ? s31 : r0 + 32;
        }
      }
      const bool has = g < r1;
      int slot = 0;
      uint32_t pos = 0, k = 0;
      float loss = 0.f, u = 0.f, x = __int_as_float(0x7FC00000), mx = 0.f;
      int seg_start = lane;  // first lane of this hit's event in the round
      if (has) {
        const int nth = g - excl[ev];
        seg_start = max(lane - nth, 0);
        if constexpr (MW == 1) {
          slot = nth_set_bit(s_maskw[0][ev], nth);
        } else {
          const uint32_t m0 = s_maskw[0][ev];
          const int c0 = __popc(m0);
          slot = nth < c0 ? nth_set_bit(m0, nth) : 32 + nth_set_bit(s_maskw[1][ev], nth - c0);
        }
        pos = sbase[ev] + (uint32_t)nth;
        k = (uint32_t)(c - beg) + (uint32_t)ev;
        bool sd0 = false, use_table = false;
        TablePiece pc;
        float tau = 0.f;
        const float cc = (CORR && P.corr != nullptr) ? __ldg(P.corr + pos) : 0.0f;
        if constexpr (TABLE) {
          // the piece index depends on the draw alone: draw first, then one 32-byte load
          const SuDraw d = su_draw(su_uniform_rk(P.rk0, P.rk1, trial, k, P.handles[slot]),
                                   cc > 0.0f ? su_uniform_corr_rk(P.rk0, P.rk1, trial, k) : 0.5f,
                                   cc);
          u = d.z;
          const int kp = ara_table_piece_q(d.lower, d.q, &tau);
          pc = ara_load_piece<false>(P.tables + (size_t)pos * kTablePieces, kp);
          sd0 = pc.flag == kPieceMean;
          mx = pc.mx;
          use_table = pc.flag == kPieceTable;
        }
        BetaRec rec;
        if constexpr (INV == 1) {
          rec = load_rec_policy(P.recs + pos, pol.keep);
          sd0 = !(rec.a > 0.f);
          mx = rec.mx;
          if (!sd0 || TRACE)
            u = su_draw(su_uniform_rk(P.rk0, P.rk1, trial, k, P.handles[slot]),
                        cc > 0.0f ? su_uniform_corr_rk(P.rk0, P.rk1, trial, k) : 0.5f, cc).z;
        }
        if constexpr (SURR) {
          // computed ahead by surrogate_segment
          loss = s_surr->loss[g - seg0];
          if constexpr (TRACE) {
            x = s_tx[g - seg0];
            u = s_tu[g - seg0];
          }
        } else if (sd0) {
          loss = mx;  // sd = 0: the mean (primary uncertainty only)
        } else {
          if (TABLE && use_table) {
            x = ara_piece_x(pc, tau);
            n_tab += 1u;
          } else {
            const IbetaResult ib =
                INV == 1 ? ara_inv_beta(rec, u,
                                        P.starts != nullptr
                                            ? start_logit_policy(P.starts + (size_t)pos *
                                                                     kStartFloats, u, pol.stream)
                                            : 1e30f)
                         : newton_fallback<false>(P.recs + pos, u);
            x = ib.x;
            nc += ib.converged ? 0u : 1u;
            n_inv += 1u;
            n_it += (unsigned)ib.iters;
            n_cf += (unsigned)ib.cf_terms;
          }
          loss = mx * x;
        }
      }
      if constexpr (TRACE) {
        const int32_t th = trace_n + g;
        if (has && th < P.trace_cap) {
          const int64_t o = w * P.trace_cap + th;
          P.tr_k[o] = (int32_t)k;
          P.tr_j[o] = slot;
          P.tr_rec[o] = (int32_t)P.rec_idx[pos];
          P.tr_u[o] = u;
          P.tr_x[o] = x;
          P.tr_loss[o] = loss;
        }
      }
      // segmented inclusive scan over lanes: segments are the runs of equal ev, lanes
      // seg_start .. lane
      const int seg = has ? ev : -1;
      float val = loss;
#pragma unroll
      for (int d = 1; d < 32; d <<= 1) {
        const float nv = __shfl_up_sync(0xFFFFFFFFu, val, d);
        if (lane - d >= seg_start) val += nv;
      }
      const int next_seg = __shfl_down_sync(0xFFFFFFFFu, seg, 1);
      const bool tail = has && (lane == 31 || next_seg != seg);
      if (tail) lsum[ev] += val;
      __syncwarp();
      r0 = r1;
    }
    if constexpr (TRACE) trace_n += run;
    n_hit += (lane == 0) ? (unsigned)run : 0u;

    // ---- occurrence terms and the year's running sum -----------------------------------------
#pragma unroll
    for (int v = 0; v < kV; ++v) {
      const int64_t q = c + v * 32 + lane;
      float o = 0.f;
      if (q < end) {
        const float l = lsum[v * 32 + lane];
        o = fminf(fmaxf(l - P.occ_ret, 0.f), P.occ_lim);
        acc.add(o);
        omax = fmaxf(omax, o);
      }
      if (evt) occurrence_outputs(P, q, end, o, q0, carry, lane);
    }
    __syncwarp();
  }

  acc.warp_reduce();
  // o >= +0 always, so the largest float is the largest bit pattern
  const unsigned om_bits = __reduce_max_sync(0xFFFFFFFFu, __float_as_uint(omax));
  nc = __reduce_add_sync(0xFFFFFFFFu, nc);
  n_inv = __reduce_add_sync(0xFFFFFFFFu, n_inv);
  n_it = __reduce_add_sync(0xFFFFFFFFu, n_it);
  n_cf = __reduce_add_sync(0xFFFFFFFFu, n_cf);
  n_tab = __reduce_add_sync(0xFFFFFFFFu, n_tab);
  n_net = __reduce_add_sync(0xFFFFFFFFu, n_net);
  if (lane == 0) {
    const double S = acc.value();
    P.ylt[w] = fmin(fmax(S - P.agg_ret, 0.0), P.agg_lim);
    if (P.oep) P.oep[w] = (double)__uint_as_float(om_bits);
    if (nc) atomicAdd(P.not_conv, (unsigned long long)nc);
    unsigned long long* st = P.stats + (blockIdx.x & (kStatStripes - 1));
    if (n_inv) atomicAdd(st + 0 * kStatStripes, (unsigned long long)n_inv);
    if (n_it) atomicAdd(st + 1 * kStatStripes, (unsigned long long)n_it);
    if (n_cf) atomicAdd(st + 2 * kStatStripes, (unsigned long long)n_cf);
    if (n_hit) atomicAdd(st + 3 * kStatStripes, (unsigned long long)n_hit);
    if (n_tab) atomicAdd(st + 4 * kStatStripes, (unsigned long long)n_tab);
    if (n_net) atomicAdd(st + 5 * kStatStripes, (unsigned long long)n_net);
    if constexpr (TRACE) P.tr_count[w] = trace_n;
  }
}

// INV: 0 certified tables (Newton fallback), 1 Newton, 2 learned surrogate (Newton fallback).
// The table and Newton paths are latency bound (dependent loads per hit; the serial continued
// fraction), so they are held to 64 registers for 32 resident warps per SM (the Newton path
// runs 4% faster so than at 24 warps with 85 registers).  The surrogate path's blocks hold the
// network's weights (22 KB) and their warps' segment lists in shared memory (45 KB a 4-warp
// block): 4 blocks per SM at up to 128 registers, on a persistent grid so that each block copies
// the weights once.
template <int INV>
constexpr int kBlocksPerSM = INV == 2 ? 4 : 32 / kWPB<INV>;

// Shared memory of the surrogate's segments (trace: each hit's x and u as well), declared only
// where INV == 2.
#define SURR_SMEM(W, INV, TRACE)                                                                 \
  __shared__ SurrWarpSmem s_surr[(INV) == 2 ? (W) : 1];                                         \
  __shared__ float s_trace[((INV) == 2 && (TRACE)) ? 2 * (W) * kSegCap : 1]
#define SURR_ARGS(INV, TRACE)                                                                    \
  &s_surr[(INV) == 2 ? wib : 0], ((INV) == 2 && (TRACE)) ? s_trace + 2 * wib * kSegCap : nullptr, \
      ((INV) == 2 && (TRACE)) ? s_trace + (2 * wib + 1) * kSegCap : nullptr

template <int MW, class Acc, bool TRACE, int INV, bool CORR>
__global__ void __launch_bounds__(kWPB<INV> * 32, kBlocksPerSM<INV>)
    trial_kernel(const __grid_constant__ TrialParams P) {
  constexpr int W = kWPB<INV>;
  __shared__ int32_t s_excl[W][kChunkOf<INV>];
  __shared__ uint32_t s_base[W][kChunkOf<INV>];
  __shared__ uint32_t s_mask[W][MW][kChunkOf<INV>];
  __shared__ float s_lsum[W][kChunkOf<INV>];
  __shared__ __align__(16) MlpSmem s_mlp[1];
  SURR_SMEM(W, INV, TRACE);
  if constexpr (INV == 2) {  // network weights, once per block, before any warp may leave
    const uint4* src = reinterpret_cast<const uint4*>(P.mlp);
    uint4* dst = reinterpret_cast<uint4*>(&s_mlp[0]);
    for (int i = threadIdx.x; i < (int)(sizeof(MlpSmem) / 16); i += blockDim.x) dst[i] = src[i];
    __syncthreads();
  }
  const int lane = threadIdx.x & 31;
  const int wib = threadIdx.x >> 5;
  // one trial per warp; a warp of a grid smaller than the launch's trials takes every
  // (grid size)-th trial (whole warps, no block-wide barrier follows)
  for (int64_t w = (int64_t)blockIdx.x * W + wib; w < P.n; w += (int64_t)gridDim.x * W)
    process_trial<MW, Acc, TRACE, INV, CORR>(P, w, lane, wib, s_excl[wib], s_base[wib],
                                             s_mask[wib], s_lsum[wib], &s_mlp[0],
                                             SURR_ARGS(INV, TRACE));
}

// One launch over many work items (serving: slices of different requests, each with its own
// layer and YLT): warp w runs trial w - warp_begin[i] of the item i with warp_begin[i] <= w.
template <int MW, class Acc, int INV>
__global__ void __launch_bounds__(kWPB<INV> * 32, kBlocksPerSM<INV>)
    batch_kernel(const TrialParams* __restrict__ items, const int64_t* __restrict__ warp_begin,
                 int n_items, int64_t total_warps) {
  constexpr int W = kWPB<INV>;
  __shared__ int32_t s_excl[W][kChunkOf<INV>];
  __shared__ uint32_t s_base[W][kChunkOf<INV>];
  __shared__ uint32_t s_mask[W][MW][kChunkOf<INV>];
  __shared__ float s_lsum[W][kChunkOf<INV>];
  __shared__ __align__(16) MlpSmem s_mlp[1];
  SURR_SMEM(W, INV, false);
  if constexpr (INV == 2) {
    const uint4* src = reinterpret_cast<const uint4*>(items[0].mlp);
    uint4* dst = reinterpret_cast<uint4*>(&s_mlp[0]);
    for (int i = threadIdx.x; i < (int)(sizeof(MlpSmem) / 16); i += blockDim.x) dst[i] = src[i];
    __syncthreads();
  }
  const int lane = threadIdx.x & 31;
  const int wib = threadIdx.x >> 5;
  for (int64_t w = (int64_t)blockIdx.x * W + wib; w < total_warps;
       w += (int64_t)gridDim.x * W) {
    int lo = 0, hi = n_items - 1;
    while (lo < hi) {  // largest item whose first warp is <= w
      const int mid = (lo + hi + 1) >> 1;
      if (warp_begin[mid] <= w) lo = mid; else hi = mid - 1;
    }
    process_trial<MW, Acc, false, INV, true>(items[lo], w - warp_begin[lo], lane, wib,
                                             s_excl[wib], s_base[wib], s_mask[wib],
                                             s_lsum[wib], &s_mlp[0], SURR_ARGS(INV, false));
  }
}

// Blocks of a launch over n warps: one warp per trial, or for the surrogate path at most
// kBlocksPerSM resident blocks per SM (a persistent grid).
template <int INV>
int64_t trial_blocks(int64_t n_warps) {
  int64_t blocks = (n_warps + kWPB<INV> - 1) / kWPB<INV>;
  if constexpr (INV == 2) {
    int dev = 0, sms = 148;
    if (cudaGetDevice(&dev) == cudaSuccess)
      cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    blocks = std::min<int64_t>(blocks, (int64_t)sms * kBlocksPerSM<INV>);
  }
  return blocks;
}

template <int MW, class Acc, bool TRACE, int INV, bool CORR = true>
cudaError_t launch_one(const TrialParams& p, cudaStream_t st) {
  const int64_t blocks = trial_blocks<INV>(p.n);
  if (blocks == 0) return cudaSuccess;
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = dim3((unsigned)blocks);
  cfg.blockDim = dim3(kWPB<INV> * 32);
  cfg.dynamicSmemBytes = 0;
  cfg.stream = st;
  const cudaError_t e = cudaLaunchKernelEx(&cfg, trial_kernel<MW, Acc, TRACE, INV, CORR>, p);
  count_launches(1);
  if (e != cudaSuccess) return e;
  return cudaGetLastError();
}

template <int INV>
cudaError_t launch_mode(const TrialParams& p, int mask_words, int precision, bool trace,
                        cudaStream_t st) {
  if (trace) {
    return mask_words == 1 ? launch_one<1, AccExact, true, INV>(p, st)
                           : launch_one<2, AccExact, true, INV>(p, st);
  }
  if (precision == 1) {
    return mask_words == 1 ? launch_one<1, AccKahan, false, INV>(p, st)
                           : launch_one<2, AccKahan, false, INV>(p, st);
  }
  // the common case (exact sums, no weights, no surrogate) compiled without the weight path
  if constexpr (INV != 2) {
    if (p.corr == nullptr)
      return mask_words == 1 ? launch_one<1, AccExact, false, INV, false>(p, st)
                             : launch_one<2, AccExact, false, INV, false>(p, st);
  }
  return mask_words == 1 ? launch_one<1, AccExact, false, INV>(p, st)
                         : launch_one<2, AccExact, false, INV>(p, st);
}

template <int MW, class Acc, int INV>
cudaError_t launch_batch_mode(const TrialParams* d_items, const int64_t* d_warp_begin,
                              int n_items, int64_t total_warps, cudaStream_t st) {
  const int64_t blocks = trial_blocks<INV>(total_warps);
  if (blocks == 0) return cudaSuccess;
  batch_kernel<MW, Acc, INV><<<(unsigned)blocks, kWPB<INV> * 32, 0, st>>>(
      d_items, d_warp_begin, n_items, total_warps);
  count_launches(1);
  return cudaGetLastError();
}

template <class Acc, int INV>
cudaError_t launch_batch_mw(const TrialParams* d_items, const int64_t* d_warp_begin,
                            int n_items, int64_t total_warps, int mask_words, cudaStream_t st) {
  return mask_words == 1
             ? launch_batch_mode<1, Acc, INV>(d_items, d_warp_begin, n_items, total_warps, st)
             : launch_batch_mode<2, Acc, INV>(d_items, d_warp_begin, n_items, total_warps, st);
}

}  // namespace

cudaError_t launch_trial_batch(const TrialParams* d_items, const int64_t* d_warp_begin,
                               int n_items, int64_t total_warps, int mask_words, int precision,
                               int inversion, cudaStream_t st) {
  const int mw = mask_words;
  if (precision == 1) {
    if (inversion == 2) return launch_batch_mw<AccKahan, 2>(d_items, d_warp_begin, n_items, total_warps, mw, st);
    if (inversion == 1) return launch_batch_mw<AccKahan, 1>(d_items, d_warp_begin, n_items, total_warps, mw, st);
    return launch_batch_mw<AccKahan, 0>(d_items, d_warp_begin, n_items, total_warps, mw, st);
  }
  if (inversion == 2) return launch_batch_mw<AccExact, 2>(d_items, d_warp_begin, n_items, total_warps, mw, st);
  if (inversion == 1) return launch_batch_mw<AccExact, 1>(d_items, d_warp_begin, n_items, total_warps, mw, st);
  return launch_batch_mw<AccExact, 0>(d_items, d_warp_begin, n_items, total_warps, mw, st);
}

cudaError_t launch_trial(const TrialParams& p, int mask_words, int precision, int inversion,
                         bool trace, cudaStream_t st) {
  if (inversion == 2) return launch_mode<2>(p, mask_words, precision, trace, st);
  return inversion == 0 ? launch_mode<0>(p, mask_words, precision, trace, st)
                        : launch_mode<1>(p, mask_words, precision, trace, st);
}

}  // namespace ara
