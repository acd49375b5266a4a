// ara_ctx.h -- the context object behind the opaque ara_ctx handle (shared by libara's host
// sources).
#pragma once

#include <cuda_runtime.h>

#include <string>
#include <vector>

#include "../../include/ara.h"
#include "ara_internal.h"

using ara::BetaRec;
using ara::EltDev;
using ara::LayerDev;
using ara::MlpDevWeights;
using ara::SortScratch;
using ara::TrialParams;
using ara::YetDev;

// Device buffers of event ids a streamed run cycles through (the first ones are filled ahead by
// ara_create_yet_host).
constexpr int kStreamBufs = 4;

struct ara_ctx {
  ara_config cfg{};
  int device = 0;
  int sm_count = 148;  // streaming multiprocessors of the device
  cudaStream_t stream = nullptr;
  std::string detail;
  std::vector<YetDev> yets;
  std::vector<EltDev> elts;
  std::vector<LayerDev> layers;
  unsigned long long* d_not_conv = nullptr;
  unsigned long long* d_stats = nullptr;  // [kStatCounters * kStatStripes]
  int32_t inversion = 0;                   // 0 certified tables + Newton fallback, 1 Newton
  // learned surrogate: FP32 master parameters, Adam moments, gradient, BF16 image, cell errors
  float *mlp_P = nullptr, *mlp_M = nullptr, *mlp_V = nullptr, *mlp_G = nullptr;
  MlpDevWeights* mlp_W = nullptr;
  float* mlp_bound = nullptr;
  float mlp_eps = 0.0f;
  bool mlp_ready = false;
  unsigned int* d_flags = nullptr;
  cudaStream_t own_stream = nullptr;
  // grow-only scratch
  SortScratch sort;
  double* d_ylt_tmp = nullptr;
  int64_t ylt_tmp_cap = 0;
  unsigned long long* d_ysum = nullptr;  // year sums in grid units (band-major runs)
  int64_t ysum_cap = 0;
  int32_t schedule = ARA_SCHED_AUTO;     // ARA_SCHED_*
  int32_t table_policy = 0;              // ARA_TABLES_EAGER or ARA_TABLES_ON_DEMAND
  uint32_t* d_sel = nullptr;             // top-k selection: flags, positions, scan scratch
  int64_t sel_cap = 0;
  // streamed runs over host-resident YETs: a copy stream, a ring of device buffers of ids filled
  // in turn, and the events that hand each buffer between the streams
  cudaStream_t copy_stream = nullptr;
  cudaEvent_t ev_ready[kStreamBufs] = {};
  cudaEvent_t ev_free[kStreamBufs] = {};
  int32_t* d_sids[kStreamBufs] = {};
  int64_t stream_cap = 0;
  int64_t stream_chunk = (int64_t)1 << 26;  // ARA_OPT_STREAM_CHUNK
  // chunks of a host YET's first run copied ahead by ara_create_yet_host: the YET, the chunk
  // size they were cut with and each one's trial range (buffer k holds chunk k)
  int32_t pf_yet = -1;
  int32_t pf_count = 0;
  int64_t pf_cap = 0;
  int64_t pf_tb[kStreamBufs] = {}, pf_te[kStreamBufs] = {};
  // staging scratch (grow-only, see ensure_scratch)
  char* d_scratch = nullptr;
  size_t scratch_cap = 0;
  int32_t band_log2w = 0;                // band width exponent for new layers (0: automatic)
  void* d_misc = nullptr;  // small staging area for tail sums
  // the device memory of YETs, ELTs and layers (see obj_alloc)
  cudaMemPool_t pool = nullptr;
};

// Internal entry points shared between the API and the serving loop.
// Builds a layer into *out (not registered in ctx->layers) with its device work on st; with
// may_build_band false an absent band-major YET copy leaves the layer trial-major; with ordered
// true its memory is stream-ordered on st (free it with free_layer_on(ctx, ..., true, stream)); with
// starts true the ELTs' start tables are packed too (runs that invert by Newton-Halley steps;
// otherwise the first such run packs them).
ara_status ara_build_layer(ara_ctx* ctx, const int32_t* elts, int32_t n_elts, double occ_ret,
                           double occ_lim, double agg_ret, double agg_lim, bool wide,
                           cudaStream_t st, bool may_build_band, bool ordered, LayerDev* out,
                           bool starts = false);
void free_layer(ara_ctx* ctx, LayerDev& l);
void free_layer_on(ara_ctx* ctx, LayerDev& l, bool ordered, cudaStream_t st);
ara_status ara_add_layer_impl(ara_ctx* ctx, const int32_t* elts, int32_t n_elts, double occ_ret,
                              double occ_lim, double agg_ret, double agg_lim, bool wide,
                              int32_t* layer_out);
int inversion_mode(const ara_ctx* ctx);
// Makes sure the YET has its band-major copy for band width 2^log2w (*available: it has).
ara_status ensure_band_variant(ara_ctx* ctx, int32_t yet, int log2w, bool* available);
bool uses_band_schedule(const ara_ctx* ctx, const LayerDev& L);
// The inversion a run over L uses: the context's, except that the table inversion falls back to
// Newton's method (1) while the layer has no packed tables (ARA_TABLES_ON_DEMAND).
int layer_inversion(const ara_ctx* ctx, const LayerDev& L);
// Rent-or-buy before a run of n trials over L: builds the tables of L's ELTs and L's packed copy
// when the accumulated Newton work reaches the build cost; else books this run as Newton work.
// With band_ok, a run that takes the band schedule first makes the layer's band-major YET copy
// if it is still wanted.
ara_status prepare_layer_for_run(ara_ctx* ctx, LayerDev& L, int64_t n, bool band_ok);
// Builds every missing table (or start table) of the live ELTs of a YET (servers need them).
ara_status ensure_yet_tables(ara_ctx* ctx, int32_t yet);
ara_status ensure_yet_starts(ara_ctx* ctx, int32_t yet);
TrialParams make_params(ara_ctx* ctx, const YetDev& Y, const LayerDev& L, int64_t t0, int64_t n,
                        double* d_ylt);
// The stream ring with buffers of at least cap ids, the copy stream and the hand-over events.
ara_status ensure_stream_ring(ara_ctx* ctx, int64_t cap);
// End of the streamed chunk that starts at trial tb: whole trials up to cap occurrences (a trial
// never exceeds cap), ending at `end` at the latest.
int64_t stream_chunk_end(const YetDev& Y, int64_t tb, int64_t end, int64_t cap);
// Copies the first chunks of a run over all trials of host YET `yet` into the stream ring ahead
// of that run, on the copy stream (nothing is waited for; a failure leaves nothing copied ahead).
void prefetch_stream(ara_ctx* ctx, int32_t yet);
