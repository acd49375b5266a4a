// ara_internal.h -- device data structures and kernel launchers shared by libara's sources.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include <string>
#include <vector>

#include "ara_ibeta.cuh"
#include "ara_mlp.cuh"

namespace ara {

constexpr int kMaxLayerElts = 64;

// A YET bucketed by catalogue band for the band-major schedule of the table path.  Band b holds
// the catalogue events [b W, (b + 1) W), W = 2^log2w.  The occurrences of band b are stored
// together, trial by trial, each trial's in its own occurrence order, as the 32-bit word
// (e - b W) << kbits | k with k the occurrence's position in its trial.  The occurrences of
// (band b, trial i) are occ[off[b N + i] .. off[b N + i + 1]) (N = trials; off[P N] = total).
struct BandedYet {
  int32_t log2w = 0;         // 0: not built
  int32_t n_bands = 0;       // P = ceil(catalog / W)
  int32_t kbits = 0;         // 32 - log2w
  uint32_t* occ = nullptr;   // [n_occ]
  uint32_t* off = nullptr;   // [P N + 1]
};
constexpr int kMaxBandVariants = 6;
constexpr int kMaxBands = 512;

// Year Event Table on the device: trial-major event ids and timestamps (paper §2.1).
struct YetDev {
  bool live = false;
  // host-resident YET (ara_create_yet_host): ids and timestamps stay in the caller's memory and
  // each run streams the trials it needs; offsets are on the device as for a resident YET
  bool host = false;
  const int32_t* h_ids = nullptr;
  const float* h_ts = nullptr;
  std::vector<int64_t> h_off;  // [n_trials + 1] (host YETs only)
  bool ts_checked = false;     // host YETs: timestamps validated (by the first run)
  int64_t n_trials = 0;
  int64_t n_occ = 0;
  int32_t catalog = 0;
  int64_t max_len = 0;       // longest trial
  int32_t* ids = nullptr;    // [n_occ] (timestamps are checked at staging and not kept)
  int64_t* offsets = nullptr;  // [n_trials + 1]
  BandedYet bands[kMaxBandVariants];  // band-major copies, built on demand per band width
  double band_rent_occ = 0.0;  // occurrences run trial-major by the table inversion (schedule AUTO)
};

// One staged ELT: event ids and the derived per-record constants, in the caller's order.
struct EltDev {
  bool live = false;
  int32_t yet = -1;
  int64_t n = 0;
  int32_t* ids = nullptr;    // [n]
  BetaRec* recs = nullptr;   // [n]
  TablePiece* tables = nullptr;  // [n * kTablePieces] certified quantile tables
  float* corr = nullptr;     // [n] normalised correlated weights (NULL: every sigma_C = 0)
  int64_t n_uncertified = 0; // records whose table failed certification
  float* starts = nullptr;   // [n * kStartFloats] start tables of the Newton-Halley inversion
                             // (built when a run or a server first needs them)
  double rent_hits = 0.0;    // expected hits per record served by Newton while tables were absent
};

// A layer: lookup structure over the YET's catalogue plus its terms (paper §2.1, §2.3).
// evt[e] holds (base, mask words...): the records of event e in the layer's ELTs are
// packed[base + r], r = rank of the ELT's slot bit among the set bits of the mask.
struct LayerDev {
  bool live = false;
  int32_t yet = -1;
  int32_t n_slots = 0;
  int32_t mask_words = 1;          // 1 (<= 32 ELTs) or 2 (<= 64)
  int32_t handles[kMaxLayerElts];  // global ELT handle per slot (keys the uniforms)
  double occ_ret = 0, occ_lim = 0, agg_ret = 0, agg_lim = 0;
  uint32_t* evt = nullptr;         // [catalog * (1 + mask_words)] entries, padded to 2 or 4 words
  BetaRec* packed = nullptr;       // [n_packed]
  TablePiece* tables = nullptr;    // [n_packed * kTablePieces] the records' tables, same order
  float* starts = nullptr;         // [n_packed * kStartFloats] the records' start tables
  uint32_t* packed_rec = nullptr;  // [n_packed] caller record index (verification)
  float* corr = nullptr;           // [n_packed] correlated weights (NULL: none in the layer)
  int64_t n_packed = 0;
  bool own_tables = false;         // tables built in place (the ELTs had none)
  int64_t n_uncertified = 0;       // records of tables built for the layer alone that failed
  int32_t band_log2w = 0;          // band width of the band-major schedule (0: trial-major only)
  int32_t band_want = 0;           // width chosen at build whose band-major YET copy is made at
                                   // the first run that takes the band schedule (0: none)
  float ev_bound = 0.f;            // largest event-loss bound (sizes the year-sum grid)
};

// Parameters of one trial-kernel launch.
struct TrialParams {
  const int32_t* ids;
  const int64_t* offsets;
  const uint32_t* evt;
  const BetaRec* recs;
  const TablePiece* tables;  // the layer's tables, kTablePieces per packed record
  const float* corr;         // packed correlated weights (paper §3.2), NULL when all are zero
  const float* starts;       // packed start tables of the Newton-Halley inversion, or NULL
  const uint32_t* rec_idx;
  int32_t handles[kMaxLayerElts];
  int32_t n_slots;
  float occ_ret, occ_lim;
  double agg_ret, agg_lim;
  uint64_t seed;
  uint32_t rk0[10], rk1[10];  // Philox round keys of seed
  int64_t t0, n;
  double* ylt;
  unsigned long long* not_conv;
  unsigned long long* stats;  // [6 x kStatStripes]: inversions, Newton iterations, CF terms,
                              //      hits, table evals, surrogate evaluations
  const MlpSmem* mlp;         // surrogate weights (inversion 2)
  const float* mlp_bound;     // certified error per cell
  float mlp_eps;
  // verification trace (TRACE instantiation only)
  int64_t trace_cap;  // hits per trial slot in the trace buffers
  int32_t* tr_k;
  int32_t* tr_j;
  int32_t* tr_rec;
  float* tr_u;
  float* tr_x;
  float* tr_loss;
  int32_t* tr_count;  // [n]
  // band-major schedule
  const uint32_t* bocc;  // BandedYet::occ
  const uint32_t* boff;  // BandedYet::off
  int64_t yet_n;         // trials of the YET (row length of boff)
  int32_t log2w, kbits, n_bands, tiles;
  unsigned long long* ysum;  // [n] year sums in grid units (band-major schedule; zeroed first)
  // grid of the exact year sums: occurrence results are rounded to multiples of q_unit = 2^e
  float q_scale;             // 2^-e
  double q_unit;             // 2^e
  // event-level output (optional): each year's largest occurrence loss, after occurrence terms
  double* oep;               // [n] or null
  unsigned int* omax;        // [n] binary32 bit patterns of the running maxima (band-major;
                             //     zeroed first; non-negative floats order like their bits)
  // host-resident YETs: ids holds occurrences [occ_base, ...) of the streamed chunk (0 for a
  // resident YET); a nonzero *abort_flag (the chunk failed validation) makes warps skip work
  int64_t occ_base;
  const unsigned int* abort_flag;
  // per-occurrence outputs (trial-major only), indexed by occurrence position - offsets[t0]
  float* olt;                // occurrence loss after occurrence terms, or null
  double* inc;               // increment of the year's net aggregate loss, or null
  // A(S) = min(max(S - AggR, 0), AggL) for S = s grid units is 0 for s <= agg_zero_max and AggL
  // for s >= agg_full_min (exact bounds of the binary64 formula), so increments there are 0
  unsigned long long agg_zero_max, agg_full_min;
};

// Work counters are striped over kStatStripes copies (counter c of stripe s at
// stats[c * kStatStripes + s]) so that blocks do not contend on one address.
constexpr int kStatCounters = 6;
constexpr int kStatStripes = 64;

// Kernel launches issued by this library since load (every launcher adds its launches).
void count_launches(int64_t n);
int64_t launches_so_far();

// ---- launchers (each returns the launch's cudaError_t) ---------------------------------------
// Trial offsets checked on the device: off[0], the first trial whose offset decreases (-1:
// none), the longest trial and off[n_trials].
struct OffsetCheck {
  int64_t first, first_decrease, max_len, last;
};
// *out (device, 32 bytes) receives the check of off[0 .. n_trials]
cudaError_t launch_check_offsets(const int64_t* off, int64_t n_trials, OffsetCheck* out,
                                 cudaStream_t st);
// Checks of a YET's trials [t_begin, t_begin + n) whose occurrences [occ_base, ...) are in
// ids / ts (ts may be null: timestamps checked elsewhere): flags bit 0 an id out of range, bit 1
// a decreasing timestamp, bit 2 a NaN timestamp; ids_out (nullable) receives a copy of the ids
// checked
cudaError_t launch_validate_yet_range(const int32_t* ids, const float* ts, int64_t occ_base,
                                      const int64_t* offsets, int64_t t_begin, int64_t n,
                                      int32_t catalog, unsigned int* d_flags, cudaStream_t st,
                                      int32_t* ids_out = nullptr);
// Checks and converts the records of up to kMaxPrepJobs ELTs in one launch: job j's ids, mean,
// sd, optional correlated sd (sdc[j] NULL: zero) and max exposure (all device-readable) into
// recs[j] / corr[j] (corr[j] NULL: none); ids_out[j] (nullable) receives a copy of the ids.
// first[j] records come before job j (first[n]: all).  d_dup[catalog] (zeroed by the caller)
// marks events per job; d_flags[j] (zeroed) receives job j's rejection flags.
constexpr int kMaxPrepJobs = 32;
struct PrepJobs {
  const int32_t* ids[kMaxPrepJobs];
  int32_t* ids_out[kMaxPrepJobs];
  const double* mean[kMaxPrepJobs];
  const double* sd[kMaxPrepJobs];
  const double* sdc[kMaxPrepJobs];
  const double* mx[kMaxPrepJobs];
  BetaRec* recs[kMaxPrepJobs];
  float* corr[kMaxPrepJobs];
  int64_t first[kMaxPrepJobs + 1];
  int n;
};
cudaError_t launch_prepare_elts(const PrepJobs& jobs, int32_t catalog, unsigned int* d_dup,
                               unsigned int* d_flags, cudaStream_t st);
cudaError_t launch_layer_mask(const EltDev& e, int slot, int mask_words, uint32_t* d_mask,
                              cudaStream_t st);
cudaError_t launch_layer_counts(const uint32_t* d_mask, int mask_words, int64_t catalog,
                                uint32_t* d_cnt, cudaStream_t st);
cudaError_t launch_exclusive_scan_u32(const uint32_t* in, uint32_t* out, int64_t n,
                                      uint32_t* d_tmp, int64_t tmp_words, cudaStream_t st);
int64_t scan_tmp_words(int64_t n);
cudaError_t launch_layer_index(const uint32_t* d_mask, const uint32_t* d_base, int mask_words,
                               int64_t catalog, uint32_t* d_evt, cudaStream_t st);
// start_src (optional): each packed record's start table in its ELT, for launch_gather_starts
cudaError_t launch_layer_scatter(const EltDev& e, int slot, int mask_words,
                                 const uint32_t* d_evt, BetaRec* packed,
                                 const TablePiece** table_src, uint32_t* packed_rec,
                                 float* packed_corr, const float** start_src, cudaStream_t st);
// *d_bound = binary32 bits of the layer's largest event-loss bound (sum over an event's records
// of max_l, or the mean where sd = 0), rounded up; 0 for a layer without records
cudaError_t launch_layer_event_bound(const uint32_t* d_evt, int mask_words, int64_t catalog,
                                     const BetaRec* packed, unsigned int* d_bound,
                                     cudaStream_t st);
// starts[n * kStartFloats]: the records' start tables of the Newton-Halley inversion
cudaError_t launch_build_starts(int64_t n, const BetaRec* recs, float* starts, cudaStream_t st);
// The certified tables of up to kMaxTableJobs ELTs in one launch: job j's records recs[j] and
// its tables tables[j] (kTablePieces pieces each); first[j] records come before job j (first[n]:
// all of them).  d_uncertified[j] (zeroed by the caller) counts job j's uncertified records.
constexpr int kMaxTableJobs = 64;
struct TableJobs {
  const BetaRec* recs[kMaxTableJobs];
  TablePiece* tables[kMaxTableJobs];
  int64_t first[kMaxTableJobs + 1];
  int n;
};
cudaError_t launch_build_tables(const TableJobs& jobs, unsigned long long* d_uncertified,
                                cudaStream_t st);
// elt_tables[n * kTablePieces] = the tables of the n records (ids) of the ELT in slot `slot` of a
// layer whose tables (layer_tables, packed order, lookup entries evt) were built in place;
// *d_uncertified (zeroed by the caller) += the records among them whose table failed.
cudaError_t launch_unpack_tables(int64_t n, const int32_t* ids, int slot, int mask_words,
                                 const uint32_t* evt, const TablePiece* layer_tables,
                                 TablePiece* elt_tables, unsigned long long* d_uncertified,
                                 cudaStream_t st);
// dst[i * kStartFloats ...] = the start table at d_src[i], for the n packed records of a layer
cudaError_t launch_gather_starts(int64_t n, const float* const* d_src, float* dst, cudaStream_t st);
// dst[i * kTablePieces ...] = the table at d_src[i], for the n packed records of a layer
cudaError_t launch_gather_tables(int64_t n, const TablePiece* const* d_src, TablePiece* dst,
                                 cudaStream_t st);
// inversion: 0 = certified tables with Newton fallback, 1 = Newton everywhere, 2 = learned
// surrogate with Newton fallback
cudaError_t launch_trial(const TrialParams& p, int mask_words, int precision, int inversion,
                         bool trace, cudaStream_t st);
// One launch over n_items work items (device array of TrialParams whose layers all use 16-byte
// index entries, i.e. mask_words = 2); warp_begin[i] = first warp of item i (device, ascending).
// Band-major schedule (certified-table inversion).
int choose_band_log2w(int64_t catalog, int64_t n_packed);
bool band_layout_fits(const YetDev& y, int log2w);
cudaError_t build_band_variant(const YetDev& y, int log2w, BandedYet& out, cudaStream_t st);
void free_band_variant(BandedYet& v);
int64_t band_tiles(int64_t n);
// exponent e of the year-sum grid for trials of at most max_len occurrences, each at most o_max
int year_grid_exponent(double o_max, int64_t max_len);
// the largest occurrence result o = min(max(l - OccR, 0), OccL) the kernels can produce when no
// event loss l exceeds ev_bound (binary32 rounding of the sums and of OccR included)
double occurrence_bound(float ev_bound, double occ_ret, double occ_lim);
// band kernel + per-trial finalisation over p.t0 .. p.t0 + p.n; p.ysum holds n words (zeroed here)
// inversion: 0 certified tables, 1 Newton-Halley from the layer's start tables (p.starts set)
cudaError_t launch_band(const TrialParams& p, int mask_words, int precision, int inversion,
                        cudaStream_t st);
// many items in one launch (serving slices, portfolio layers), all with mask_words-word lookup
// entries: items with their band fields set (tiles = band_tiles(n), ysum zeroed); block_begin[i]
// = first block of item i (n_bands * tiles blocks each), trial_begin[i] = its first trial
// corr: some item carries correlated weights
cudaError_t launch_band_batch(const TrialParams* d_items, const int64_t* d_block_begin,
                              const int64_t* d_trial_begin, int n_items, int64_t total_blocks,
                              int64_t total_trials, int mask_words, bool corr, int precision,
                              cudaStream_t st);
// warp_begin[i] = first warp of item i (one warp per trial)
cudaError_t launch_trial_batch(const TrialParams* d_items, const int64_t* d_warp_begin,
                               int n_items, int64_t total_warps, int mask_words, int precision,
                               int inversion, cudaStream_t st);

// Radix sort of binary64 year losses (descending, ties by index) and tail sums.
struct SortScratch {
  uint64_t* keys[2] = {nullptr, nullptr};
  uint32_t* vals[2] = {nullptr, nullptr};
  uint32_t* hist = nullptr;       // [256 * tiles]
  uint32_t* scan_tmp = nullptr;
  uint32_t* digit_flags = nullptr;  // [4]: varying-bit mask (2 words), NaN flag, spare
  int64_t cap = 0;                // elements
  int64_t hist_cap = 0;
  int64_t scan_cap = 0;
};
int64_t sort_tiles(int64_t n);
// Sorts ylt[n] (device) -> the permutation is left in vals[result_buf]; returns that index via
// *which.  Uses the scratch buffers only.
cudaError_t sort_ylt_desc(const double* d_ylt, int64_t n, SortScratch& s, int* which,
                          cudaStream_t st);
cudaError_t launch_tail_sums(const double* d_ylt, const uint32_t* d_order, int64_t n,
                             const int64_t* d_k, int32_t m, double* d_pml, double* d_tvar,
                             cudaStream_t st);
cudaError_t launch_order_to_i64(const uint32_t* d_order, int64_t n, int64_t* d_out,
                                cudaStream_t st);
// The first k entries of d_order (ranks), written to d_out in ascending index order; flags and
// pos hold n words each, tmp the scan's scratch.
cudaError_t launch_top_k_in_index_order(const double* d_y, const uint32_t* d_order, int64_t n,
                                       int64_t k, uint32_t* flags, uint32_t* pos, uint32_t* tmp,
                                       int64_t tmp_words, double* d_out, cudaStream_t st);
cudaError_t launch_check_nan(const double* d_ylt, int64_t n, unsigned int* d_flag,
                             cudaStream_t st);

// Tail counts passed by value to a kernel (no device buffer needed).
constexpr int kMaxTailCounts = 16;
struct TailCounts {
  int64_t k[kMaxTailCounts];
};
// Same ordering as sort_ylt_desc on caller-provided buffers, with every radix pass run and no
// host round trip; *order receives the buffer holding the permutation.  flags4 is cleared here
// and flags4[2] is raised if the YLT holds a NaN.
cudaError_t sort_ylt_desc_no_sync(const double* d_ylt, int64_t n, uint64_t* keys0,
                                  uint64_t* keys1, uint32_t* vals0, uint32_t* vals1,
                                  uint32_t* hist, uint32_t* scan_tmp, int64_t scan_cap,
                                  uint32_t* flags4, const uint32_t** order, cudaStream_t st);
cudaError_t launch_tail_sums_flagged(const double* d_ylt, const uint32_t* d_order,
                                     const TailCounts& ks, int32_t m,
                                     const unsigned int* d_nan_flag, double* d_pml,
                                     double* d_tvar, cudaStream_t st);

// ---- learned surrogate (ara_mlp.cu) -------------------------------------------------------------
constexpr int kCert0 = 32, kCert1 = 32, kCert2 = 64;  // certification grid over the inputs
constexpr int64_t kCertCells = (int64_t)kCert0 * kCert1 * kCert2;

struct MlpScratch {  // per-step buffers of a training batch of B rows (transposed, BF16)
  __nv_bfloat16 *HT0 = nullptr, *HT1 = nullptr, *HT2 = nullptr, *HT3 = nullptr;
  __nv_bfloat16 *DZT1 = nullptr, *DZT2 = nullptr, *DZT3 = nullptr;
  int64_t B = 0;
};
cudaError_t launch_mlp_gen(int64_t n, uint64_t seed, int64_t first, float* Z, float* X, float* T,
                           unsigned int* bad, cudaStream_t st);
cudaError_t launch_mlp_pack(const float* P, MlpDevWeights* Wd, cudaStream_t st);
cudaError_t launch_mlp_step(const MlpDevWeights* Wd, const float* Z, const float* X,
                            const float* T, int64_t B, MlpScratch& s, float* grad, float* loss_acc,
                            cudaStream_t st);
cudaError_t launch_mlp_adam(float* P, float* M, float* V, float* G, float lr, int64_t step,
                            cudaStream_t st);
cudaError_t launch_mlp_eval(const MlpDevWeights* Wd, const float* Z, int64_t n, float* Y,
                            cudaStream_t st);
cudaError_t launch_mlp_cert_points(int64_t n_cells, int samples, uint64_t seed, float* Z, float* X,
                                   unsigned int* bad, cudaStream_t st);
cudaError_t launch_mlp_cert_reduce(int64_t n_cells, int samples, const float* X, const float* Y,
                                   float* bound, cudaStream_t st);

}  // namespace ara
