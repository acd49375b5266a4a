/*
 * ara.h -- C ABI of libara: aggregate risk analysis with secondary uncertainty on one B300 GPU.
 *
 * Method: Varghese & Rau-Chaplin, "Accounting for Secondary Uncertainty: Efficient Computation of
 * Portfolio Risk Measures on Multi and Many Core Architectures" (WHPCF'13), Algorithm 1 with the
 * secondary-uncertainty model of its §3.  For every trial of a Year Event Table and every event
 * in timestamp order, each ELT of a layer is looked up; a hit draws a loss
 * max_l * InvCDF_beta(u; alpha, beta) from the moment-matched beta distribution; the losses of an
 * event are summed, the occurrence terms applied, the results summed over the year and the
 * aggregate terms applied, giving one Year Loss Table entry per trial.  PML and TVaR follow
 * from the ordered YLT.
 *
 * Conventions shared by every call:
 *   - Every call returns an ara_status; outputs are written only on ARA_OK unless a call says
 *     otherwise.  ara_last_error_detail() gives a one-line reason for the last failure.
 *   - Handles (YET, ELT, layer) are small non-negative integers owned by the context; they stay
 *     valid until freed or until ara_destroy().
 *   - Input arrays may be host or device pointers (the library tells them apart through unified
 *     addressing) and are copied: the caller keeps ownership and may free them on return.
 *   - The library never frees caller memory; ara_destroy() frees everything it allocated.
 *   - A context is used by one host thread at a time.
 *   - Device work runs on the context's own stream unless a call takes a stream argument.
 *   - Nothing in the library traps, spins without bound or aborts the process: device-side
 *     iteration caps are reported as ARA_ERR_NOT_CONVERGED with the results still written.
 */
#ifndef ARA_H
#define ARA_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

#define ARA_API __attribute__((visibility("default")))

typedef struct ara_ctx ara_ctx;

typedef enum {
  ARA_OK = 0,
  ARA_ERR_INVALID_ARG = 1,   /* a size, pointer, value or ordering rule was broken      */
  ARA_ERR_BAD_HANDLE = 2,    /* unknown or freed YET / ELT / layer handle                */
  ARA_ERR_OOM = 3,           /* device or host allocation failed                         */
  ARA_ERR_CUDA = 4,          /* a CUDA runtime call failed (detail holds its message)    */
  ARA_ERR_NOT_CONVERGED = 5, /* some inversions hit the iteration cap; results written    */
  ARA_ERR_BUSY = 6,          /* the serving queue is full                                */
  ARA_ERR_NO_DEVICE = 7      /* no usable CUDA device                                    */
} ara_status;

/* Per-trial accumulation of occurrence losses into the year's aggregate (paper §2.3):
 * ARA_ACC_FP64 sums in binary64; ARA_ACC_KAHAN32 sums in binary32 with Kahan compensation.
 * Sampling, event sums and occurrence terms are binary32 in both; PML/TVaR tails are binary64. */
#define ARA_ACC_FP64 0
#define ARA_ACC_KAHAN32 1

typedef struct {
  uint64_t seed;       /* Philox key for the secondary-uncertainty uniforms (42 by convention) */
  int32_t precision;   /* ARA_ACC_FP64 or ARA_ACC_KAHAN32                                      */
  int32_t use_surrogate; /* 0 = exact inversion everywhere; 1 = learned surrogate with fallback */
  int32_t device;      /* CUDA device ordinal                                                   */
  int32_t reserved;
} ara_config;

/* Context ------------------------------------------------------------------------------------- */
ARA_API ara_status ara_create(const ara_config* cfg, ara_ctx** out);
ARA_API void ara_destroy(ara_ctx* ctx); /* NULL-safe; waits for the context's device work */
ARA_API const char* ara_status_string(ara_status s);
/* Copies the detail of the last failed call on ctx (NUL-terminated, truncated to n bytes). */
ARA_API ara_status ara_last_error_detail(const ara_ctx* ctx, char* buf, size_t n);
/* Options settable after creation: ARA_OPT_PRECISION (value ARA_ACC_*), ARA_OPT_SEED,
 * ARA_OPT_SURROGATE (0/1), ARA_OPT_INVERSION (value ARA_INV_*), ARA_OPT_SCHEDULE (ARA_SCHED_*).
 * Inversion of the beta CDF (paper §3.3, InvCDF_beta):
 *   ARA_INV_TABLE (default): each record's quantile function, tabulated (ARA_OPT_TABLES says
 *     when): 32 quintic pieces per tail in t = sqrt(-2 ln u), 2 KB per record, built from
 *     binary32 Newton-Halley inversions at the knots and checked at every piece's midpoint
 *     against that inversion: within 1e-6 relative in x / (1 - x), plus the binary32 rounding of
 *     the log-odds and of the inversion itself (the latter capped at 1e-5); records failing the
 *     check use Newton;
 *   ARA_INV_NEWTON: Halley's method (Newton's step with the free second derivative) in ln x on
 *     the continued fraction for every hit, started from the record's start table (16 binary32
 *     quintic pieces of the log-odds, 512 bytes per record, built when a run or a server first
 *     needs them), one step in almost every case; also used by runs over ELTs whose tables are
 *     deferred (ARA_OPT_TABLES). */
#define ARA_OPT_PRECISION 1
#define ARA_OPT_SEED 2
#define ARA_OPT_SURROGATE 3
#define ARA_OPT_INVERSION 4
#define ARA_INV_TABLE 0
#define ARA_INV_NEWTON 1
/* ARA_OPT_SCHEDULE (value ARA_SCHED_*):
 *   ARA_SCHED_AUTO (default): trial-major (as ARA_SCHED_TRIAL) until the runs of the table
 *     inversion over a YET have covered ARA_BAND_BUY_PASSES times its occurrences, then band-major
 *     (as ARA_SCHED_BAND): the band-major copy is bought once it has paid for itself in the
 *     time it saves per occurrence (rent-or-buy, never more than twice the cheaper of the two
 *     in hindsight), so a single pass never makes one;
 *   ARA_SCHED_BAND: the catalogue is cut into bands of 2^w events (w chosen per layer so that
 *     one band's lookup entries, record headers and tables fit in L2); the layer's first run
 *     with the table inversion makes a band-major copy of the YET's event ids for that w, once
 *     per w and YET (4 bytes per occurrence plus 4 per (band, trial)), and ara_run visits the
 *     work band by band, each band's year sums kept apart and combined exactly.  A run with the
 *     Newton-Halley inversion takes this schedule too where that copy exists already (it never
 *     makes one: a single pass gains far less than the copy costs);
 *   ARA_SCHED_TRIAL: one warp per trial over its events in order (also used by the surrogate
 *     inversion, by per-occurrence outputs, and by layers whose YET cannot be banded: more than
 *     2^32 occurrences, trials longer than 2^(32-w) events, or more than 512 bands).
 * All give the same hits, uniforms, losses and year losses, bit for bit. */
#define ARA_OPT_SCHEDULE 5
#define ARA_SCHED_BAND 0
#define ARA_SCHED_TRIAL 1
#define ARA_SCHED_AUTO 2
#define ARA_BAND_BUY_PASSES 3.0
/* ARA_OPT_BAND_WIDTH: the band width 2^w (value w in 10..20) of layers created afterwards;
 * 0 (default) chooses w per layer from its record count.  Results do not depend on w. */
#define ARA_OPT_BAND_WIDTH 6
/* ARA_OPT_TABLES: when the certified quantile tables of ELTs staged afterwards are built.
 *   ARA_TABLES_EAGER (default): by ara_add_elt.
 *   ARA_TABLES_ON_DEMAND: not at staging; a run of the table inversion over a layer whose ELTs
 *     lack tables uses Newton's method instead, and the ELTs' tables are built together (and
 *     the layer's packed copy gathered) before the first run at which each such ELT's Newton
 *     work so far plus this run's would reach the cost of building its tables: rent-or-buy,
 *     never more than twice the cheaper of the two in hindsight.  Work is counted in expected
 *     hits per record, (occurrences of the run's trials) / (catalogue size), against
 *     ARA_TABLE_BUY_HITS, the measured break-even of build time per record over the per-hit
 *     saving of a table (a paper-scale pass, ~400 hits per record, buys at once).  A layer none
 *     of whose ELTs has tables yet gets them built straight into its own packed order (the ELTs
 *     keep none and go on renting for other layers).  Results of a
 *     run are those of the inversion it used (both are checked against the oracle).
 *   A server (ara_server_create) builds every missing table of its YET's ELTs when created. */
#define ARA_OPT_TABLES 7
#define ARA_TABLES_EAGER 0
#define ARA_TABLES_ON_DEMAND 1
#define ARA_TABLE_BUY_HITS 260.0
/* ARA_OPT_STREAM_CHUNK: occurrences per copied chunk of a host-resident YET's runs (1024 .. 2^30;
 * default 2^26, a ring of four buffers of 4 bytes per occurrence on the device; a chunk always
 * holds whole trials, so it grows to the longest trial if needed). */
#define ARA_OPT_STREAM_CHUNK 8
ARA_API ara_status ara_set_option(ara_ctx* ctx, int32_t option, int64_t value);

/* Year Event Table (paper §2.1) ------------------------------------------------------------------
 * Trial i owns occurrences trial_offsets[i] .. trial_offsets[i+1]-1 of event_ids/timestamps, in
 * ascending timestamp order (ties keep the stored order).  trial_offsets[0] = 0 and offsets are
 * nondecreasing (an empty trial is allowed).  Event ids must lie in [0, catalog_size).
 * Rejected with ARA_ERR_INVALID_ARG: n_trials < 0, catalog_size <= 0, bad offsets, an id out of
 * range, a timestamp below its predecessor in the same trial, a NaN timestamp.
 * Device copy: int32 ids, trial-major, 4 bytes per occurrence.  Runs never read timestamps, so
 * they are checked and not stored: host ones on host threads while the ids are copied, device
 * ones where they are, on the device.  The context's device memory (YETs, ELTs, layers) comes
 * from a memory pool of its own that keeps up to 32 GiB of freed memory for later staging (it is
 * handed back when an allocation would otherwise fail, and at ara_destroy). */
ARA_API ara_status ara_create_yet(ara_ctx* ctx, int64_t n_trials, const int64_t* trial_offsets,
                                  const int32_t* event_ids, const float* timestamps,
                                  int32_t catalog_size, int32_t* yet_out);
/* Host-resident YET for single passes: the same arrays and checks as ara_create_yet, but only
 * trial_offsets is copied (to the device, 8 B per trial); event_ids and timestamps stay in the
 * caller's host memory, which must stay valid and unchanged until ara_free_yet.  Each ara_run /
 * ara_run_ep / ara_run_events over it (blocking; stream must be NULL) copies the event ids of
 * the trials it needs in chunks of whole trials (ARA_OPT_STREAM_CHUNK) on a copy stream into a
 * ring of four device buffers, while earlier chunks' ids are checked and the chunks are run
 * trial-major on the compute stream, so the PCIe copy of a pass overlaps its computation.  This
 * call already starts the copies of the first four chunks of a run over all trials (nothing
 * waits for them), so they cross while the caller stages ELTs and layers; a first run that
 * starts at trial 0 with the same chunk size uses them, any other call that needs the ring
 * drops them, and ara_free_yet waits for them.  The timestamps never cross: the first run
 * checks them on host threads meanwhile.  An id out of
 * range or a timestamp out of order makes the run return ARA_ERR_INVALID_ARG without writing
 * its outputs.  Page-locked host memory (cudaHostAlloc, or registered)
 * gives the overlap; pageable memory still works, with staged copies.  Layers over it run
 * trial-major; ara_run_portfolio, ara_trace_hits and servers need a device-resident YET
 * (ARA_ERR_INVALID_ARG).  A second pass copies the YET again: keep a YET that several passes
 * read with ara_create_yet. */
ARA_API ara_status ara_create_yet_host(ara_ctx* ctx, int64_t n_trials,
                                       const int64_t* trial_offsets, const int32_t* event_ids,
                                       const float* timestamps, int32_t catalog_size,
                                       int32_t* yet_out);
ARA_API ara_status ara_free_yet(ara_ctx* ctx, int32_t yet);

/* Extended Event Loss Table (paper §2.1, §3.1, §3.3) ----------------------------------------------
 * n records (n >= 0) with distinct event ids in the YET's catalogue: mean loss mu_l > 0,
 * standard deviation sigma >= 0 and maximum exposure max_l > mu_l when sigma > 0.  Events absent
 * from the table have zero loss (paper §4.1).  A record with sigma = 0 contributes its mean
 * (primary uncertainty only).  Values are staged in FP64 once: alpha, beta (moment matching with
 * the sigma_beta_max clamp of §3.3, sigma_beta set to sigma_beta_max (1 - 2^-20) when above it)
 * and the constants of the inversion, then stored as binary32 (32 bytes per record); the record's
 * certified quantile table is built at the same time (2 KB per record, see ARA_OPT_INVERSION;
 * deferred under ARA_TABLES_ON_DEMAND); its start table (512 bytes per record) when a
 * Newton-Halley run first needs it.
 * The handle number keys the record's uniforms: Philox4x32-10 counter (k, i_lo, elt/4, i_hi),
 * key (seed_lo, seed_hi), word elt mod 4, for occurrence k of trial i.  The arrays may be host or
 * device memory; device memory and page-locked host memory mapped into the device's address
 * space are read in place by the staging kernel, pageable host memory is copied first.  The call
 * returns once the records are checked (blocking). */
ARA_API ara_status ara_add_elt(ara_ctx* ctx, int32_t yet, int64_t n, const int32_t* event_ids,
                               const double* mean, const double* sd, const double* max_exposure,
                               int32_t* elt_out);
/* Several ELTs of one YET staged together, each as ara_add_elt_corr stages it: ELT j has n[j]
 * records in event_ids[j], mean[j], sd[j] (sigma_I), sd_corr[j] (sigma_C; sd_corr itself or any
 * entry NULL: all zero) and max_exposure[j].  Their staging is queued back to back and checked
 * once at the end (one synchronisation for all of them), and under ARA_TABLES_EAGER their tables
 * are built in one launch.  Handles go to elts_out[0 .. n_elts) in order.  All or nothing: if an
 * ELT is rejected none is added, and the error detail names the first rejected ELT. */
ARA_API ara_status ara_add_elts(ara_ctx* ctx, int32_t yet, int32_t n_elts, const int64_t* n,
                                const int32_t* const* event_ids, const double* const* mean,
                                const double* const* sd, const double* const* sd_corr,
                                const double* const* max_exposure, int32_t* elts_out);
/* The same with the two standard deviations of paper §3.1: sd_indep (sigma_I) and sd_corr
 * (sigma_C, NULL = all zero), both >= 0.  sigma = sigma_I + sigma_C feeds the moments (§3.2 step
 * 1).  A hit's uniform follows §3.2 steps 2-5: the hit's own Philox uniform above plays
 * z_(Prog,E); z_(E), the same for every ELT and every layer, is one Philox uniform per (trial,
 * event position), counter (k, i_lo, 0xFFFFFFFF, i_hi), word 0; v = sqrt(1 - c^2) Phi^-1(z_P) +
 * c Phi^-1(z_E) with c = (sigma_C/sigma) / |(sigma_I, sigma_C)/sigma|, and z = Phi(v) is inverted
 * (Phi and Phi^-1 in binary32).  sigma_C = 0 gives z = z_P exactly, as ara_add_elt. */
ARA_API ara_status ara_add_elt_corr(ara_ctx* ctx, int32_t yet, int64_t n, const int32_t* event_ids,
                                    const double* mean, const double* sd_indep,
                                    const double* sd_corr, const double* max_exposure,
                                    int32_t* elt_out);
ARA_API ara_status ara_free_elt(ara_ctx* ctx, int32_t elt);

/* Layer (paper §2.1: XELT set plus terms (OccR, OccL, AggR, AggL)) ----------------------------
 * elts[n_elts] (1 <= n_elts <= 64, distinct, same YET): the order fixes the order in which one
 * event's ELT losses are summed.  All terms must be finite and >= 0.  Builds the layer's lookup
 * structure on the device: per catalogue event an 8- (n_elts <= 32) or 16-byte entry (base,
 * ELT bit mask) plus the event's records packed in layer order, sized to stay L2-resident. */
ARA_API ara_status ara_add_layer(ara_ctx* ctx, const int32_t* elts, int32_t n_elts,
                                 double occ_ret, double occ_lim, double agg_ret, double agg_lim,
                                 int32_t* layer_out);
ARA_API ara_status ara_free_layer(ara_ctx* ctx, int32_t layer);

/* Algorithm 1 -------------------------------------------------------------------------------------
 * Year losses of trials [t0, t0+n) of yet under layer -> ylt[0..n-1] (binary64):
 *   Y_i = min(max(S_i - AggR, 0), AggL),  S_i = sum_k min(max(l_ik - OccR, 0), OccL),
 *   l_ik = sum over the layer's ELTs holding event e_ik of max_l * InvCDF_beta(u; alpha, beta).
 * ylt may be host or device memory.  stream == NULL: blocking, on the context's stream, and
 * ARA_ERR_NOT_CONVERGED is returned (with ylt written) if any inversion hit its cap.
 * stream != NULL (a cudaStream_t): asynchronous on that stream, ylt must be device memory, and
 * the convergence count is read later with ara_not_converged(). */
ARA_API ara_status ara_run(ara_ctx* ctx, int32_t yet, int32_t layer, int64_t t0, int64_t n,
                           double* ylt, void* stream);
/* Event-level output beside the aggregate one, in the same pass: as ara_run, and when oep is not
 * NULL also oep[i] = max_k min(max(l_ik - OccR, 0), OccL) (0 for a year without occurrences),
 * the year's largest occurrence loss after occurrence terms (the OEP year table; paper §2.1's
 * occurrence terms applied per event, before the aggregate terms).  The maximum is taken over
 * the binary32 occurrence results, so it is one of them exactly and does not depend on the
 * schedule or on the trial range.  oep (binary64, n entries) must be the same kind of memory as
 * ylt (both host or both device); ARA_ERR_INVALID_ARG otherwise. */
ARA_API ara_status ara_run_ep(ara_ctx* ctx, int32_t yet, int32_t layer, int64_t t0, int64_t n,
                              double* ylt, double* oep, void* stream);
/* Per-occurrence outputs (Algorithm 1 applies the occurrence terms to every event and the
 * aggregate terms to the running year sum after every event; §2.3): for the occurrences of
 * trials [t0, t0+n), indexed by occurrence position - trial_offsets[t0] (so the caller sizes
 * them trial_offsets[t0+n] - trial_offsets[t0]):
 *   olt[q] (binary32) = min(max(l_q - OccR, 0), OccL), the occurrence loss the year sum takes;
 *   inc[q] (binary64) = A(S_q) - A(S_q - o_q), A(S) = min(max(S - AggR, 0), AggL), S_q the
 *     running year sum through occurrence q; A of the trial's last occurrence is its ylt entry
 *     bit for bit, and the increments sum to it up to binary64 rounding.
 * Any of oep, olt, inc may be NULL; all given outputs must be the same kind of memory as ylt.
 * Per-occurrence outputs are written in trial order, so such a call runs the trial-major
 * schedule; inc needs ARA_ACC_FP64 (ARA_ERR_INVALID_ARG otherwise).  With host outputs the
 * library stages them in stream-ordered device memory for the call. */
ARA_API ara_status ara_run_events(ara_ctx* ctx, int32_t yet, int32_t layer, int64_t t0, int64_t n,
                                  double* ylt, double* oep, float* olt, double* inc,
                                  void* stream);
/* Portfolio (paper §2.1: a portfolio groups programs, a program groups layers; Algorithm 1 loops
 * over programs, then layers, then trials): the YLTs of n_layers layers of one YET over trials
 * [t0, t0+n) from one call, ylt[i*n + j] = the year loss of trial t0+j under layers[i], equal bit
 * for bit to ara_run of that layer.  The caller lists the layers of its programs in any order
 * (a layer may appear more than once).  Layers sharing a schedule and lookup-entry width share
 * one batched launch, so a portfolio of many small layers fills the GPU as one large layer does.
 * ylt: n_layers*n binary64, host or device (stream as for ara_run); layers: host array. */
ARA_API ara_status ara_run_portfolio(ara_ctx* ctx, int32_t yet, const int32_t* layers,
                                     int32_t n_layers, int64_t t0, int64_t n, double* ylt,
                                     void* stream);
/* Inversions that hit the iteration cap since the context was created (blocks on its work). */
ARA_API ara_status ara_not_converged(ara_ctx* ctx, int64_t* count);
/* Work counters accumulated by every ara_run since the context was created (blocks on its work):
 * out[0] Newton inversions, out[1] Newton iterations, out[2] continued-fraction terms,
 * out[3] inversions that hit the iteration cap, out[4] hits (ELT records met, sigma = 0 ones
 * included), out[5] kernel launches issued by the library in this process (all contexts),
 * out[6] table evaluations, out[7] records whose table failed certification (those of live ELTs,
 * and of live layers whose tables were built for the layer alone),
 * out[8] surrogate evaluations.  They state the algorithmic work of a launch. */
ARA_API ara_status ara_get_stats(ara_ctx* ctx, int64_t out[9]);

/* Risk measures (paper §2.4) ---------------------------------------------------------------------
 * ylt[n] (host or device, n >= 1, no NaN), rps[m] return periods (> 1, host).  With
 * k = n/rp (rounded up when not an integer; 1 <= k <= n) and the trials ordered by year loss
 * descending, ties by ascending trial index:  pml[q] = the loss at rank k,
 * tvar[q] = the mean of ranks 1..k (binary64 sums).  pml/tvar are host arrays of m values.
 * Ordering by a device LSD radix sort (stable) of the losses' order-preserving bit patterns. */
ARA_API ara_status ara_risk_measures(ara_ctx* ctx, const double* ylt, int64_t n,
                                     const double* rps, int32_t m, double* pml, double* tvar);
/* The same ordering exposed: order[r] = index of the r-th largest entry of ylt[n]; order may be
 * host or device memory (int64). */
ARA_API ara_status ara_rank_ylt(ara_ctx* ctx, const double* ylt, int64_t n, int64_t* order);

/* Trial shards (one process per GPU, trials split into contiguous ranges, one collective):
 * the global PML/TVaR of N_total trials needs, for each return period, the k = N_total/RP
 * largest year losses of all shards.  Each shard sends the k_max largest of its own (k_max for
 * the smallest RP), in ascending trial order; concatenated in shard order they are in global trial
 * order, so ordering them by (loss descending, position ascending) is the global ordering of
 * §2.4 restricted to the candidates, which contain every trial a tail needs.
 *   ara_top_k: out[k] = the k largest entries of ylt[n] (ties: lower index first), in ascending
 *     index order (0 <= k <= n; ylt and out host or device).
 *   ara_risk_measures_n: PML/TVaR as ara_risk_measures over values[n] with the tail counts of
 *     n_total trials, k = n_total/RP; ARA_ERR_INVALID_ARG if some k exceeds n. */
ARA_API ara_status ara_top_k(ara_ctx* ctx, const double* ylt, int64_t n, int64_t k, double* out);
ARA_API ara_status ara_risk_measures_n(ara_ctx* ctx, const double* values, int64_t n,
                                       int64_t n_total, const double* rps, int32_t m, double* pml,
                                       double* tvar);

/* Learned surrogate of InvCDF_beta ----------------------------------------------------------------
 * A 3 -> 64 -> 64 -> 64 -> 1 SiLU network (BF16 weights, FP32 accumulation, tensor-core MMA) maps
 * (ln alpha, ln beta, logit u), normalised over the box alpha, beta in [0.1, 50], to logit x.
 * Training rounds inputs and activations to BF16; evaluation, certification and ara_run carry
 * them as hi + lo BF16 pairs (about 16 significant bits).
 * Trained on the GPU by this library's own forward/backward/Adam kernels on (alpha, beta, u, x)
 * tuples generated by the exact inversion (polished in binary64); then certified: on a 32 x 32 x 64
 * grid of cells over the normalised inputs, each cell's largest |x_net - x| over its corners and
 * cert_samples - 8 further points is recorded.  With ARA_OPT_SURROGATE = 1, ara_run uses the
 * network for a hit only inside the box and where its cell's recorded error is <= eps * mu_beta,
 * mu_beta = alpha / (alpha + beta) being the record's mean loss over its maximum exposure: a served
 * loss is then within eps times the record's mean loss, and a year's sum of served losses within
 * eps of its expected value.  Every other hit falls back to the exact Newton inversion. */
typedef struct {
  int64_t n_samples;    /* training tuples generated (e.g. 50,000,000)                       */
  int64_t steps;        /* Adam steps                                                          */
  int32_t batch;        /* rows per step, a multiple of 128                                    */
  int32_t cert_samples; /* points per certification cell (>= 8)                                */
  float lr, lr_final;   /* cosine schedule from lr to lr_final                                 */
  float eps;            /* accepted error: a cell serves a record when its error in x is     */
                        /* <= eps * mu_beta (eps relative to the record's mean loss)         */
  float reserved;
  uint64_t seed;        /* stream of the training tuples and of the initial weights            */
} ara_surrogate_config;
typedef struct {
  double loss_first, loss_last;   /* mean loss of the first and last 1% of steps                */
  double gen_ms, train_ms, cert_ms;
  double cells_accepted;          /* fraction of certification cells with error <= eps, i.e.    */
                                  /* usable by records of mu_beta = 1 (fewer serve a smaller one) */
  double err_median, err_p99;     /* over cells: recorded |x_net - x|                            */
  int64_t bad_targets;            /* training tuples and certification points whose exact        */
                                  /* inversion reported non-convergence (such a point rejects     */
                                  /* its cell)                                                    */
} ara_surrogate_report;
ARA_API ara_status ara_train_surrogate(ara_ctx* ctx, const ara_surrogate_config* cfg,
                                       ara_surrogate_report* report);
/* Serialised surrogate: header, 8,641 FP32 parameters, 65,536 FP32 cell errors.  save writes at
 * most cap bytes (*bytes receives the size needed); load replaces the context's surrogate. */
ARA_API ara_status ara_save_surrogate(ara_ctx* ctx, void* blob, size_t cap, size_t* bytes);
ARA_API ara_status ara_load_surrogate(ara_ctx* ctx, const void* blob, size_t bytes);
/* Sets the accepted error eps (relative to a record's mean loss, as above) of the loaded surrogate
 * (the cell table is kept). */
ARA_API ara_status ara_set_surrogate_eps(ara_ctx* ctx, float eps);
/* Network evaluation and gradient with caller parameters (host FP32 vector of 8,641 in the order
 * W1[64,3], b1, W2[64,64], b2, W3[64,64], b3, W4[64], b4; NULL = the context's trained network):
 * z[n][3] normalised inputs (host), y[n] outputs (host).  ara_mlp_grad also takes x[n] and the
 * clipped logit targets t[n] (both host) and returns the loss of one training step and its
 * gradient (host, 8,641 values) as the training kernels compute them. */
ARA_API ara_status ara_mlp_eval(ara_ctx* ctx, const float* params, const float* z, int64_t n,
                                float* y);
ARA_API ara_status ara_mlp_grad(ara_ctx* ctx, const float* params, const float* z, const float* x,
                                const float* t, int64_t n, float* grad, double* loss);

/* Verification ------------------------------------------------------------------------------------
 * Re-runs trials [t0, t0+n) with the same device code as ara_run (trial-major, after the same
 * preparation of the layer: tables or start tables as a run of these trials would build them),
 * additionally listing every
 * (trial, event, ELT) hit in event order, then layer order: the trial offset from t0, the event
 * position k within its trial, the layer slot j, the record index in the caller's ELT order, the
 * uniform u, the beta quantile x (NaN for a sigma = 0 record) and the loss.  Host arrays of
 * max_hits entries; *n_hits receives the total (entries beyond max_hits are dropped).  Sized for
 * small runs: the device buffer holds n * (longest trial) * n_elts hits. */
ARA_API ara_status ara_trace_hits(ara_ctx* ctx, int32_t yet, int32_t layer, int64_t t0,
                                  int64_t n, int64_t max_hits, int32_t* hit_trial,
                                  int32_t* hit_k, int32_t* hit_j, int32_t* hit_rec,
                                  float* hit_u, float* hit_x, float* hit_loss, double* ylt,
                                  int64_t* n_hits);

/* Risk measures without any allocation ---------------------------------------------------------
 * The paper has no counterpart: this entry point exists for callers that cannot allocate device
 * memory when they need PML/TVaR (code running inside a pre-sized pool or another allocator that
 * owns the device's memory, real-time loops that must not meet cudaMalloc's implicit
 * synchronisation or its failure under memory pressure, callers holding no ara_ctx).  It computes
 * what ara_risk_measures computes, with the same kernels, and calls no cudaMalloc, cudaFree or
 * other allocating routine.
 *   ylt[n]       device memory of the current device, 1 <= n <= ARA_NOALLOC_MAX_TRIALS;
 *   rps[m]       host array, 0 <= m <= 16, each finite and > 1;
 *   pml, tvar    device memory of the current device, m values each (caller-owned);
 *   stream       cudaStream_t (NULL = the legacy default stream); the call is asynchronous and
 *                the outputs are valid once the stream has passed it.
 * Scratch is a fixed device array inside the library (about 29 MB, held by every GPU that loads
 * the library until the process exits).  Every call looks up that array's device address on the
 * current device; the first call on a device also loads the library's device code there (make it
 * before any stream capture).  Calls share the array: calls whose work overlaps
 * on the GPU race and must not be made.  A YLT holding NaN yields NaN outputs.
 * Returns ARA_ERR_INVALID_ARG for a size above the maximum, host pointers or a bad return
 * period; ARA_ERR_CUDA if a launch fails; ARA_ERR_NO_DEVICE without a current device. */
#define ARA_NOALLOC_MAX_TRIALS (1 << 20)
ARA_API ara_status ara_risk_measures_noalloc(const double* ylt, int64_t n, const double* rps,
                                             int32_t m, double* pml, double* tvar,
                                             void* stream);

/* Continuous-batching service (paper §1: re-pricing layers while the client waits) ------------
 * A server owns one context and one YET staged in it; the ELTs referenced by requests must be
 * staged in the same context before the server is created, and while a server exists the context
 * is used only through it (a worker thread issues all of the context's device work on the
 * server's streams).  A request names a layer (ELT handles in summation order and the four terms,
 * as ara_add_layer), trials [t0, t0 + n_trials) of the YET and up to ARA_MAX_RPS return periods;
 * its result is the YLT of those trials and the PML/TVaR of that YLT, identical to ara_run +
 * ara_risk_measures on the same inputs whatever else is in flight.
 * Scheduling: a pending request is admitted, in arrival order, when fewer than max_inflight
 * requests are running and the device memory it needs (its layer's lookup structure, 16 bytes per
 * catalogue event, its packed records and its YLT) fits hbm_budget; its layer is built then.  Each
 * kernel launch takes the next slice (up to slice_trials trials) of every running request, up to
 * max_batch_trials trials in all, so a request arriving while others run joins the next launch.
 * A finished request's memory is released at once; its results stay in host memory until
 * ara_server_release.  Requests that fail (allocation, invalid layer) are marked FAILED with the
 * status; the server keeps running. */
#define ARA_MAX_RPS 16
#define ARA_REQ_PENDING 0
#define ARA_REQ_RUNNING 1
#define ARA_REQ_DONE 2
#define ARA_REQ_FAILED 3
typedef struct ara_server ara_server;
typedef struct {
  int32_t yet;              /* YET handle of the context                                         */
  int32_t max_inflight;     /* requests running at once (>= 1)                                  */
  int64_t slice_trials;     /* trials of one request per launch (>= 1)                           */
  int64_t max_batch_trials; /* trials per launch over all requests (>= slice_trials)             */
  int64_t max_queue;        /* pending requests beyond which submit returns ARA_ERR_BUSY         */
  int64_t hbm_budget;       /* bytes of device memory requests may hold; 0 = free memory - 4 GiB */
  int32_t use_surrogate;    /* 1: the context's learned surrogate with exact fallback           */
  int32_t inversion;        /* ARA_INV_TABLE or ARA_INV_NEWTON when use_surrogate = 0           */
} ara_server_config;
typedef struct {
  int32_t elts[64];         /* ELT handles, n_elts of them                                       */
  int32_t n_elts;
  int32_t n_rps;            /* 0 .. ARA_MAX_RPS                                                  */
  double occ_ret, occ_lim, agg_ret, agg_lim;
  int64_t t0, n_trials;     /* trial range of the server's YET                                   */
  double rps[ARA_MAX_RPS];  /* return periods, each > 1                                          */
} ara_request;
typedef struct {
  int32_t state;            /* ARA_REQ_*                                                         */
  int32_t error;            /* ara_status of a FAILED request                                    */
  double submit_s, admit_s, done_s; /* seconds since the server was created                      */
  int64_t n_trials;
  double pml[ARA_MAX_RPS], tvar[ARA_MAX_RPS];
} ara_request_status;
typedef struct {
  int64_t completed, failed, launches, pending, active;
  double mean_items_per_launch;   /* requests sharing one launch, averaged                     */
  int64_t hbm_budget, hbm_used;
  double latency_p50_s, latency_p99_s, latency_max_s; /* submit -> done of completed requests */
  double requests_per_s;          /* completed / (last completion - first submission)          */
} ara_server_stats;
ARA_API ara_status ara_server_create(ara_ctx* ctx, const ara_server_config* cfg,
                                     ara_server** out);
/* Queues a request (copied); *ticket identifies it.  ARA_ERR_BUSY when max_queue requests are
 * pending; ARA_ERR_INVALID_ARG / ARA_ERR_BAD_HANDLE for a request that could never run. */
ARA_API ara_status ara_server_submit(ara_server* s, const ara_request* req, int64_t* ticket);
/* Blocks until the request is DONE (ARA_OK) or FAILED (its status), or timeout_s passes
 * (ARA_ERR_BUSY). */
ARA_API ara_status ara_server_wait(ara_server* s, int64_t ticket, double timeout_s);
/* State, timings and risk measures of a request; with ylt != NULL (host, ylt_len >= n_trials) the
 * YLT of a DONE request is copied out. */
ARA_API ara_status ara_server_result(ara_server* s, int64_t ticket, ara_request_status* st,
                                     double* ylt, int64_t ylt_len);
/* Drops a finished request's host results (ARA_ERR_BUSY while it is pending or running). */
ARA_API ara_status ara_server_release(ara_server* s, int64_t ticket);
ARA_API ara_status ara_server_get_stats(ara_server* s, ara_server_stats* out);
/* Stops the worker after the launches in flight, frees the server's memory and gives the context
 * back the stream and the inversion options (ARA_OPT_SURROGATE, ARA_OPT_INVERSION) it had before
 * ara_server_create.  Requests not yet finished are dropped.  NULL-safe. */
ARA_API void ara_server_destroy(ara_server* s);

/* Synchronises the context's stream. */
ARA_API ara_status ara_synchronize(ara_ctx* ctx);
/* Issues all later device work of the context on stream (a cudaStream_t of the context's device;
 * NULL restores the context's own stream).  Blocking calls then synchronise that stream. */
ARA_API ara_status ara_set_stream(ara_ctx* ctx, void* stream);

#ifdef __cplusplus
}
#endif

#endif /* ARA_H */
