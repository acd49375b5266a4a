// ara_serve.cu -- continuous-batching service for real-time layer re-pricing.
//
// The paper's motivating scenario (§1): an underwriter evaluates different contractual terms while
// talking to a client, which routine batch runs cannot serve.  Here the YET and the ELTs stay
// resident on the device; each request names a layer (a subset of the resident ELTs and its
// occurrence/aggregate terms), a trial range and return periods, and receives its YLT, PML and
// TVaR.
//
// Two host threads share the work:
//   builder    admits a pending request when a slot is free and its device memory (layer lookup
//              structure, packed records and tables, YLT, year sums) fits the HBM budget, and
//              builds its layer on its own stream, so that launches in flight never wait for a
//              build; it also frees the memory of finished requests (cudaFree waits for the
//              device, so the launching thread never calls it);
//   worker     each launch takes the next slice (up to slice_trials trials) of every running
//              request, up to max_batch_trials in all, and runs them in one batched kernel launch
//              (each warp reading its own request's layer), so requests that arrive while others
//              run join the very next launch; a request whose last slice has finished gets its
//              PML/TVaR on the device and its YLT copied out, on a stream of its own.
// Results do not depend on batching: a trial's year loss depends only on (trial, layer, seed).
#include <cuda_runtime.h>
#include <math.h>
#include <string.h>

#include <algorithm>
#include <atomic>
#include <chrono>
#include <condition_variable>
#include <deque>
#include <map>
#include <memory>
#include <mutex>
#include <thread>
#include <vector>

#include "ara_ctx.h"

namespace {

using Clock = std::chrono::steady_clock;

struct Request {
  int64_t ticket = 0;
  ara_request req{};
  int32_t state = ARA_REQ_PENDING;
  double submit_s = 0, admit_s = 0, done_s = 0;
  LayerDev layer;          // the request's own layer (not registered in the context)
  bool has_layer = false;
  double* d_ylt = nullptr;
  unsigned long long* d_ysum = nullptr;  // year sums in grid units (band-major schedule)
  bool band = false;
  int64_t next = 0;        // next trial offset to schedule
  int64_t finished = 0;    // trials whose launch has completed
  int64_t bytes = 0;       // device memory held
  std::vector<double> ylt; // host copy once done
  double pml[ARA_MAX_RPS] = {}, tvar[ARA_MAX_RPS] = {};
  ara_status error = ARA_OK;
};

// Device memory of a finished request, freed by the builder thread.
struct Retired {
  LayerDev layer;
  bool has_layer = false;
  double* d_ylt = nullptr;
  unsigned long long* d_ysum = nullptr;
  int64_t bytes = 0;
};

struct Launch {
  cudaEvent_t done = nullptr;
  std::vector<std::pair<int64_t, int64_t>> parts;  // (ticket, trials)
  TrialParams* h_items = nullptr;  // pinned staging
  int64_t* h_begin = nullptr;  // [3 cap]: trial-major warp_begin, band block_begin, trial_begin
  TrialParams* d_items = nullptr;
  int64_t* d_begin = nullptr;
  int cap = 0;
};

}  // namespace

struct ara_server {
  ara_ctx* ctx = nullptr;
  ara_server_config cfg{};
  cudaStream_t stream = nullptr;      // batched trial launches
  cudaStream_t fin_stream = nullptr;  // ordering, tail sums and copies of finished requests
  cudaStream_t build_stream = nullptr;  // layer builds
  std::mutex mu;
  std::condition_variable cv;        // wakes the worker
  std::condition_variable cv_build;  // wakes the builder
  std::thread worker, builder;
  int building = 0;                  // requests whose layer is being built
  std::deque<Retired> retired;
  std::atomic<bool> stop{false};
  Clock::time_point t0;
  int64_t next_ticket = 1;
  std::map<int64_t, std::unique_ptr<Request>> reqs;
  std::deque<int64_t> pending;
  std::vector<int64_t> active;
  int64_t budget = 0, used = 0;
  std::deque<Launch> inflight;
  std::vector<Launch> pool;
  // statistics
  int64_t n_launches = 0, n_items = 0, n_done = 0, n_failed = 0;
  std::vector<double> latencies;
  double first_submit = -1, last_done = 0;
  SortScratch sort;  // the server's own ordering buffers
  int64_t* d_k = nullptr;
  double *d_pml = nullptr, *d_tvar = nullptr;
  // the context's stream and inversion options before the server took it over (restored when
  // the server is destroyed)
  cudaStream_t saved_stream = nullptr;
  int32_t saved_surrogate = 0, saved_inversion = 0;
  bool saved = false;
};

namespace {

double now_s(const ara_server* s) {
  return std::chrono::duration<double>(Clock::now() - s->t0).count();
}

int64_t tail_count_rp(int64_t n, double rp) {
  const double q = (double)n / rp;
  const double r = nearbyint(q);
  int64_t k = (fabs(q - r) <= 1e-9 * fmax(1.0, q)) ? (int64_t)r : (int64_t)ceil(q);
  return std::min<int64_t>(std::max<int64_t>(k, 1), n);
}

// Device bytes a request holds: 16-byte index entries over the catalogue, its packed records
// (BetaRec, record index) with a copy of their tables, its YLT and its exact year sums.
int64_t request_bytes(const ara_server* s, const ara_request& r) {
  const ara_ctx* c = s->ctx;
  const YetDev& Y = c->yets[s->cfg.yet];
  const int64_t C = Y.catalog;
  int64_t recs = 0;
  for (int j = 0; j < r.n_elts; ++j) recs += c->elts[r.elts[j]].n;
  // per packed record: header, caller index, table copy, and the start table of Newton servers
  const int64_t per_rec = (int64_t)(sizeof(BetaRec) + 4 + ara::kTablePieces * sizeof(ara::TablePiece)) +
                          (inversion_mode(c) >= 1 ? (int64_t)(ara::kStartFloats * sizeof(float)) : 0);
  return C * 16 + recs * per_rec + r.n_trials * 16 + (1 << 20);
}

bool ensure_launch_capacity(Launch& L, int n) {
  if (n <= L.cap) return true;
  if (L.h_items) cudaFreeHost(L.h_items);
  if (L.h_begin) cudaFreeHost(L.h_begin);
  if (L.d_items) cudaFree(L.d_items);
  if (L.d_begin) cudaFree(L.d_begin);
  L.h_items = nullptr; L.h_begin = nullptr; L.d_items = nullptr; L.d_begin = nullptr; L.cap = 0;
  if (cudaMallocHost(&L.h_items, sizeof(TrialParams) * n) != cudaSuccess ||
      cudaMallocHost(&L.h_begin, sizeof(int64_t) * 3 * n) != cudaSuccess ||
      cudaMalloc(&L.d_items, sizeof(TrialParams) * n) != cudaSuccess ||
      cudaMalloc(&L.d_begin, sizeof(int64_t) * 3 * n) != cudaSuccess) {
    cudaGetLastError();
    return false;
  }
  L.cap = n;
  return true;
}

// Hands a request's device memory to the builder thread for freeing (server lock held).
void retire(ara_server* s, Request& r) {
  Retired f;
  f.layer = r.layer;
  f.has_layer = r.has_layer;
  f.d_ylt = r.d_ylt;
  f.d_ysum = r.d_ysum;
  f.bytes = r.bytes;
  s->retired.push_back(f);
  r.has_layer = false;
  r.layer = LayerDev();
  r.d_ylt = nullptr;
  r.d_ysum = nullptr;
  r.bytes = 0;
  s->cv_build.notify_one();
}

void fail_request(ara_server* s, Request& r, ara_status st) {
  cudaStreamSynchronize(s->stream);  // no launch in flight may still use its memory
  cudaGetLastError();
  retire(s, r);
  r.error = st;
  r.state = ARA_REQ_FAILED;
  r.done_s = now_s(s);
  s->n_failed++;
}

// PML/TVaR and the host copy of a finished request.  Its last launch has completed, so this runs
// on the finishing stream without waiting for the launches in flight on the trial stream.
void finish(ara_server* s, Request& r) {
  cudaStream_t fs = s->fin_stream;
  const int64_t n = r.req.n_trials;
  cudaError_t e = cudaSuccess;
  const int m = r.req.n_rps;
  if (m > 0) {
    int which = 0;
    e = ara::sort_ylt_desc(r.d_ylt, n, s->sort, &which, fs);
    int64_t ks[ARA_MAX_RPS];
    for (int q = 0; q < m; ++q) ks[q] = tail_count_rp(n, r.req.rps[q]);
    if (e == cudaSuccess)
      e = cudaMemcpyAsync(s->d_k, ks, sizeof(int64_t) * m, cudaMemcpyHostToDevice, fs);
    if (e == cudaSuccess)
      e = ara::launch_tail_sums(r.d_ylt, s->sort.vals[which], n, s->d_k, m, s->d_pml, s->d_tvar,
                                fs);
    if (e == cudaSuccess)
      e = cudaMemcpyAsync(r.pml, s->d_pml, sizeof(double) * m, cudaMemcpyDeviceToHost, fs);
    if (e == cudaSuccess)
      e = cudaMemcpyAsync(r.tvar, s->d_tvar, sizeof(double) * m, cudaMemcpyDeviceToHost, fs);
  }
  r.ylt.resize(n);
  if (e == cudaSuccess)
    e = cudaMemcpyAsync(r.ylt.data(), r.d_ylt, sizeof(double) * n, cudaMemcpyDeviceToHost, fs);
  if (e == cudaSuccess) e = cudaStreamSynchronize(fs);
  if (e != cudaSuccess) {
    cudaGetLastError();
    fail_request(s, r, ARA_ERR_CUDA);
    return;
  }
  retire(s, r);
  r.state = ARA_REQ_DONE;
  r.done_s = now_s(s);
  s->n_done++;
  s->latencies.push_back(r.done_s - r.submit_s);
  s->last_done = r.done_s;
}

// Builder thread: frees retired memory, admits pending requests in arrival order while slots and
// memory allow, and builds their layers on the build stream without holding the server lock.
void builder_loop(ara_server* s) {
  cudaSetDevice(s->ctx->device);
  std::unique_lock<std::mutex> lk(s->mu);
  while (!s->stop.load()) {
    if (!s->retired.empty()) {
      Retired f = s->retired.front();
      s->retired.pop_front();
      lk.unlock();
      // the request's launches and copies are complete: stream-ordered frees, no host wait
      if (f.has_layer) free_layer_on(s->ctx, f.layer, true, s->build_stream);
      if (f.d_ylt) cudaFreeAsync(f.d_ylt, s->build_stream);
      if (f.d_ysum) cudaFreeAsync(f.d_ysum, s->build_stream);
      cudaGetLastError();
      lk.lock();
      s->used -= f.bytes;
      continue;
    }
    if (s->pending.empty() || (int)s->active.size() + s->building >= s->cfg.max_inflight) {
      s->cv_build.wait_for(lk, std::chrono::milliseconds(2));
      continue;
    }
    const int64_t tk = s->pending.front();
    Request& r0 = *s->reqs[tk];
    const int64_t need = request_bytes(s, r0.req);
    if (s->used + need > s->budget && !(s->active.empty() && s->building == 0)) {
      s->cv_build.wait_for(lk, std::chrono::milliseconds(2));  // wait for memory to free
      continue;
    }
    s->pending.pop_front();
    r0.bytes = need;
    s->used += need;
    s->building++;
    const ara_request req = r0.req;
    lk.unlock();
    LayerDev L;
    double* ylt = nullptr;
    unsigned long long* ysum = nullptr;
    bool band = false;
    ara_status st = ara_build_layer(s->ctx, req.elts, req.n_elts, req.occ_ret, req.occ_lim,
                                    req.agg_ret, req.agg_lim, true, s->build_stream, false, true,
                                    &L, inversion_mode(s->ctx) >= 1);
    if (st == ARA_OK) {
      band = uses_band_schedule(s->ctx, L);
      const size_t n = (size_t)std::max<int64_t>(1, req.n_trials);
      if (cudaMallocAsync(&ylt, sizeof(double) * n, s->build_stream) != cudaSuccess ||
          (band && (cudaMallocAsync(&ysum, sizeof(unsigned long long) * n, s->build_stream) !=
                        cudaSuccess ||
                    cudaMemsetAsync(ysum, 0, sizeof(unsigned long long) * n,
                                    s->build_stream) != cudaSuccess)) ||
          cudaStreamSynchronize(s->build_stream) != cudaSuccess) {
        cudaGetLastError();
        st = ARA_ERR_OOM;
      }
    }
    lk.lock();
    s->building--;
    Request& r = *s->reqs[tk];  // a request can be released only once done or failed
    r.layer = L;
    r.has_layer = st == ARA_OK || L.live;
    r.d_ylt = ylt;
    r.d_ysum = ysum;
    if (st != ARA_OK) {
      retire(s, r);
      r.error = st;
      r.state = ARA_REQ_FAILED;
      r.done_s = now_s(s);
      s->n_failed++;
      continue;
    }
    r.band = band;
    r.state = ARA_REQ_RUNNING;
    r.admit_s = now_s(s);
    s->active.push_back(tk);
    s->cv.notify_all();
  }
}

// Collects finished launches; completes requests whose trials are all done.
void reap(ara_server* s, bool block) {
  while (!s->inflight.empty()) {
    Launch& L = s->inflight.front();
    const cudaError_t q = block ? cudaEventSynchronize(L.done) : cudaEventQuery(L.done);
    if (q == cudaErrorNotReady) return;
    for (auto& p : L.parts) {
      auto it = s->reqs.find(p.first);
      if (it == s->reqs.end()) continue;
      Request& r = *it->second;
      if (q != cudaSuccess) {
        if (r.state == ARA_REQ_RUNNING) fail_request(s, r, ARA_ERR_CUDA);
        continue;
      }
      r.finished += p.second;
      if (r.state == ARA_REQ_RUNNING && r.finished >= r.req.n_trials) {
        finish(s, r);
        s->active.erase(std::remove(s->active.begin(), s->active.end(), r.ticket), s->active.end());
      }
    }
    if (q != cudaSuccess) cudaGetLastError();
    s->pool.push_back(L);
    s->inflight.pop_front();
  }
}

// Builds and issues one batched launch over the next slices of the admitted requests.
bool issue(ara_server* s) {
  std::vector<std::pair<Request*, int64_t>> take;
  int64_t total = 0;
  for (int64_t tk : s->active) {
    Request& r = *s->reqs[tk];
    if (r.state != ARA_REQ_RUNNING || r.next >= r.req.n_trials) continue;
    const int64_t n = std::min({s->cfg.slice_trials, r.req.n_trials - r.next,
                                s->cfg.max_batch_trials - total});
    if (n <= 0) break;
    take.emplace_back(&r, n);
    total += n;
  }
  if (take.empty()) return false;
  Launch L;
  if (!s->pool.empty()) {
    L = s->pool.back();
    s->pool.pop_back();
  }
  L.parts.clear();
  if (!L.done && cudaEventCreateWithFlags(&L.done, cudaEventDisableTiming) != cudaSuccess) {
    cudaGetLastError();
    return false;
  }
  if (!ensure_launch_capacity(L, (int)take.size())) {
    for (auto& t : take) fail_request(s, *t.first, ARA_ERR_OOM);
    s->pool.push_back(L);
    return false;
  }
  // batched band-major items first (items [0, kb)), then trial-major ones (items [kb, kb + kt))
  std::stable_partition(take.begin(), take.end(),
                        [](const std::pair<Request*, int64_t>& t) { return t.first->band; });
  const YetDev& Y = s->ctx->yets[s->cfg.yet];
  const int k = (int)take.size();
  const int cap = L.cap;
  int kb = 0, kt = 0;
  int64_t warp = 0, blocks = 0, trials = 0;
  bool band_corr = false;  // some batched band item carries correlated weights
  cudaError_t e = cudaSuccess;
  // a slice whose own grid is many waves deep runs as its own launch (parameters in the constant
  // bank); the others share one batched launch per schedule
  const int64_t big_warps = 12ll * s->ctx->sm_count * 32;  // 12 waves of 32 resident warps per SM
  for (int i = 0; i < k; ++i) {
    Request& r = *take[i].first;
    const int64_t n = take[i].second;
    const LayerDev& Ld = r.layer;
    TrialParams p = make_params(s->ctx, Y, Ld, r.req.t0 + r.next, n, r.d_ylt + r.next);
    const int64_t own_warps = r.band ? (int64_t)p.n_bands * ((n + 31) / 32) : n;
    if (own_warps >= big_warps) {
      if (r.band) {
        p.ysum = r.d_ysum + r.next;
        if (e == cudaSuccess) e = ara::launch_band(p, 2, s->ctx->cfg.precision, 0, s->stream);
      } else if (e == cudaSuccess) {
        e = ara::launch_trial(p, 2, s->ctx->cfg.precision, inversion_mode(s->ctx), false,
                              s->stream);
      }
      r.next += n;
      L.parts.emplace_back(r.ticket, n);
      continue;
    }
    if (r.band) {
      p.tiles = (int32_t)ara::band_tiles(n);
      p.ysum = r.d_ysum + r.next;
      L.h_begin[cap + kb] = blocks;
      L.h_begin[2 * cap + kb] = trials;
      blocks += (int64_t)p.n_bands * p.tiles;
      trials += n;
      band_corr = band_corr || p.corr != nullptr;
      L.h_items[kb++] = p;
    } else {
      // every band item precedes every trial-major one in take, so kb is final here
      L.h_begin[kt] = warp;
      warp += n;
      L.h_items[kb + kt++] = p;
    }
    r.next += n;
    L.parts.emplace_back(r.ticket, n);
  }
  if (e == cudaSuccess && kb + kt > 0)
    e = cudaMemcpyAsync(L.d_items, L.h_items, sizeof(TrialParams) * (kb + kt),
                        cudaMemcpyHostToDevice, s->stream);
  if (e == cudaSuccess && kb + kt > 0)
    e = cudaMemcpyAsync(L.d_begin, L.h_begin, sizeof(int64_t) * 3 * cap, cudaMemcpyHostToDevice,
                        s->stream);
  if (e == cudaSuccess && kb > 0)
    e = ara::launch_band_batch(L.d_items, L.d_begin + cap, L.d_begin + 2 * cap, kb, blocks,
                               trials, 2, band_corr, s->ctx->cfg.precision, s->stream);
  if (e == cudaSuccess && kt > 0)
    e = ara::launch_trial_batch(L.d_items + kb, L.d_begin, kt, warp, 2,
                                s->ctx->cfg.precision, inversion_mode(s->ctx), s->stream);
  if (e == cudaSuccess) e = cudaEventRecord(L.done, s->stream);
  if (e != cudaSuccess) {
    cudaGetLastError();
    for (auto& t : take) fail_request(s, *t.first, ARA_ERR_CUDA);
    s->pool.push_back(L);
    return false;
  }
  s->n_launches++;
  s->n_items += k;
  s->inflight.push_back(L);
  return true;
}

void worker_loop(ara_server* s) {
  cudaSetDevice(s->ctx->device);
  std::unique_lock<std::mutex> lk(s->mu);
  while (!s->stop.load()) {
    reap(s, false);
    // keep two launches in flight: the next one is built while the previous runs
    bool issued = false;
    while (s->inflight.size() < 2 && issue(s)) issued = true;
    if (!issued) {
      if (!s->inflight.empty()) {
        lk.unlock();
        cudaEventSynchronize(s->inflight.front().done);  // host waits on the device, bounded
        lk.lock();
      } else {
        s->cv.wait_for(lk, std::chrono::milliseconds(2));
      }
    }
  }
  reap(s, true);
}

}  // namespace

extern "C" {

ara_status ara_server_create(ara_ctx* ctx, const ara_server_config* cfg, ara_server** out) {
  if (!ctx || !cfg || !out) return ARA_ERR_INVALID_ARG;
  *out = nullptr;
  if (cfg->yet < 0 || cfg->yet >= (int32_t)ctx->yets.size() || !ctx->yets[cfg->yet].live)
    return ARA_ERR_BAD_HANDLE;
  if (ctx->yets[cfg->yet].host) return ARA_ERR_INVALID_ARG;  // a server keeps its YET resident
  if (cfg->slice_trials < 1 || cfg->max_batch_trials < cfg->slice_trials || cfg->max_inflight < 1)
    return ARA_ERR_INVALID_ARG;
  if (cudaSetDevice(ctx->device) != cudaSuccess) return ARA_ERR_CUDA;
  // the server's layers carry the tables of their ELTs (build any that staging deferred), or,
  // for Newton-Halley steps and the surrogate's fallbacks, their start tables
  {
    const ara_status ts = (!cfg->use_surrogate && cfg->inversion == ARA_INV_TABLE)
                              ? ensure_yet_tables(ctx, cfg->yet)
                              : ensure_yet_starts(ctx, cfg->yet);
    if (ts != ARA_OK) return ts;
  }
  ara_server* s = new ara_server();
  s->ctx = ctx;
  s->cfg = *cfg;
  s->t0 = Clock::now();
  size_t free_b = 0, total_b = 0;
  // layer builds and the finishing of requests are on the latency path: their streams have the
  // greatest priority, so their few blocks are scheduled ahead of the batched launches' blocks
  int prio_least = 0, prio_greatest = 0;
  cudaDeviceGetStreamPriorityRange(&prio_least, &prio_greatest);
  if (cudaStreamCreateWithFlags(&s->stream, cudaStreamNonBlocking) != cudaSuccess ||
      cudaStreamCreateWithPriority(&s->fin_stream, cudaStreamNonBlocking, prio_greatest) !=
          cudaSuccess ||
      cudaStreamCreateWithPriority(&s->build_stream, cudaStreamNonBlocking, prio_greatest) !=
          cudaSuccess ||
      cudaMemGetInfo(&free_b, &total_b) != cudaSuccess ||
      cudaMalloc(&s->d_k, sizeof(int64_t) * ARA_MAX_RPS) != cudaSuccess ||
      cudaMalloc(&s->d_pml, sizeof(double) * ARA_MAX_RPS) != cudaSuccess ||
      cudaMalloc(&s->d_tvar, sizeof(double) * ARA_MAX_RPS) != cudaSuccess) {
    cudaGetLastError();
    ara_server_destroy(s);
    return ARA_ERR_CUDA;
  }
  {  // freed request memory stays in the device's pool for the next request's layer
    cudaMemPool_t pool;
    if (cudaDeviceGetDefaultMemPool(&pool, ctx->device) == cudaSuccess) {
      uint64_t keep = UINT64_MAX;
      cudaMemPoolSetAttribute(pool, cudaMemPoolAttrReleaseThreshold, &keep);
    }
    cudaGetLastError();
  }
  s->budget = cfg->hbm_budget > 0 ? cfg->hbm_budget
                                  : std::max<int64_t>(0, (int64_t)free_b - ((int64_t)4 << 30));
  // the server owns the context's device work while it runs
  s->saved_stream = ctx->stream;
  s->saved_surrogate = ctx->cfg.use_surrogate;
  s->saved_inversion = ctx->inversion;
  s->saved = true;
  ara_set_stream(ctx, s->stream);
  if (cfg->use_surrogate) {
    if (ara_set_option(ctx, ARA_OPT_SURROGATE, 1) != ARA_OK) {
      ara_server_destroy(s);
      return ARA_ERR_INVALID_ARG;
    }
  } else {
    ara_set_option(ctx, ARA_OPT_SURROGATE, 0);
    ara_set_option(ctx, ARA_OPT_INVERSION, cfg->inversion);
  }
  // band-major copies of the YET for every band width a request's layer can take (from all
  // ELTs of the YET down to its smallest one), so that no request waits for one to be built
  {
    int64_t total = 0, smallest = -1;
    for (const auto& e : ctx->elts)
      if (e.live && e.yet == cfg->yet) {
        total += e.n;
        if (smallest < 0 || e.n < smallest) smallest = e.n;
      }
    if (total > 0 && !cfg->use_surrogate && cfg->inversion == ARA_INV_TABLE) {
      const int64_t C = ctx->yets[cfg->yet].catalog;
      const int lo = ara::choose_band_log2w(C, total), hi = ara::choose_band_log2w(C, smallest);
      for (int w = lo; w <= hi; w += 2) {
        bool ok = false;
        if (ensure_band_variant(ctx, cfg->yet, w, &ok) != ARA_OK) {
          ara_server_destroy(s);
          return ARA_ERR_OOM;
        }
      }
    }
  }
  // ordering buffers sized for the whole YET
  const int64_t nmax = ctx->yets[cfg->yet].n_trials;
  SortScratch& so = s->sort;
  const int64_t hist_n = 256 * ara::sort_tiles(std::max<int64_t>(1, nmax));
  so.scan_cap = ara::scan_tmp_words(hist_n);
  if (cudaMalloc(&so.keys[0], sizeof(uint64_t) * std::max<int64_t>(1, nmax)) != cudaSuccess ||
      cudaMalloc(&so.keys[1], sizeof(uint64_t) * std::max<int64_t>(1, nmax)) != cudaSuccess ||
      cudaMalloc(&so.vals[0], sizeof(uint32_t) * std::max<int64_t>(1, nmax)) != cudaSuccess ||
      cudaMalloc(&so.vals[1], sizeof(uint32_t) * std::max<int64_t>(1, nmax)) != cudaSuccess ||
      cudaMalloc(&so.hist, sizeof(uint32_t) * hist_n) != cudaSuccess ||
      cudaMalloc(&so.scan_tmp, sizeof(uint32_t) * so.scan_cap) != cudaSuccess ||
      cudaMalloc(&so.digit_flags, sizeof(uint32_t) * 4) != cudaSuccess) {
    cudaGetLastError();
    ara_server_destroy(s);
    return ARA_ERR_OOM;
  }
  so.cap = nmax;
  so.hist_cap = hist_n;
  s->worker = std::thread(worker_loop, s);
  s->builder = std::thread(builder_loop, s);
  *out = s;
  return ARA_OK;
}

ara_status ara_server_submit(ara_server* s, const ara_request* req, int64_t* ticket) {
  if (!s || !req || !ticket) return ARA_ERR_INVALID_ARG;
  const ara_ctx* c = s->ctx;
  if (req->n_elts < 1 || req->n_elts > 64 || req->n_trials < 1 || req->t0 < 0 ||
      req->t0 + req->n_trials > c->yets[s->cfg.yet].n_trials || req->n_rps < 0 ||
      req->n_rps > ARA_MAX_RPS)
    return ARA_ERR_INVALID_ARG;
  for (int q = 0; q < req->n_rps; ++q)
    if (!(req->rps[q] > 1.0)) return ARA_ERR_INVALID_ARG;
  for (int j = 0; j < req->n_elts; ++j) {
    const int32_t h = req->elts[j];
    if (h < 0 || h >= (int32_t)c->elts.size() || !c->elts[h].live || c->elts[h].yet != s->cfg.yet)
      return ARA_ERR_BAD_HANDLE;
  }
  std::lock_guard<std::mutex> lk(s->mu);
  if ((int64_t)s->pending.size() >= s->cfg.max_queue) return ARA_ERR_BUSY;
  auto r = std::make_unique<Request>();
  r->ticket = s->next_ticket++;
  r->req = *req;
  r->submit_s = now_s(s);
  if (s->first_submit < 0) s->first_submit = r->submit_s;
  *ticket = r->ticket;
  s->pending.push_back(r->ticket);
  s->reqs[r->ticket] = std::move(r);
  s->cv_build.notify_one();
  return ARA_OK;
}

ara_status ara_server_result(ara_server* s, int64_t ticket, ara_request_status* st, double* ylt,
                             int64_t ylt_len) {
  if (!s || !st) return ARA_ERR_INVALID_ARG;
  std::lock_guard<std::mutex> lk(s->mu);
  auto it = s->reqs.find(ticket);
  if (it == s->reqs.end()) return ARA_ERR_BAD_HANDLE;
  const Request& r = *it->second;
  st->state = r.state;
  st->error = r.error;
  st->submit_s = r.submit_s;
  st->admit_s = r.admit_s;
  st->done_s = r.done_s;
  st->n_trials = r.req.n_trials;
  for (int q = 0; q < ARA_MAX_RPS; ++q) {
    st->pml[q] = r.pml[q];
    st->tvar[q] = r.tvar[q];
  }
  if (ylt && r.state == ARA_REQ_DONE) {
    if (ylt_len < r.req.n_trials) return ARA_ERR_INVALID_ARG;
    memcpy(ylt, r.ylt.data(), sizeof(double) * r.req.n_trials);
  }
  return ARA_OK;
}

ara_status ara_server_release(ara_server* s, int64_t ticket) {
  if (!s) return ARA_ERR_INVALID_ARG;
  std::lock_guard<std::mutex> lk(s->mu);
  auto it = s->reqs.find(ticket);
  if (it == s->reqs.end()) return ARA_ERR_BAD_HANDLE;
  if (it->second->state != ARA_REQ_DONE && it->second->state != ARA_REQ_FAILED)
    return ARA_ERR_BUSY;
  s->reqs.erase(it);
  return ARA_OK;
}

ara_status ara_server_wait(ara_server* s, int64_t ticket, double timeout_s) {
  if (!s) return ARA_ERR_INVALID_ARG;
  const auto until = Clock::now() + std::chrono::duration_cast<Clock::duration>(
                                        std::chrono::duration<double>(timeout_s));
  for (;;) {
    {
      std::lock_guard<std::mutex> lk(s->mu);
      auto it = s->reqs.find(ticket);
      if (it == s->reqs.end()) return ARA_ERR_BAD_HANDLE;
      const int32_t state = it->second->state;
      if (state == ARA_REQ_DONE) return ARA_OK;
      if (state == ARA_REQ_FAILED) return it->second->error;
    }
    if (Clock::now() >= until) return ARA_ERR_BUSY;
    std::this_thread::sleep_for(std::chrono::microseconds(200));
  }
}

ara_status ara_server_get_stats(ara_server* s, ara_server_stats* out) {
  if (!s || !out) return ARA_ERR_INVALID_ARG;
  std::lock_guard<std::mutex> lk(s->mu);
  memset(out, 0, sizeof *out);
  out->completed = s->n_done;
  out->failed = s->n_failed;
  out->launches = s->n_launches;
  out->mean_items_per_launch = s->n_launches ? (double)s->n_items / (double)s->n_launches : 0.0;
  out->pending = (int64_t)s->pending.size();
  out->active = (int64_t)s->active.size();
  out->hbm_budget = s->budget;
  out->hbm_used = s->used;
  if (!s->latencies.empty()) {
    std::vector<double> l = s->latencies;
    std::sort(l.begin(), l.end());
    auto pct = [&](double q) { return l[std::min(l.size() - 1, (size_t)(q * (l.size() - 1) + 0.5))]; };
    out->latency_p50_s = pct(0.50);
    out->latency_p99_s = pct(0.99);
    out->latency_max_s = l.back();
    const double span = s->last_done - s->first_submit;
    out->requests_per_s = span > 0 ? (double)s->n_done / span : 0.0;
  }
  return ARA_OK;
}

void ara_server_destroy(ara_server* s) {
  if (!s) return;
  s->stop.store(true);
  s->cv.notify_all();
  s->cv_build.notify_all();
  if (s->worker.joinable()) s->worker.join();
  if (s->builder.joinable()) s->builder.join();
  if (s->stream) cudaStreamSynchronize(s->stream);
  for (auto& kv : s->reqs) retire(s, *kv.second);
  for (auto& f : s->retired) {
    if (f.has_layer) free_layer_on(s->ctx, f.layer, true, s->build_stream);
    if (f.d_ylt) cudaFreeAsync(f.d_ylt, s->build_stream);
    if (f.d_ysum) cudaFreeAsync(f.d_ysum, s->build_stream);
  }
  s->retired.clear();
  auto drop = [](Launch& L) {
    if (L.done) cudaEventDestroy(L.done);
    if (L.h_items) cudaFreeHost(L.h_items);
    if (L.h_begin) cudaFreeHost(L.h_begin);
    if (L.d_items) cudaFree(L.d_items);
    if (L.d_begin) cudaFree(L.d_begin);
  };
  for (auto& L : s->inflight) drop(L);
  for (auto& L : s->pool) drop(L);
  for (int b = 0; b < 2; ++b) {
    if (s->sort.keys[b]) cudaFree(s->sort.keys[b]);
    if (s->sort.vals[b]) cudaFree(s->sort.vals[b]);
  }
  if (s->sort.hist) cudaFree(s->sort.hist);
  if (s->sort.scan_tmp) cudaFree(s->sort.scan_tmp);
  if (s->sort.digit_flags) cudaFree(s->sort.digit_flags);
  if (s->d_k) cudaFree(s->d_k);
  if (s->d_pml) cudaFree(s->d_pml);
  if (s->d_tvar) cudaFree(s->d_tvar);
  if (s->ctx) {
    if (s->saved) {  // the context as it was before the server
      ara_set_stream(s->ctx, s->saved_stream == s->ctx->own_stream ? nullptr : s->saved_stream);
      s->ctx->cfg.use_surrogate = s->saved_surrogate;
      s->ctx->inversion = s->saved_inversion;
    } else {
      ara_set_stream(s->ctx, nullptr);
    }
  }
  for (cudaStream_t st : {s->stream, s->fin_stream, s->build_stream}) {
    if (!st) continue;
    cudaStreamSynchronize(st);
    cudaStreamDestroy(st);
  }
  {  // hand the pooled request memory back and restore the pool's default release threshold
    cudaMemPool_t pool;
    if (s->ctx && cudaDeviceGetDefaultMemPool(&pool, s->ctx->device) == cudaSuccess) {
      cudaMemPoolTrimTo(pool, 0);
      uint64_t zero = 0;
      cudaMemPoolSetAttribute(pool, cudaMemPoolAttrReleaseThreshold, &zero);
    }
  }
  cudaGetLastError();
  delete s;
}

}  // extern "C"
