// Request server: continuous batching of independent TNMC requests on one GPU.
//
// Each request is one disorder realization (seed, L, chi, p, beta, n_samples) of the 2D +-J
// model run through the whole method of Sec. III: couplings (Sec. III.A), environments by
// boundary-MPS contraction (Sec. II.B), tensor-network proposals with their log q (Sec. II.C)
// and the Metropolis filter with the observables of Sec. III.C.  Realizations never interact,
// so the server may group any requests of equal (L, chi) into one batch: a batch runs on a
// pooled context, several batches overlap on the device (each on one of max_inflight CUDA
// streams made when the server starts), and a finished batch frees its slot for the next one
// at once.  The streams are few and fixed so that each can keep a hardware queue of its own:
// streams sharing a queue serialise, and a short batch would wait behind a long one.
//
// Results do not depend on the mix: every draw is keyed by the request's own seed and counted
// by (site, step, chain), a batch samples in fixed-size steps (opts.chunk proposals per chain
// per launch), and the Metropolis kernel stops each realization at its own n_samples, so a
// request gives the same bits alone and in any batch.
//
// One scheduler thread owns every CUDA call of the server; client threads only touch the
// request queue and the result map under the server mutex.
#include <cuda_runtime.h>

#include <algorithm>
#include <atomic>
#include <chrono>
#include <cmath>
#include <condition_variable>
#include <cstring>
#include <deque>
#include <map>
#include <memory>
#include <mutex>
#include <string>
#include <thread>
#include <vector>

#include "../../include/tnmc.h"
#include "ctx_internal.h"
#include "kernels.h"

namespace {

using Clock = std::chrono::steady_clock;

struct Pending {
  int64_t id;
  tnmc_request r;
  double t_submit;
};

// A pooled context and the pinned host buffers its batches read back into.
struct Pooled {
  tnmc_ctx* ctx = nullptr;
  cudaStream_t stream = nullptr;  // the stream of the batch it runs (set per batch)
  cudaEvent_t done = nullptr;
  int L = 0, chi = 0, cap = 0;
  size_t bytes = 0;
  bool busy = false;
  double last_used = 0;
  double* acc_h = nullptr;
  int64_t* clamps_h = nullptr;
  double* logz_h = nullptr;
  long long* stats_h = nullptr;
  unsigned* status_h = nullptr;
  unsigned* rstatus_h = nullptr;
  unsigned char* host = nullptr;   // the pinned block the six pointers above live in
};

size_t host_bytes(int cap) { return (size_t)cap * (8 * tnmc::ACC_SLOTS + 8 + 8 + 32 + 4) + 16; }

struct Batch {
  Pooled* pool = nullptr;
  int slot = -1;                    // index of the server stream it runs on
  std::vector<Pending> reqs;
  double t_start = 0;
};

}  // namespace

struct tnmc_server {
  tnmc_server_opts opts{};
  size_t budget = 0;
  Clock::time_point t0;
  std::thread worker;
  std::mutex mu;
  std::condition_variable cv_work;     // wakes the scheduler: new request or stop
  std::condition_variable cv_result;   // wakes waiting clients: a result arrived
  bool stop = false;
  std::string err;
  int64_t next_id = 1;
  std::deque<Pending> queue;           // submitted, not yet taken by the scheduler
  std::map<int64_t, tnmc_result> results;
  std::deque<int64_t> result_order;    // completion order for polling
  int64_t open_requests = 0;           // submitted and not yet completed
  // scheduler-owned (no lock)
  std::vector<std::unique_ptr<Pooled>> pool;
  std::vector<Batch> inflight;
  std::vector<cudaStream_t> streams;   // one per in-flight slot
  std::vector<bool> stream_busy;
  cudaStream_t reaper = nullptr;       // evicted contexts are freed on it; nothing waits on it
  size_t bytes_in_use = 0;
  // statistics (read under mu)
  int64_t st_submitted = 0, st_completed = 0, st_failed = 0, st_batches = 0, st_created = 0, st_evicted = 0;
  size_t st_peak_bytes = 0;
  int64_t st_launches = 0;

  double now() const { return std::chrono::duration<double>(Clock::now() - t0).count(); }
};

namespace {

tnmc_status status_from_word(unsigned st) {
  if (st & tnmc::ST_NUMERIC) return TNMC_ERR_NUMERIC;
  if (st & tnmc::ST_TIMEOUT) return TNMC_ERR_TIMEOUT;
  if (st & tnmc::ST_ARG) return TNMC_ERR_ARG;
  return TNMC_OK;
}

tnmc_opts ctx_opts(const tnmc_server* s, cudaStream_t st) {
  tnmc_opts o{};
  o.precision = s->opts.precision;
  o.n_chains = s->opts.n_chains;
  o.n_therm = s->opts.n_therm;
  o.stream = reinterpret_cast<void*>(st);
  return o;
}

// Realizations per batch for (L, chi): opts.max_batch, halved until one context fits the budget.
int capacity_for(const tnmc_server* s, int L, int chi, size_t* bytes) {
  tnmc_opts o = ctx_opts(s, nullptr);
  int cap = s->opts.max_batch;
  size_t b = tnmc_estimate_device_bytes(L, cap, chi, &o, s->opts.chunk);
  while (cap > 1 && b > s->budget) {
    cap = (cap + 1) / 2;
    b = tnmc_estimate_device_bytes(L, cap, chi, &o, s->opts.chunk);
  }
  *bytes = b;
  return cap;
}

void free_pooled(tnmc_server* s, Pooled* p) {
  if (p->ctx) tnmc::ctx_release(p->ctx, s->reaper);  // its last batch has completed
  if (p->done) cudaEventDestroy(p->done);
  tnmc::pinned_put(p->host, host_bytes(p->cap));
  s->bytes_in_use -= p->bytes;
}

void evict(tnmc_server* s, size_t idx) {
  free_pooled(s, s->pool[idx].get());
  s->pool.erase(s->pool.begin() + (long)idx);
  std::lock_guard<std::mutex> lk(s->mu);
  ++s->st_evicted;
}

// A new pooled context for (L, chi) with the given capacity; nullptr and *why on failure.
Pooled* create_pooled(tnmc_server* s, int L, int chi, int cap, size_t bytes, cudaStream_t stream, tnmc_status* why,
                      std::string* msg) {
  auto p = std::make_unique<Pooled>();
  p->L = L; p->chi = chi; p->cap = cap; p->bytes = bytes;
  p->stream = stream;
  cudaError_t e = cudaEventCreateWithFlags(&p->done, cudaEventDisableTiming);
  if (e == cudaSuccess) {
    p->host = static_cast<unsigned char*>(tnmc::pinned_get(host_bytes(cap)));
    if (!p->host) e = cudaErrorMemoryAllocation;
  }
  if (e == cudaSuccess) {  // one pinned block: accumulators, log Z, clamps, build statistics, status
    p->acc_h = reinterpret_cast<double*>(p->host);
    p->logz_h = p->acc_h + (size_t)cap * tnmc::ACC_SLOTS;
    p->clamps_h = reinterpret_cast<int64_t*>(p->logz_h + cap);
    p->stats_h = reinterpret_cast<long long*>(p->clamps_h + cap);
    p->status_h = reinterpret_cast<unsigned*>(p->stats_h + 4 * (size_t)cap);
    p->rstatus_h = p->status_h + 1;
  }
  if (e != cudaSuccess) {
    cudaGetLastError();
    *why = TNMC_ERR_OOM;
    *msg = std::string("server context resources: ") + cudaGetErrorString(e);
    s->bytes_in_use += p->bytes;
    free_pooled(s, p.get());
    return nullptr;
  }
  // placeholder inputs: every batch overwrites couplings, seeds and temperatures
  std::vector<int8_t> J((size_t)2 * L * (L - 1) * cap, 1);
  std::vector<double> beta(cap, 1.0);
  std::vector<uint64_t> seeds(cap, 0);
  tnmc_opts o = ctx_opts(s, p->stream);
  tnmc_status st = tnmc_create(L, cap, J.data(), beta.data(), seeds.data(), chi, &o, &p->ctx);
  s->bytes_in_use += p->bytes;
  if (st != TNMC_OK) {
    *why = st;
    *msg = std::string("server context: ") + tnmc_last_error(nullptr);
    free_pooled(s, p.get());
    return nullptr;
  }
  const size_t actual = tnmc_device_bytes(p->ctx);
  if (actual > p->bytes) { s->bytes_in_use += actual - p->bytes; p->bytes = actual; }
  s->pool.push_back(std::move(p));
  std::lock_guard<std::mutex> lk(s->mu);
  ++s->st_created;
  s->st_peak_bytes = std::max(s->st_peak_bytes, s->bytes_in_use);
  return s->pool.back().get();
}

void finish_request(tnmc_server* s, const Pending& q, tnmc_status st, int batch_size, double t_start,
                    const Pooled* p, int k) {
  tnmc_result r{};
  r.id = q.id;
  r.status = st;
  r.batch_size = batch_size;
  r.t_submit = q.t_submit;
  r.t_start = t_start;
  r.t_done = s->now();
  r.obs.status = st;
  if (p && st == TNMC_OK) {
    tnmc::obs_from_acc(p->acc_h + (size_t)k * tnmc::ACC_SLOTS, p->clamps_h[k], &r.obs);
    r.log_z = p->logz_h[k];
    for (int j = 0; j < 4; ++j) r.build_stats[j] = p->stats_h[4 * k + j];
  }
  std::lock_guard<std::mutex> lk(s->mu);
  s->results[q.id] = r;
  s->result_order.push_back(q.id);
  --s->open_requests;
  ++s->st_completed;
  if (st != TNMC_OK) ++s->st_failed;
}

// Queue one batch on pooled context p: couplings, environments, sampling in fixed steps of
// opts.chunk proposals per chain, Metropolis, result copies, completion event.
tnmc_status enqueue_batch(tnmc_server* s, Pooled* p, const std::vector<Pending>& reqs) {
  const int n = (int)reqs.size();
  std::vector<uint64_t> seeds(n);
  std::vector<double> betas(n), ps(n);
  std::vector<int> lims(n);
  int n_max = 0;
  for (int k = 0; k < n; ++k) {
    seeds[k] = reqs[k].r.seed; betas[k] = reqs[k].r.beta; ps[k] = reqs[k].r.p; lims[k] = reqs[k].r.n_samples;
    n_max = std::max(n_max, lims[k]);
  }
  tnmc_ctx* c = p->ctx;
  const int64_t l0 = tnmc_launch_count(c);
  tnmc_status st = tnmc::ctx_begin_batch(c, n, seeds.data(), betas.data(), ps.data(), lims.data());
  if (!st) st = tnmc_build_env(c, nullptr);
  const int C = s->opts.chunk;
  for (int64_t step0 = 0; !st && step0 < n_max; step0 += C) {
    const int m = (int)std::min<int64_t>(C, n_max - step0);
    st = tnmc_propose(c, m, (uint64_t)step0, nullptr, nullptr, nullptr);
    if (!st) st = tnmc_accept(c, nullptr, nullptr);
  }
  if (!st) st = tnmc::ctx_enqueue_readback(c, p->acc_h, p->clamps_h, p->logz_h, p->stats_h, p->status_h,
                                           p->rstatus_h);
  if (!st && cudaEventRecord(p->done, p->stream) != cudaSuccess) { cudaGetLastError(); st = TNMC_ERR_CUDA; }
  std::lock_guard<std::mutex> lk(s->mu);
  s->st_launches += tnmc_launch_count(c) - l0;
  return st;
}

// Retire finished batches; true if any finished.
bool retire(tnmc_server* s) {
  bool any = false;
  for (size_t i = 0; i < s->inflight.size();) {
    Batch& b = s->inflight[i];
    const cudaError_t e = cudaEventQuery(b.pool->done);
    if (e == cudaErrorNotReady) { ++i; continue; }
    any = true;
    // a timeout or argument error taints the whole batch; a numeric failure only the
    // realizations whose proposals met it
    tnmc_status st = TNMC_OK;
    if (e != cudaSuccess) { cudaGetLastError(); st = TNMC_ERR_CUDA; }
    else st = status_from_word(*b.pool->status_h & ~(unsigned)tnmc::ST_NUMERIC);
    const int bs = (int)b.reqs.size();
    for (int k = 0; k < bs; ++k) {
      tnmc_status sk = st;
      if (sk == TNMC_OK) sk = status_from_word(b.pool->rstatus_h[k]);
      finish_request(s, b.reqs[k], sk, bs, b.t_start, b.pool, k);
    }
    b.pool->busy = false;
    b.pool->last_used = s->now();
    s->stream_busy[(size_t)b.slot] = false;
    if (st != TNMC_OK) {  // a context whose batch failed is not reused
      for (size_t j = 0; j < s->pool.size(); ++j)
        if (s->pool[j].get() == b.pool) { evict(s, j); break; }
    }
    s->inflight.erase(s->inflight.begin() + (long)i);
  }
  if (any) s->cv_result.notify_all();
  return any;
}

// Launch batches while slots are free.  `local` holds the requests taken from the queue, in
// submission order.  Returns true if anything launched or failed.
bool schedule(tnmc_server* s, std::deque<Pending>& local, bool& waiting_linger) {
  bool progress = false;
  waiting_linger = false;
  while (!local.empty() && (int)s->inflight.size() < s->opts.max_inflight) {
    if (s->streams.empty()) {  // the server could not make a stream: refuse
      const Pending q = local.front();
      local.pop_front();
      finish_request(s, q, TNMC_ERR_CUDA, 0, s->now(), nullptr, 0);
      s->cv_result.notify_all();
      progress = true;
      continue;
    }
    // the bucket of the oldest request goes first
    const int L = local.front().r.L, chi = local.front().r.chi;
    size_t bytes = 0;
    const int cap = capacity_for(s, L, chi, &bytes);
    std::vector<size_t> idx;
    for (size_t i = 0; i < local.size() && (int)idx.size() < cap; ++i)
      if (local[i].r.L == L && local[i].r.chi == chi) idx.push_back(i);
    if ((int)idx.size() < cap && s->opts.linger_us > 0 &&
        s->now() - local.front().t_submit < 1e-6 * s->opts.linger_us) {
      waiting_linger = true;
      break;
    }
    // a context: the smallest idle one of this key that holds the batch, else a new one sized
    // to the batch (next power of two, at most cap) within the budget
    int slot = 0;
    while (slot < (int)s->streams.size() && s->stream_busy[(size_t)slot]) ++slot;
    if (slot == (int)s->streams.size()) break;
    Pooled* p = nullptr;
    const int need = (int)idx.size();
    for (auto& q : s->pool)
      if (!q->busy && q->L == L && q->chi == chi && q->cap >= need && (!p || q->cap < p->cap)) p = q.get();
    int cap_new = 1;
    while (cap_new < need) cap_new *= 2;
    if (cap_new > cap) cap_new = cap;
    if (!p && cap_new < cap) {
      tnmc_opts o = ctx_opts(s, nullptr);
      bytes = tnmc_estimate_device_bytes(L, cap_new, chi, &o, s->opts.chunk);
    }
    if (!p && bytes > s->budget) {  // even one realization can never fit: refuse at once
      const Pending q = local.front();
      local.pop_front();
      {
        std::lock_guard<std::mutex> lk(s->mu);
        s->err = "request needs " + std::to_string(bytes) + " device bytes; the budget is " +
                 std::to_string(s->budget);
      }
      finish_request(s, q, TNMC_ERR_OOM, 0, s->now(), nullptr, 0);
      s->cv_result.notify_all();
      progress = true;
      continue;
    }
    if (!p) {
      size_t busy_bytes = 0;
      for (auto& q : s->pool)
        if (q->busy) busy_bytes += q->bytes;
      if (busy_bytes + bytes > s->budget && !s->inflight.empty()) break;  // only a finishing batch can make room
      while (s->bytes_in_use + bytes > s->budget) {  // evict idle contexts, least recently used first
        long victim = -1;
        for (size_t j = 0; j < s->pool.size(); ++j)
          if (!s->pool[j]->busy && (victim < 0 || s->pool[j]->last_used < s->pool[(size_t)victim]->last_used))
            victim = (long)j;
        if (victim < 0) break;
        evict(s, (size_t)victim);
      }
      if (s->bytes_in_use + bytes > s->budget) {
        if (!s->inflight.empty()) break;  // wait for a batch to finish and free its context
        // nothing runs and nothing is idle: the request can never fit
        const Pending q = local.front();
        local.pop_front();
        {
          std::lock_guard<std::mutex> lk(s->mu);
          s->err = "request needs " + std::to_string(bytes) + " device bytes; the budget is " +
                   std::to_string(s->budget);
        }
        finish_request(s, q, TNMC_ERR_OOM, 0, s->now(), nullptr, 0);
        s->cv_result.notify_all();
        progress = true;
        continue;
      }
      tnmc_status why = TNMC_OK;
      std::string msg;
      p = create_pooled(s, L, chi, cap_new, bytes, s->streams[(size_t)slot], &why, &msg);
      if (!p) {
        if (!s->inflight.empty() && why == TNMC_ERR_OOM) break;  // retry once memory frees up
        const Pending q = local.front();
        local.pop_front();
        {
          std::lock_guard<std::mutex> lk(s->mu);
          s->err = msg;
        }
        finish_request(s, q, why, 0, s->now(), nullptr, 0);
        s->cv_result.notify_all();
        progress = true;
        continue;
      }
    }
    Batch b;
    b.pool = p;
    b.slot = slot;
    b.t_start = s->now();
    p->stream = s->streams[(size_t)slot];
    tnmc::ctx_set_stream(p->ctx, p->stream);
    s->stream_busy[(size_t)slot] = true;
    for (size_t i : idx) b.reqs.push_back(local[i]);
    for (size_t j = idx.size(); j-- > 0;) local.erase(local.begin() + (long)idx[j]);
    p->busy = true;
    const tnmc_status st = enqueue_batch(s, p, b.reqs);
    progress = true;
    if (st != TNMC_OK) {
      {
        std::lock_guard<std::mutex> lk(s->mu);
        s->err = std::string("batch launch: ") + tnmc_last_error(p->ctx);
      }
      cudaStreamSynchronize(p->stream);
      cudaGetLastError();
      s->stream_busy[(size_t)slot] = false;
      for (const Pending& q : b.reqs) finish_request(s, q, st, (int)b.reqs.size(), b.t_start, nullptr, 0);
      for (size_t j = 0; j < s->pool.size(); ++j)
        if (s->pool[j].get() == p) { evict(s, j); break; }
      s->cv_result.notify_all();
      continue;
    }
    {
      std::lock_guard<std::mutex> lk(s->mu);
      ++s->st_batches;
    }
    s->inflight.push_back(std::move(b));
  }
  return progress;
}

void worker_main(tnmc_server* s) {
  cudaSetDevice(s->opts.device);
  for (int k = 0; k < s->opts.max_inflight; ++k) {
    cudaStream_t st = nullptr;
    if (cudaStreamCreateWithFlags(&st, cudaStreamNonBlocking) != cudaSuccess) { cudaGetLastError(); break; }
    s->streams.push_back(st);
    s->stream_busy.push_back(false);
  }
  if (cudaStreamCreateWithFlags(&s->reaper, cudaStreamNonBlocking) != cudaSuccess) {
    cudaGetLastError();
    s->reaper = nullptr;
  }
  if (s->streams.empty()) {  // no stream at all: every request fails
    std::lock_guard<std::mutex> lk(s->mu);
    s->err = "could not create a CUDA stream";
  }
  std::deque<Pending> local;
  for (;;) {
    {
      std::unique_lock<std::mutex> lk(s->mu);
      while (!s->queue.empty()) { local.push_back(s->queue.front()); s->queue.pop_front(); }
      if (s->stop && local.empty() && s->inflight.empty()) break;
    }
    const bool retired = retire(s);
    bool lingering = false;
    const bool launched = schedule(s, local, lingering);
    if (retired || launched) continue;
    std::unique_lock<std::mutex> lk(s->mu);
    if (!s->queue.empty() || (s->stop && local.empty() && s->inflight.empty())) continue;
    if (s->inflight.empty() && !lingering && local.empty())
      s->cv_work.wait(lk, [s] { return s->stop || !s->queue.empty(); });
    else
      s->cv_work.wait_for(lk, std::chrono::microseconds(100));
  }
  while (!s->pool.empty()) evict(s, s->pool.size() - 1);
  for (cudaStream_t st : s->streams) {
    cudaStreamSynchronize(st);
    cudaStreamDestroy(st);
  }
  if (s->reaper) {
    cudaStreamSynchronize(s->reaper);
    cudaStreamDestroy(s->reaper);
  }
}

}  // namespace

extern "C" {

tnmc_status tnmc_server_create(const tnmc_server_opts* opts, tnmc_server** out) {
  if (!opts || !out) return TNMC_ERR_ARG;
  *out = nullptr;
  if (opts->precision < 0 || opts->precision > 3 || opts->n_chains < 1 || opts->n_chains > 8 ||
      opts->n_therm < 0 || opts->chunk < 1 || opts->max_batch < 1 || opts->max_inflight < 1 ||
      opts->linger_us < 0)
    return TNMC_ERR_ARG;
  int ndev = 0;
  if (cudaGetDeviceCount(&ndev) != cudaSuccess || opts->device < 0 || opts->device >= ndev) {
    cudaGetLastError();
    return TNMC_ERR_ARG;
  }
  auto s = new tnmc_server();
  s->opts = *opts;
  s->t0 = Clock::now();
  s->budget = opts->mem_budget;
  if (s->budget == 0) {
    int prev = 0;
    cudaGetDevice(&prev);
    cudaSetDevice(opts->device);
    size_t fr = 0, tot = 0;
    const cudaError_t e = cudaMemGetInfo(&fr, &tot);
    cudaSetDevice(prev);
    if (e != cudaSuccess) { cudaGetLastError(); delete s; return TNMC_ERR_CUDA; }
    s->budget = fr / 10 * 9;
  }
  s->worker = std::thread(worker_main, s);
  *out = s;
  return TNMC_OK;
}

tnmc_status tnmc_server_submit(tnmc_server* s, const tnmc_request* req, int64_t* id_out) {
  if (!s || !req || !id_out) return TNMC_ERR_ARG;
  const tnmc_request& r = *req;
  const int chi_max = s->opts.precision == TNMC_FP64 ? 32 : 64;
  if (r.L < 2 || r.L > 4096 || r.chi < 1 || r.chi > chi_max || !(r.p >= 0.0 && r.p <= 1.0) ||
      !(r.beta > 0.0) || !std::isfinite(r.beta) || r.n_samples < 1) {
    std::lock_guard<std::mutex> lk(s->mu);
    s->err = "request: need 2 <= L <= 4096, 1 <= chi <= 64 (32 in FP64), 0 <= p <= 1, finite beta > 0, n_samples >= 1";
    return TNMC_ERR_ARG;
  }
  {
    std::lock_guard<std::mutex> lk(s->mu);
    if (s->stop) { s->err = "server is stopping"; return TNMC_ERR_STATE; }
    Pending q{s->next_id++, r, s->now()};
    *id_out = q.id;
    s->queue.push_back(q);
    ++s->open_requests;
    ++s->st_submitted;
  }
  s->cv_work.notify_one();
  return TNMC_OK;
}

int tnmc_server_poll(tnmc_server* s, tnmc_result* out_host, int max_results) {
  if (!s || !out_host || max_results < 1) return 0;
  std::lock_guard<std::mutex> lk(s->mu);
  int got = 0;
  while (got < max_results && !s->result_order.empty()) {
    const int64_t id = s->result_order.front();
    s->result_order.pop_front();
    auto it = s->results.find(id);
    if (it == s->results.end()) continue;  // already taken by tnmc_server_wait
    out_host[got++] = it->second;
    s->results.erase(it);
  }
  return got;
}

tnmc_status tnmc_server_wait(tnmc_server* s, int64_t id, double timeout_s, tnmc_result* out_host) {
  if (!s || !out_host) return TNMC_ERR_ARG;
  std::unique_lock<std::mutex> lk(s->mu);
  if (id < 1 || id >= s->next_id) { s->err = "unknown request id"; return TNMC_ERR_ARG; }
  const auto deadline = Clock::now() + std::chrono::duration_cast<Clock::duration>(
                                           std::chrono::duration<double>(timeout_s < 0 ? 1e9 : timeout_s));
  while (s->results.find(id) == s->results.end()) {
    if (s->cv_result.wait_until(lk, deadline) == std::cv_status::timeout &&
        s->results.find(id) == s->results.end()) {
      s->err = "request not finished within the timeout (or already collected)";
      return TNMC_ERR_TIMEOUT;
    }
  }
  auto it = s->results.find(id);
  *out_host = it->second;
  s->results.erase(it);
  return TNMC_OK;
}

tnmc_status tnmc_server_drain(tnmc_server* s, double timeout_s) {
  if (!s) return TNMC_ERR_ARG;
  std::unique_lock<std::mutex> lk(s->mu);
  const auto deadline = Clock::now() + std::chrono::duration_cast<Clock::duration>(
                                           std::chrono::duration<double>(timeout_s < 0 ? 1e9 : timeout_s));
  while (s->open_requests > 0) {
    if (s->cv_result.wait_until(lk, deadline) == std::cv_status::timeout && s->open_requests > 0) {
      s->err = "requests still open at the timeout";
      return TNMC_ERR_TIMEOUT;
    }
  }
  return TNMC_OK;
}

tnmc_status tnmc_server_stats(tnmc_server* s, int64_t* out_host) {
  if (!s || !out_host) return TNMC_ERR_ARG;
  std::lock_guard<std::mutex> lk(s->mu);
  out_host[0] = s->st_submitted;
  out_host[1] = s->st_completed;
  out_host[2] = s->st_failed;
  out_host[3] = s->st_batches;
  out_host[4] = s->st_created;
  out_host[5] = s->st_evicted;
  out_host[6] = (int64_t)s->st_peak_bytes;
  out_host[7] = s->st_launches;
  return TNMC_OK;
}

const char* tnmc_server_last_error(tnmc_server* s) {
  static thread_local std::string copy;
  if (!s) return "NULL server";
  std::lock_guard<std::mutex> lk(s->mu);
  copy = s->err;
  return copy.c_str();
}

double tnmc_server_now(tnmc_server* s) { return s ? s->now() : 0.0; }

tnmc_status tnmc_server_destroy(tnmc_server* s) {
  if (!s) return TNMC_OK;
  {
    std::lock_guard<std::mutex> lk(s->mu);
    s->stop = true;
  }
  s->cv_work.notify_all();
  if (s->worker.joinable()) s->worker.join();
  delete s;
  return TNMC_OK;
}

}  // extern "C"
