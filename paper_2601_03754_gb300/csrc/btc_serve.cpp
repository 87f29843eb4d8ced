// Serving loop: a continuous-batching request server on top of the plan API.
//
// Requests (factor + refined solve of one system, or a re-solve with a cached
// factor) enter a FIFO queue. `slots` worker threads, each with its own CUDA
// stream, take the oldest request that is admissible — a slot is free and the
// HBM footprint of the request fits in the budget together with everything in
// flight and every cached factor (least-recently-used cached factors are
// evicted to make room) — so requests that arrive while others run are
// admitted as slots and memory free up, and their kernels overlap on the GPU.
//
// Plans are made per (block size, bucket of N): a plan for N_b blocks serves
// every request with N <= N_b. The request is copied into plan-owned staging
// buffers and padded to N_b blocks with identity diagonal blocks, zero
// coupling blocks and a zero right-hand side; the padded system is block
// diagonal between the request's blocks and the pad, the pad's solution is
// exactly zero and the residual norms are the request's (the matrix norm is
// max(||Psi||, 1)). Because the staging pointers of a plan never change, the
// plan's captured refinement graph is replayed by every request it serves.
// Buckets grow geometrically (ratio 2^(1/4), at most 19 % of padding), so a
// random mix of N meets a few dozen plan shapes instead of one per request;
// btc_server_prewarm builds, tunes and captures them ahead of the traffic, and
// plans made on the request path never run tuning trials (they take a
// configuration tuned earlier in the process for the shape, if any). A new
// factor request takes an idle plan of its bucket, else the plan of the
// bucket's least recently used cached factor (dropping that factor), and
// builds a plan only when the bucket has neither. Latency = completion time
// minus submission time (host steady clock).
#include <cuda_runtime.h>

#include <algorithm>
#include <chrono>
#include <cmath>
#include <condition_variable>
#include <deque>
#include <list>
#include <map>
#include <mutex>
#include <thread>
#include <unordered_map>
#include <vector>

#include "../../include/btc.h"

namespace btc {
int fail(int code, const char *fmt, ...);
bool dtype_mixed(int dtype);
// Sets the diagonal entries of nblocks consecutive n x n FP64 blocks to 1 (btc_api.cu).
int set_unit_diagonal(double *D, int64_t nblocks, int n, void *stream);
}

namespace {

using Clock = std::chrono::steady_clock;

struct Job {
  int64_t ticket;
  btc_request req;
  Clock::time_point t_submit;
  int64_t bytes;  // device bytes a fresh plan of this shape needs
};

struct Result {
  bool done = false;
  int status = BTC_OK;
  int iters = 0;
  double relres = 0.0;
  double latency_us = 0.0;
  double queue_us = 0.0;  // submission -> a slot took it
};

// A server plan: a plan for N_b blocks of size n and its staging copies of the
// padded system (D, B, b, x, FP64).
struct SPlan {
  btc_plan_t plan = nullptr;
  int Nb = 0, n = 0;
  double *sD = nullptr, *sB = nullptr, *sb = nullptr, *sx = nullptr;
  int64_t bytes = 0;
};

struct Cached {
  SPlan sp;
  int N, n;  // the request's own size
};

// Bucket of a system size: N itself up to 16, then the smallest ceil(16 * 2^(k/4)) >= N.
int bucket_of(int N) {
  if (N <= 16) return N;
  for (int k = 1;; ++k) {
    const int b = (int)std::ceil(16.0 * std::pow(2.0, k / 4.0) - 1e-9);
    if (b >= N) return b;
  }
}

int64_t staging_bytes(int Nb, int n) { return (2 * (int64_t)Nb * n * n + 2 * (int64_t)Nb * n) * (int64_t)sizeof(double); }

void free_splan(SPlan &sp) {
  if (sp.plan) btc_free(sp.plan);
  for (double *q : {sp.sD, sp.sB, sp.sb, sp.sx})
    if (q) cudaFree(q);
  sp = SPlan();
}

}  // namespace

struct btc_server_s {
  int dtype = BTC_MIXED_F32;
  int slots = 1;
  int64_t budget = 0;
  bool cache = true;
  std::mutex mu;
  std::condition_variable cv_work, cv_done;
  std::deque<Job> queue;
  std::unordered_map<int64_t, Result> results;
  // factor cache: factor id -> plan, LRU order
  std::unordered_map<int64_t, Cached> cached;
  std::list<int64_t> lru;  // front = most recent
  std::unordered_map<int64_t, int> pinned;  // cached factors in use by a running re-solve
  std::multimap<std::pair<int, int>, SPlan> free_plans;  // idle plans by (N_b, n)
  int64_t in_flight_bytes = 0, cached_bytes = 0, free_bytes = 0;
  int64_t next_ticket = 0;
  bool stopping = false;
  std::vector<std::thread> workers;
  std::vector<cudaStream_t> streams;
  // statistics
  std::vector<double> latencies, queue_times, service_times;
  int64_t completed = 0, failed = 0, evictions = 0, cache_hits = 0, cache_misses = 0;
  Clock::time_point t_first, t_last;
  bool any = false;
};

namespace {

// Device bytes of a server plan for bucket Nb: the plan's pools and work vectors, and the staging.
int64_t plan_bytes(int Nb, int n, int dtype) {
  btc_plan_info info;
  if (btc_describe(Nb, n, dtype, &info) != BTC_OK) return -1;
  return info.device_bytes + staging_bytes(Nb, n);
}

// A new server plan for (Nb, n) on `stream`. tune: run the plan's tuning on its first factorization
// (prewarm); otherwise only a configuration remembered for the shape is used.
int make_splan(btc_server_s *s, int Nb, int n, cudaStream_t stream, bool tune, SPlan *out) {
  SPlan sp;
  sp.Nb = Nb;
  sp.n = n;
  sp.bytes = plan_bytes(Nb, n, s->dtype);
  int rc = btc_plan(&sp.plan, Nb, n, s->dtype, stream);
  if (rc) return rc;
  btc_plan_set_autotune(sp.plan, tune ? 1 : 2);
  const size_t nn = (size_t)n * n * sizeof(double);
  cudaError_t e;
  if ((e = cudaMalloc(&sp.sD, nn * Nb)) != cudaSuccess || (e = cudaMalloc(&sp.sB, nn * std::max(Nb - 1, 1))) != cudaSuccess ||
      (e = cudaMalloc(&sp.sb, sizeof(double) * (size_t)Nb * n)) != cudaSuccess ||
      (e = cudaMalloc(&sp.sx, sizeof(double) * (size_t)Nb * n)) != cudaSuccess) {
    free_splan(sp);
    return btc::fail(e == cudaErrorMemoryAllocation ? BTC_ERR_OOM : BTC_ERR_CUDA, "server staging: %s",
                     cudaGetErrorString(e));
  }
  *out = sp;
  return BTC_OK;
}

// Copy a request of N blocks into the staging of sp, padded to sp.Nb blocks (identity diagonal
// blocks, zero coupling blocks; D, B omitted: the right-hand side only, for a re-solve).
int stage_request(const SPlan &sp, int N, const double *D, const double *B, const double *b, cudaStream_t st) {
  const size_t nn = (size_t)sp.n * sp.n, Nb = sp.Nb;
  cudaError_t e = cudaSuccess;
  if (D) {
    if (e == cudaSuccess) e = cudaMemcpyAsync(sp.sD, D, nn * N * sizeof(double), cudaMemcpyDeviceToDevice, st);
    if (e == cudaSuccess && Nb > (size_t)N)
      e = cudaMemsetAsync(sp.sD + nn * N, 0, nn * (Nb - N) * sizeof(double), st);
    if (e == cudaSuccess && N > 1)
      e = cudaMemcpyAsync(sp.sB, B, nn * (N - 1) * sizeof(double), cudaMemcpyDeviceToDevice, st);
    if (e == cudaSuccess && Nb > (size_t)N)
      e = cudaMemsetAsync(sp.sB + nn * (N - 1), 0, nn * (Nb - N) * sizeof(double), st);
    if (e == cudaSuccess && Nb > (size_t)N) {
      const int rc = btc::set_unit_diagonal(sp.sD + nn * N, (int64_t)(Nb - N), sp.n, st);
      if (rc) return rc;
    }
  }
  if (e == cudaSuccess) e = cudaMemcpyAsync(sp.sb, b, sizeof(double) * (size_t)N * sp.n, cudaMemcpyDeviceToDevice, st);
  if (e == cudaSuccess && Nb > (size_t)N)
    e = cudaMemsetAsync(sp.sb + (size_t)N * sp.n, 0, sizeof(double) * (Nb - N) * sp.n, st);
  if (e != cudaSuccess) return btc::fail(BTC_ERR_CUDA, "server staging copy: %s", cudaGetErrorString(e));
  return BTC_OK;
}

// Drop LRU cached factors (not pinned) until `need` more bytes fit. Caller holds mu.
void evict_for(btc_server_s *s, int64_t need) {
  auto total = [&] { return s->in_flight_bytes + s->cached_bytes + s->free_bytes; };
  // idle plans first
  while (total() + need > s->budget && !s->free_plans.empty()) {
    auto it = s->free_plans.begin();
    s->free_bytes -= it->second.bytes;
    free_splan(it->second);
    s->free_plans.erase(it);
  }
  for (auto it = s->lru.end(); total() + need > s->budget && it != s->lru.begin();) {
    --it;
    const int64_t id = *it;
    if (s->pinned.count(id)) continue;
    Cached c = s->cached[id];
    s->cached.erase(id);
    s->cached_bytes -= c.sp.bytes;
    free_splan(c.sp);
    it = s->lru.erase(it);
    ++s->evictions;
  }
}

// The least recently used cached factor (not pinned) whose plan has bucket (Nb, n), or -1. Caller holds mu.
int64_t lru_cached_of_bucket(btc_server_s *s, int Nb, int n) {
  for (auto it = s->lru.rbegin(); it != s->lru.rend(); ++it) {
    const Cached &c = s->cached[*it];
    if (c.sp.Nb == Nb && c.sp.n == n && !s->pinned.count(*it)) return *it;
  }
  return -1;
}

// The oldest admissible job, or -1. Caller holds mu. A re-solve whose cached
// factor is in use by a running re-solve waits (the plan's work vectors,
// norms and stream are per plan, so two solves on one plan would overwrite
// each other's state); the jobs behind it may pass it. Every other job keeps
// FIFO order.
long pick(btc_server_s *s) {
  for (size_t i = 0; i < s->queue.size(); ++i) {
    const Job &j = s->queue[i];
    const bool resolve = j.req.factor_id >= 0 && s->cached.count(j.req.factor_id);
    if (resolve && s->pinned.count(j.req.factor_id)) continue;
    // an idle plan of the bucket, or a cached factor's plan of the bucket that the request may take
    // over, is already counted in the budget
    const bool reuse = !resolve && (s->free_plans.count({bucket_of(j.req.N), j.req.n}) ||
                                    lru_cached_of_bucket(s, bucket_of(j.req.N), j.req.n) >= 0);
    const int64_t need = (resolve || reuse) ? 0 : j.bytes;
    if (s->in_flight_bytes + s->cached_bytes + s->free_bytes + need <= s->budget) return (long)i;
    evict_for(s, need);
    if (s->in_flight_bytes + s->cached_bytes + s->free_bytes + need <= s->budget) return (long)i;
    return -1;  // FIFO: do not overtake a job that does not fit yet
  }
  return -1;
}

void worker(btc_server_s *s, int slot) {
  cudaStream_t stream = s->streams[slot];
  for (;;) {
    Job job;
    SPlan sp;
    bool resolve = false;
    int64_t reserved = 0;
    Clock::time_point t_start;
    {
      std::unique_lock<std::mutex> lk(s->mu);
      long idx = -1;
      s->cv_work.wait(lk, [&] { return (idx = pick(s)) >= 0 || (s->stopping && s->queue.empty()); });
      if (idx < 0) return;  // stopping and the queue is drained
      job = s->queue[idx];
      s->queue.erase(s->queue.begin() + idx);
      t_start = Clock::now();
      const int64_t fid = job.req.factor_id;
      if (fid >= 0 && s->cached.count(fid)) {
        resolve = true;
        sp = s->cached[fid].sp;
        s->pinned[fid]++;
        s->lru.remove(fid);
        s->lru.push_front(fid);
        ++s->cache_hits;
      } else {
        if (fid >= 0) ++s->cache_misses;
        const int Nb = bucket_of(job.req.N);
        auto it = s->free_plans.find({Nb, job.req.n});
        if (it != s->free_plans.end()) {  // an idle plan of the bucket
          sp = it->second;
          s->free_bytes -= sp.bytes;
          s->free_plans.erase(it);
        } else {  // else the plan of the bucket's least recently used cached factor (that factor is dropped)
          const int64_t old = lru_cached_of_bucket(s, Nb, job.req.n);
          if (old >= 0) {
            sp = s->cached[old].sp;
            s->cached.erase(old);
            s->cached_bytes -= sp.bytes;
            s->lru.remove(old);
            ++s->evictions;
          }
        }
        reserved = job.bytes;
        s->in_flight_bytes += reserved;
      }
    }
    int rc = BTC_OK;
    if (!resolve && !sp.plan) rc = make_splan(s, bucket_of(job.req.N), job.req.n, stream, false, &sp);
    if (rc == BTC_OK) rc = btc_plan_set_stream(sp.plan, stream);  // plans move between slots
    int iters = 0;
    double rel = 0.0;
    if (rc == BTC_OK)
      rc = stage_request(sp, job.req.N, resolve ? nullptr : job.req.D, job.req.B, job.req.b, stream);
    if (rc == BTC_OK && !resolve)  // factor with the forward sweep interlaced, then refine
      rc = btc_factor_solve_refined(sp.plan, sp.sD, sp.sB, sp.sb, sp.sx, 1, job.req.tol, job.req.maxit, &iters, &rel);
    else if (rc == BTC_OK)
      rc = btc_solve_refined(sp.plan, sp.sb, sp.sx, 1, job.req.tol, job.req.maxit, &iters, &rel);
    if (rc == BTC_OK || rc == BTC_ERR_NOT_CONVERGED)
      cudaMemcpyAsync(job.req.x, sp.sx, sizeof(double) * (size_t)job.req.N * job.req.n, cudaMemcpyDeviceToDevice,
                      stream);
    cudaStreamSynchronize(stream);
    const auto t_done = Clock::now();
    {
      std::lock_guard<std::mutex> lk(s->mu);
      const int64_t fid = job.req.factor_id;
      if (resolve) {
        if (--s->pinned[fid] == 0) s->pinned.erase(fid);
      } else {
        s->in_flight_bytes -= reserved;
        const int64_t my_id = job.ticket;  // a new factor is cached under its request's ticket
        if (sp.plan && rc == BTC_OK && s->cache) {
          s->cached[my_id] = Cached{sp, job.req.N, job.req.n};
          s->cached_bytes += sp.bytes;
          s->lru.push_front(my_id);
        } else if (sp.plan) {
          s->free_plans.insert({{sp.Nb, sp.n}, sp});
          s->free_bytes += sp.bytes;
        }
      }
      Result &r = s->results[job.ticket];
      r.done = true;
      r.status = rc;
      r.iters = iters;
      r.relres = rel;
      r.latency_us = std::chrono::duration<double, std::micro>(t_done - job.t_submit).count();
      r.queue_us = std::chrono::duration<double, std::micro>(t_start - job.t_submit).count();
      if (rc == BTC_OK) {
        s->latencies.push_back(r.latency_us);
        s->queue_times.push_back(r.queue_us);
        s->service_times.push_back(r.latency_us - r.queue_us);
        ++s->completed;
      } else {
        ++s->failed;
      }
      if (!s->any) s->t_first = job.t_submit;
      s->any = true;
      s->t_last = t_done;
    }
    s->cv_done.notify_all();
    s->cv_work.notify_all();
  }
}

double percentile(std::vector<double> v, double p) {
  if (v.empty()) return 0.0;
  std::sort(v.begin(), v.end());
  const double pos = p / 100.0 * (v.size() - 1);
  const size_t lo = (size_t)pos;
  const size_t hi = std::min(v.size() - 1, lo + 1);
  return v[lo] + (pos - lo) * (v[hi] - v[lo]);
}

}  // namespace

extern "C" {

int btc_server_start(btc_server_t *out, int dtype, int slots, int64_t hbm_budget_bytes, int cache_factors) {
  if (!out || slots < 1 || slots > 64 || hbm_budget_bytes <= 0)
    return btc::fail(BTC_ERR_ARG, "btc_server_start: invalid arguments");
  if (dtype != BTC_F64 && !btc::dtype_mixed(dtype))
    return btc::fail(BTC_ERR_ARG, "btc_server_start: dtype must be BTC_F64 or one of the BTC_MIXED_* dtypes");
  btc_server_s *s = new btc_server_s();
  s->dtype = dtype;
  s->slots = slots;
  s->budget = hbm_budget_bytes;
  s->cache = cache_factors != 0;
  s->streams.resize(slots);
  for (int i = 0; i < slots; ++i)
    if (cudaStreamCreateWithFlags(&s->streams[i], cudaStreamNonBlocking) != cudaSuccess) {
      for (int k = 0; k < i; ++k) cudaStreamDestroy(s->streams[k]);
      delete s;
      return btc::fail(BTC_ERR_CUDA, "btc_server_start: stream creation failed");
    }
  for (int i = 0; i < slots; ++i) s->workers.emplace_back(worker, s, i);
  *out = s;
  return BTC_OK;
}

int btc_server_submit(btc_server_t s, const btc_request *req, int64_t *ticket) {
  if (!s || !req || !req->b || !req->x || req->N < 1 || req->n < 1 || !req->D || (req->N > 1 && !req->B))
    return btc::fail(BTC_ERR_ARG, "btc_server_submit: invalid request");
  const int64_t bytes = plan_bytes(bucket_of(req->N), req->n, s->dtype);
  if (bytes < 0) return btc::fail(BTC_ERR_UNSUPPORTED, "btc_server_submit: block size %d not compiled", req->n);
  if (bytes > s->budget) return btc::fail(BTC_ERR_OOM, "btc_server_submit: request larger than the HBM budget");
  {
    std::lock_guard<std::mutex> lk(s->mu);
    if (s->stopping) return btc::fail(BTC_ERR_ARG, "btc_server_submit: server is stopping");
    Job j;
    j.ticket = s->next_ticket++;
    j.req = *req;
    j.t_submit = Clock::now();
    j.bytes = bytes;
    s->queue.push_back(j);
    s->results[j.ticket] = Result();
    if (ticket) *ticket = j.ticket;
  }
  s->cv_work.notify_one();
  return BTC_OK;
}

int btc_server_poll(btc_server_t s, int64_t ticket, int wait, int *status, int *iters, double *relres,
                    double *latency_us) {
  if (!s) return btc::fail(BTC_ERR_ARG, "btc_server_poll: NULL server");
  std::unique_lock<std::mutex> lk(s->mu);
  auto it = s->results.find(ticket);
  if (it == s->results.end()) return btc::fail(BTC_ERR_ARG, "btc_server_poll: unknown ticket");
  if (wait) s->cv_done.wait(lk, [&] { return s->results[ticket].done; });
  const Result &r = s->results[ticket];
  if (!r.done) return 1;  // still queued or running
  if (status) *status = r.status;
  if (iters) *iters = r.iters;
  if (relres) *relres = r.relres;
  if (latency_us) *latency_us = r.latency_us;
  return BTC_OK;
}

int btc_server_stats(btc_server_t s, btc_server_stats_t *st) {
  if (!s || !st) return btc::fail(BTC_ERR_ARG, "btc_server_stats: NULL argument");
  std::lock_guard<std::mutex> lk(s->mu);
  st->completed = s->completed;
  st->failed = s->failed;
  st->queued = (int64_t)s->queue.size();
  st->evictions = s->evictions;
  st->cache_hits = s->cache_hits;
  st->cache_misses = s->cache_misses;
  st->p50_us = percentile(s->latencies, 50.0);
  st->p99_us = percentile(s->latencies, 99.0);
  st->mean_us = 0.0;
  for (double v : s->latencies) st->mean_us += v;
  if (!s->latencies.empty()) st->mean_us /= (double)s->latencies.size();
  const double span = s->any ? std::chrono::duration<double>(s->t_last - s->t_first).count() : 0.0;
  st->solves_per_s = span > 0 ? (double)s->completed / span : 0.0;
  st->device_bytes = s->in_flight_bytes + s->cached_bytes + s->free_bytes;
  st->p50_queue_us = percentile(s->queue_times, 50.0);
  st->p99_queue_us = percentile(s->queue_times, 99.0);
  st->p50_service_us = percentile(s->service_times, 50.0);
  st->p99_service_us = percentile(s->service_times, 99.0);
  return BTC_OK;
}

int btc_server_reset_stats(btc_server_t s) {
  if (!s) return btc::fail(BTC_ERR_ARG, "btc_server_reset_stats: NULL server");
  std::lock_guard<std::mutex> lk(s->mu);
  s->latencies.clear();
  s->queue_times.clear();
  s->service_times.clear();
  s->completed = s->failed = s->evictions = s->cache_hits = s->cache_misses = 0;
  s->any = false;
  return BTC_OK;
}

int btc_server_footprint(int dtype, int N, int n, int64_t *bytes) {
  if (N < 1 || n < 1 || !bytes) return btc::fail(BTC_ERR_ARG, "btc_server_footprint: invalid arguments");
  const int64_t b = plan_bytes(bucket_of(N), n, dtype);
  if (b < 0) return btc::fail(BTC_ERR_UNSUPPORTED, "btc_server_footprint: block size %d not compiled", n);
  *bytes = b;
  return BTC_OK;
}

int btc_server_prewarm(btc_server_t s, int n, int N_max, int copies) {
  if (!s || n < 1 || N_max < 1 || copies < 1) return btc::fail(BTC_ERR_ARG, "btc_server_prewarm: invalid arguments");
  if (plan_bytes(1, n, s->dtype) < 0)
    return btc::fail(BTC_ERR_UNSUPPORTED, "btc_server_prewarm: block size %d not compiled", n);
  cudaStream_t st = s->streams[0];
  const int top = bucket_of(N_max);
  for (int Nb = 1, made = 0; Nb <= top; made = (made + 1) % copies, Nb = made ? Nb : bucket_of(Nb + 1)) {
    const int64_t bytes = plan_bytes(Nb, n, s->dtype);
    {
      std::lock_guard<std::mutex> lk(s->mu);
      if ((int)s->free_plans.count({Nb, n}) > made) continue;
      if (s->in_flight_bytes + s->cached_bytes + s->free_bytes + bytes > s->budget) break;
      s->in_flight_bytes += bytes;  // reserved while it is built
    }
    SPlan sp;
    int rc = make_splan(s, Nb, n, st, true, &sp);
    // a system that is its own pad (identity blocks, no coupling): one factor + refined solve tunes the
    // plan's launch configuration and captures its refinement graph on the staging pointers
    const size_t nn = (size_t)n * n;
    if (rc == BTC_OK && (cudaMemsetAsync(sp.sD, 0, nn * Nb * sizeof(double), st) != cudaSuccess ||
                         cudaMemsetAsync(sp.sB, 0, nn * std::max(Nb - 1, 1) * sizeof(double), st) != cudaSuccess ||
                         cudaMemsetAsync(sp.sb, 0, sizeof(double) * (size_t)Nb * n, st) != cudaSuccess))
      rc = btc::fail(BTC_ERR_CUDA, "btc_server_prewarm: memset");
    if (rc == BTC_OK) rc = btc::set_unit_diagonal(sp.sD, Nb, n, st);
    int it = 0;
    double rel = 0.0;
    if (rc == BTC_OK) {
      btc_plan_set_stream(sp.plan, st);
      for (int rep = 0; rep < 3 && rc == BTC_OK; ++rep)  // tuning, capture, replay
        rc = btc_factor_solve_refined(sp.plan, sp.sD, sp.sB, sp.sb, sp.sx, 1, 1e-10, 5, &it, &rel);
    }
    cudaStreamSynchronize(st);
    std::lock_guard<std::mutex> lk(s->mu);
    s->in_flight_bytes -= bytes;
    if (rc != BTC_OK) {
      free_splan(sp);
      return rc;
    }
    s->free_plans.insert({{Nb, n}, sp});
    s->free_bytes += sp.bytes;
  }
  return BTC_OK;
}

int btc_server_stop(btc_server_t s) {
  if (!s) return BTC_OK;
  {
    std::lock_guard<std::mutex> lk(s->mu);
    s->stopping = true;
  }
  s->cv_work.notify_all();
  // workers finish every queued job that can still be admitted, then exit
  for (std::thread &t : s->workers) t.join();
  for (auto &kv : s->cached) free_splan(kv.second.sp);
  for (auto &kv : s->free_plans) free_splan(kv.second);
  for (cudaStream_t st : s->streams) cudaStreamDestroy(st);
  delete s;
  return BTC_OK;
}

}  // extern "C"
