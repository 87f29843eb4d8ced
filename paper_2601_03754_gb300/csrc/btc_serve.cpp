// Serving loop: a continuous-batching request server on top of the plan API.
//
// Requests (factor + refined solve of one system, or a re-solve with a cached
// factor) enter a FIFO queue. `slots` worker threads, each with its own CUDA
// stream, take the oldest request that is admissible — a slot is free and the
// HBM footprint of the request fits in the budget together with everything in
// flight and every cached factor (least-recently-used cached factors are
// evicted to make room) — so requests that arrive while others run are
// admitted as slots and memory free up, and their kernels overlap on the GPU.
// Plans (device pools) are reused across requests of the same shape; a plan
// that holds a cached factor is kept until evicted. Latency = completion time
// minus submission time (host steady clock).
#include <cuda_runtime.h>

#include <algorithm>
#include <chrono>
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
};

struct Cached {
  btc_plan_t plan;
  int64_t bytes;
  int N, n;
};

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
  std::multimap<std::pair<int, int>, std::pair<btc_plan_t, int64_t>> free_plans;
  int64_t in_flight_bytes = 0, cached_bytes = 0, free_bytes = 0;
  int64_t next_ticket = 0;
  bool stopping = false;
  std::vector<std::thread> workers;
  std::vector<cudaStream_t> streams;
  // statistics
  std::vector<double> latencies;
  int64_t completed = 0, failed = 0, evictions = 0, cache_hits = 0, cache_misses = 0;
  Clock::time_point t_first, t_last;
  bool any = false;
};

namespace {

int64_t plan_bytes(int N, int n, int dtype) {
  btc_plan_info info;
  if (btc_describe(N, n, dtype, &info) != BTC_OK) return -1;
  return info.device_bytes;
}

// Drop LRU cached factors (not pinned) until `need` more bytes fit. Caller holds mu.
void evict_for(btc_server_s *s, int64_t need) {
  auto total = [&] { return s->in_flight_bytes + s->cached_bytes + s->free_bytes; };
  // idle plans first
  while (total() + need > s->budget && !s->free_plans.empty()) {
    auto it = s->free_plans.begin();
    btc_free(it->second.first);
    s->free_bytes -= it->second.second;
    s->free_plans.erase(it);
  }
  for (auto it = s->lru.end(); total() + need > s->budget && it != s->lru.begin();) {
    --it;
    const int64_t id = *it;
    if (s->pinned.count(id)) continue;
    Cached c = s->cached[id];
    s->cached.erase(id);
    s->cached_bytes -= c.bytes;
    btc_free(c.plan);
    it = s->lru.erase(it);
    ++s->evictions;
  }
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
    const int64_t need = resolve ? 0 : j.bytes;
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
    btc_plan_t plan = nullptr;
    bool resolve = false, fresh = false;
    int64_t reserved = 0;
    {
      std::unique_lock<std::mutex> lk(s->mu);
      long idx = -1;
      s->cv_work.wait(lk, [&] { return (idx = pick(s)) >= 0 || (s->stopping && s->queue.empty()); });
      if (idx < 0) return;  // stopping and the queue is drained
      job = s->queue[idx];
      s->queue.erase(s->queue.begin() + idx);
      const int64_t fid = job.req.factor_id;
      if (fid >= 0 && s->cached.count(fid)) {
        resolve = true;
        plan = s->cached[fid].plan;
        s->pinned[fid]++;
        s->lru.remove(fid);
        s->lru.push_front(fid);
        ++s->cache_hits;
      } else {
        if (fid >= 0) ++s->cache_misses;
        auto it = s->free_plans.find({job.req.N, job.req.n});
        if (it != s->free_plans.end()) {
          plan = it->second.first;
          s->free_bytes -= it->second.second;
          s->free_plans.erase(it);
        }
        reserved = job.bytes;
        s->in_flight_bytes += reserved;
      }
    }
    int rc = BTC_OK;
    if (!resolve && !plan) {
      rc = btc_plan(&plan, job.req.N, job.req.n, s->dtype, stream);
      fresh = rc == BTC_OK;
    }
    (void)fresh;
    if (rc == BTC_OK) rc = btc_plan_set_stream(plan, stream);  // plans move between slots
    int iters = 0;
    double rel = 0.0;
    if (rc == BTC_OK && !resolve)  // factor with the forward sweep interlaced, then refine
      rc = btc_factor_solve_refined(plan, job.req.D, job.req.B, job.req.b, job.req.x, 1, job.req.tol, job.req.maxit,
                                    &iters, &rel);
    else if (rc == BTC_OK)
      rc = btc_solve_refined(plan, job.req.b, job.req.x, 1, job.req.tol, job.req.maxit, &iters, &rel);
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
        if (plan && rc == BTC_OK && s->cache) {
          s->cached[my_id] = Cached{plan, reserved, job.req.N, job.req.n};
          s->cached_bytes += reserved;
          s->lru.push_front(my_id);
        } else if (plan) {
          s->free_plans.insert({{job.req.N, job.req.n}, {plan, reserved}});
          s->free_bytes += reserved;
        }
      }
      Result &r = s->results[job.ticket];
      r.done = true;
      r.status = rc;
      r.iters = iters;
      r.relres = rel;
      r.latency_us = std::chrono::duration<double, std::micro>(t_done - job.t_submit).count();
      if (rc == BTC_OK) {
        s->latencies.push_back(r.latency_us);
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
  const int64_t bytes = plan_bytes(req->N, req->n, s->dtype);
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
  for (auto &kv : s->cached) btc_free(kv.second.plan);
  for (auto &kv : s->free_plans) btc_free(kv.second.first);
  for (cudaStream_t st : s->streams) cudaStreamDestroy(st);
  delete s;
  return BTC_OK;
}

}  // extern "C"
