// Batched plans: many independent block-tridiagonal systems of different
// (N, n) factored and solved together. Instances are grouped by padded block
// size; each group runs ONE persistent dataflow launch for the factor and one
// for the solve, whose work items are the (instance, node) eliminations of all
// instances in level order. Each item waits only for the producer nodes of its
// own instance (bounded waits), so short instances finish early and long ones
// keep the SMs busy.
#include <cuda_runtime.h>

#include <algorithm>
#include <cstring>
#include <map>
#include <string>
#include <vector>

#include "../../include/btc.h"
#include "btc_factor.cuh"
#include "btc_internal.h"
#include "btc_kernels.h"
#include "btc_runtime.h"
#include "btc_solve.cuh"

namespace btc {

// Per global node of a group: its instance and block row.
struct BatchNode {
  int32_t inst;
  int32_t row;
};

// Per instance: the caller's right-hand side / solution (FP64 or FP32).
struct BatchVec {
  const void *b;
  void *x;
};

// y (group layout [node][np]) <- b of each node's instance (type S), zero padding.
template <typename T, typename S>
__global__ void k_batch_pack(T *y, const BatchNode *nodes, const InstDesc *inst, const BatchVec *vec, int np) {
  const BatchNode nd = nodes[blockIdx.x];
  const int n = inst[nd.inst].n;
  const S *b = reinterpret_cast<const S *>(vec[nd.inst].b);
  for (int r = threadIdx.x; r < np; r += blockDim.x)
    y[(size_t)blockIdx.x * np + r] = r < n ? (T)b[(size_t)nd.row * n + r] : T(0);
}

// x of each node's instance <- y (or += y when accumulate).
template <typename T, typename S>
__global__ void k_batch_unpack(const T *y, const BatchNode *nodes, const InstDesc *inst, const BatchVec *vec, int np,
                               int accumulate) {
  const BatchNode nd = nodes[blockIdx.x];
  const int n = inst[nd.inst].n;
  S *x = reinterpret_cast<S *>(vec[nd.inst].x);
  for (int r = threadIdx.x; r < n; r += blockDim.x) {
    const S v = (S)y[(size_t)blockIdx.x * np + r];
    S *dst = x + (size_t)nd.row * n + r;
    *dst = accumulate ? *dst + v : v;
  }
}

// FP64 residual of one block row of one instance (one RHS): r -> y (type T),
// max|r| and max|x| into norms[3*inst + 0/1]. Same arithmetic as the single-
// instance residual kernel (fixed-order partial sums).
template <typename T>
__global__ void __launch_bounds__(kResThreads) k_batch_residual(T *y, const BatchNode *nodes, const InstDesc *inst,
                                                                const BatchVec *vec, int np, double *norms) {
  constexpr int NMAX = 128;  // largest compiled block size
  __shared__ double xs[3 * NMAX];
  __shared__ double ps[kResParts * NMAX];
  const BatchNode nd = nodes[blockIdx.x];
  const InstDesc in = inst[nd.inst];
  const int n = in.n, N = in.N, i = nd.row;
  const double *D = reinterpret_cast<const double *>(in.D);
  const double *B = reinterpret_cast<const double *>(in.B);
  const double *x = reinterpret_cast<const double *>(vec[nd.inst].x);
  const double *b = reinterpret_cast<const double *>(vec[nd.inst].b);
  for (int q = threadIdx.x; q < 3 * n; q += blockDim.x) {
    const int which = q / n, off = q % n, row = i - 1 + which;
    xs[which * NMAX + off] = (row >= 0 && row < N) ? x[(size_t)row * n + off] : 0.0;
  }
  __syncthreads();
  const size_t bs = (size_t)n * n;
  const double *Di = D + i * bs;
  const double *Bl = i > 0 ? B + (i - 1) * bs : nullptr;
  const double *Br = i + 1 < N ? B + i * bs : nullptr;
  const int chunk = (n + kResParts - 1) / kResParts;
  for (int idx = threadIdx.x; idx < kResParts * n; idx += blockDim.x) {
    const int part = idx / n, r = idx % n;
    const int c0 = part * chunk, c1 = min(n, c0 + chunk);
    double v = 0.0;
    for (int c = c0; c < c1; ++c) v = fma(r >= c ? Di[r * n + c] : Di[c * n + r], xs[NMAX + c], v);
    if (Bl)
      for (int c = c0; c < c1; ++c) v = fma(Bl[r * n + c], xs[c], v);
    if (Br)
      for (int c = c0; c < c1; ++c) v = fma(Br[c * n + r], xs[2 * NMAX + c], v);
    ps[part * NMAX + r] = v;
  }
  __syncthreads();
  double rmax = 0.0, xmax = 0.0;
  for (int r = threadIdx.x; r < np; r += blockDim.x) {
    if (r < n) {
      double ax = 0.0;
#pragma unroll
      for (int k = 0; k < kResParts; ++k) ax += ps[k * NMAX + r];
      const double v = b[(size_t)i * n + r] - ax;
      y[(size_t)blockIdx.x * np + r] = (T)v;
      rmax = nan_max(rmax, fabs(v));
      xmax = nan_max(xmax, fabs(xs[NMAX + r]));
    } else {
      y[(size_t)blockIdx.x * np + r] = T(0);
    }
  }
  for (int o = 16; o > 0; o >>= 1) {
    rmax = nan_max(rmax, __shfl_xor_sync(0xffffffffu, rmax, o));
    xmax = nan_max(xmax, __shfl_xor_sync(0xffffffffu, xmax, o));
  }
  if ((threadIdx.x & 31) == 0) {
    atomic_max_nonneg(norms + 3 * nd.inst + 0, rmax);
    atomic_max_nonneg(norms + 3 * nd.inst + 1, xmax);
  }
}

// Clears the residual and solution norm slots (norms[3k], norms[3k+1]) of every
// instance in one launch; the matrix-norm slot norms[3k+2] is kept.
__global__ void k_batch_clear_norms(double *norms, int count) {
  const int k = blockIdx.x * blockDim.x + threadIdx.x;
  if (k < count) {
    norms[3 * k] = 0.0;
    norms[3 * k + 1] = 0.0;
  }
}

// Lower bound of ||Psi||_inf per instance into norms[3*inst + 2] for the
// refinement's stopping test: each |a_ij| rounded toward zero to FP32, row
// sums with round-toward-zero additions, so the bound never exceeds the norm.
__global__ void k_batch_anorm_lb(const BatchNode *nodes, const InstDesc *inst, double *norms) {
  const BatchNode nd = nodes[blockIdx.x];
  const InstDesc in = inst[nd.inst];
  const int n = in.n, N = in.N, i = nd.row;
  const double *D = reinterpret_cast<const double *>(in.D);
  const double *B = reinterpret_cast<const double *>(in.B);
  const size_t bs = (size_t)n * n;
  const double *Di = D + i * bs;
  float best = 0.0f;
  for (int r = threadIdx.x; r < n; r += blockDim.x) {
    float s = 0.0f;
    for (int c = 0; c < n; ++c) s = __fadd_rz(s, abs_lower_f32(r >= c ? Di[r * n + c] : Di[c * n + r]));
    if (i > 0)
      for (int c = 0; c < n; ++c) s = __fadd_rz(s, abs_lower_f32(B[(i - 1) * bs + r * n + c]));
    if (i + 1 < N)
      for (int c = 0; c < n; ++c) s = __fadd_rz(s, abs_lower_f32(B[i * bs + c * n + r]));
    best = fmaxf(best, s);
  }
  for (int o = 16; o > 0; o >>= 1) best = fmaxf(best, __shfl_xor_sync(0xffffffffu, best, o));
  if ((threadIdx.x & 31) == 0) atomic_max_nonneg(norms + 3 * nd.inst + 2, (double)best);
}

template <typename T, typename S>
struct BatchVecKernels {
  static const void *pack() { return (const void *)&k_batch_pack<T, S>; }
  static const void *unpack() { return (const void *)&k_batch_unpack<T, S>; }
  static const void *resid() { return (const void *)&k_batch_residual<T>; }
};

struct BatchGroup {
  int np = 0;
  const KernelSet *ks = nullptr;
  std::vector<int> inst;  // global instance ids
  void *dpool = nullptr, *epool = nullptr, *y = nullptr;
  FactorItem *d_fac = nullptr;
  int32_t *d_fac_deps = nullptr;
  int n_fac = 0, n_first = 0;
  FactorItem *d_roots = nullptr;  // top-separator roots (mixed path, FP64 Cholesky): [level-1 roots | other roots]
  int n_roots_first = 0, n_roots_rest = 0;
  SolveFlowItem *d_solve = nullptr;
  int n_solve = 0;
  int *d_flow = nullptr;
  int fac_grid = 0, solve_grid = 0;
  BatchNode *d_nodes = nullptr;
  int n_nodes = 0;
  const void *pack = nullptr, *unpack = nullptr, *resid = nullptr;
  double flops = 0;
  cudaStream_t s = nullptr;  // the group's own stream: groups run concurrently
  cudaEvent_t ev = nullptr;  // its join point
};

}  // namespace btc

using namespace btc;

struct btc_batch_s {
  int count = 0, dtype = 0;
  cudaStream_t stream = nullptr;
  std::vector<int> N, n;
  std::vector<BatchGroup> groups;
  InstDesc *d_inst = nullptr;
  BatchVec *d_vec = nullptr;
  unsigned long long *d_info = nullptr;
  double *d_norms = nullptr;
  double *h_norms = nullptr;
  unsigned long long *h_info = nullptr;
  int *h_status = nullptr;
  bool factored = false, anorm_valid = false;
  std::vector<InstDesc> inst_host;
  double flops = 0;
  int64_t device_bytes = 0;
  cudaEvent_t fork_ev = nullptr;  // work queued on the batch stream before the groups start
};

namespace btc {

static int batch_alloc(void **p, size_t bytes, int64_t *acc) {
  cudaError_t e = cudaMalloc(p, std::max<size_t>(bytes, 16));
  if (e != cudaSuccess)
    return fail(e == cudaErrorMemoryAllocation ? BTC_ERR_OOM : BTC_ERR_CUDA, "batch allocation of %zu bytes: %s",
                bytes, cudaGetErrorString(e));
  *acc += (int64_t)bytes;
  return BTC_OK;
}

template <typename V>
static int upload(V **dst, const std::vector<V> &src, int64_t *acc) {
  int rc = batch_alloc((void **)dst, src.size() * sizeof(V), acc);
  if (rc) return rc;
  if (!src.empty()) BTC_CUDA(cudaMemcpy(*dst, src.data(), src.size() * sizeof(V), cudaMemcpyHostToDevice));
  return BTC_OK;
}

// Build the merged schedules of one group.
static int build_group(btc_batch_s *bt, BatchGroup &g) {
  const bool mixed = dtype_mixed(bt->dtype);
  const KernelSet &ks = *g.ks;
  const int64_t bs = (int64_t)g.np * g.np;
  int64_t d_base = 0, e_base = 0, y_base = 0;
  struct Ref {
    int level, k, local;
  };
  std::vector<HostPlan> hps(g.inst.size());
  std::vector<Ref> frefs, srefs;
  std::vector<BatchNode> nodes;
  for (size_t k = 0; k < g.inst.size(); ++k) {
    const int id = g.inst[k];
    HostPlan &hp = hps[k];
    build_host_plan(bt->N[id], bt->n[id], g.np, d_base, e_base, y_base, id, &hp);
    g.flops += hp.factor_flops;
    int local = 0;
    for (int l = 1; l <= hp.levels; ++l)
      for (size_t q = 0; q < hp.lv[l - 1].fac.size(); ++q) frefs.push_back({l, (int)k, local++});
    for (size_t q = 0; q < hp.solve_flow.size(); ++q) {
      // forward items carry their level through y_self's survival stride; recover the
      // phase-major order: forward by ascending level, backward by descending level
      srefs.push_back({0, (int)k, (int)q});
    }
    for (int r = 0; r < bt->N[id]; ++r) nodes.push_back({id, r});
    d_base += bt->N[id];
    e_base += std::max<int64_t>(hp.offdiag, 0);
    y_base += bt->N[id];
  }
  g.n_nodes = (int)nodes.size();
  // ---- factor: merged level-major order, roots split off on the mixed path
  std::stable_sort(frefs.begin(), frefs.end(), [](const Ref &a, const Ref &b) { return a.level < b.level; });
  std::vector<std::vector<FactorItem>> flat(g.inst.size());
  for (size_t k = 0; k < g.inst.size(); ++k)
    for (int l = 1; l <= hps[k].levels; ++l)
      for (const FactorItem &it : hps[k].lv[l - 1].fac) flat[k].push_back(it);
  std::vector<std::vector<int32_t>> merged_of(g.inst.size());
  for (size_t k = 0; k < g.inst.size(); ++k) merged_of[k].assign(flat[k].size(), -1);
  std::vector<FactorItem> fac, roots_first, roots_rest;
  std::vector<int32_t> deps;
  for (const Ref &r : frefs) {
    const FactorItem &it = flat[r.k][r.local];
    if (mixed && (it.flags & FI_ROOT)) {
      (r.level == 1 ? roots_first : roots_rest).push_back(it);
      continue;
    }
    merged_of[r.k][r.local] = (int32_t)fac.size();
    fac.push_back(it);
    if (r.level == 1) g.n_first = (int)fac.size();
  }
  deps.assign(3 * fac.size(), -1);
  for (const Ref &r : frefs) {
    const int32_t m = merged_of[r.k][r.local];
    if (m < 0) continue;
    for (int j = 0; j < 3; ++j) {
      const int32_t d = hps[r.k].fac_deps[3 * (size_t)r.local + j];
      deps[3 * (size_t)m + j] = d >= 0 ? merged_of[r.k][d] : -1;
    }
  }
  g.n_fac = (int)fac.size();
  g.n_roots_first = (int)roots_first.size();
  g.n_roots_rest = (int)roots_rest.size();
  std::vector<FactorItem> roots = roots_first;
  roots.insert(roots.end(), roots_rest.begin(), roots_rest.end());
  // ---- solve: forward items by ascending level, then backward items by descending level
  struct SRef {
    int phase, key, k, local;
  };
  std::vector<SRef> sr;
  for (size_t k = 0; k < g.inst.size(); ++k) {
    const HostPlan &hp = hps[k];
    // the per-instance solve list is [fwd level 1 .. L][bwd level L .. 1]; recover levels
    int q = 0;
    for (int l = 1; l <= hp.levels; ++l)
      for (size_t t = 0; t < hp.lv[l - 1].fwd.size(); ++t) sr.push_back({0, l, (int)k, q++});
    for (int l = hp.levels; l >= 1; --l)
      for (size_t t = 0; t < hp.lv[l - 1].bwd.size(); ++t) sr.push_back({1, -l, (int)k, q++});
  }
  std::stable_sort(sr.begin(), sr.end(),
                   [](const SRef &a, const SRef &b) { return a.phase != b.phase ? a.phase < b.phase : a.key < b.key; });
  std::vector<std::vector<int32_t>> smerged(g.inst.size());
  for (size_t k = 0; k < g.inst.size(); ++k) smerged[k].assign(hps[k].solve_flow.size(), -1);
  for (size_t t = 0; t < sr.size(); ++t) smerged[sr[t].k][sr[t].local] = (int32_t)t;
  std::vector<SolveFlowItem> solve(sr.size());
  for (size_t t = 0; t < sr.size(); ++t) {
    SolveFlowItem q = hps[sr[t].k].solve_flow[sr[t].local];
    for (int j = 0; j < 3; ++j) q.dep[j] = q.dep[j] >= 0 ? smerged[sr[t].k][q.dep[j]] : -1;
    solve[t] = q;
  }
  g.n_solve = (int)solve.size();
  (void)srefs;
  // ---- device memory
  int rc;
  int64_t *acc = &bt->device_bytes;
  if ((rc = batch_alloc(&g.dpool, (size_t)d_base * bs * ks.elem, acc)) ||
      (rc = batch_alloc(&g.epool, (size_t)std::max<int64_t>(e_base, 1) * bs * ks.elem, acc)) ||
      (rc = batch_alloc(&g.y, (size_t)y_base * g.np * ks.elem, acc)) || (rc = upload(&g.d_fac, fac, acc)) ||
      (rc = upload(&g.d_fac_deps, deps, acc)) || (rc = upload(&g.d_roots, roots, acc)) ||
      (rc = upload(&g.d_solve, solve, acc)) || (rc = upload(&g.d_nodes, nodes, acc)))
    return rc;
  const size_t nflags = kFlowHeader + (size_t)std::max(g.n_fac, g.n_solve);
  if ((rc = batch_alloc((void **)&g.d_flow, nflags * sizeof(int), acc))) return rc;
  BTC_CUDA(cudaMemset(g.d_flow, 0, nflags * sizeof(int)));
  if ((rc = set_smem(ks.fac_flow, ks.fac_smem)) || (rc = set_smem(ks.solve_flow, ks.fwd_smem(1))) ||
      (rc = set_smem(ks.root64_first, ks.root_smem)) || (rc = set_smem(ks.root64_rest, ks.root_smem)))
    return rc;
  int dev = 0, sms = 0, bf = 0, bsl = 0;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  BTC_CUDA(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&bf, ks.fac_flow, ks.fac_threads, ks.fac_smem));
  BTC_CUDA(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&bsl, ks.solve_flow, kSolveThreads, ks.fwd_smem(1)));
  g.fac_grid = std::max(1, bf * sms);
  g.solve_grid = std::max(1, bsl * sms);
  if (bt->dtype == BTC_F32) {
    g.pack = BatchVecKernels<float, float>::pack();
    g.unpack = BatchVecKernels<float, float>::unpack();
    g.resid = nullptr;
  } else if (bt->dtype == BTC_F64) {
    g.pack = BatchVecKernels<double, double>::pack();
    g.unpack = BatchVecKernels<double, double>::unpack();
    g.resid = BatchVecKernels<double, double>::resid();
  } else {
    g.pack = BatchVecKernels<float, double>::pack();
    g.unpack = BatchVecKernels<float, double>::unpack();
    g.resid = BatchVecKernels<float, double>::resid();
  }
  return BTC_OK;
}

static FlowSync group_sync(BatchGroup &g, int which) {
  FlowSync fs;
  fs.ticket = g.d_flow + which;
  fs.status = g.d_flow + 2;
  fs.done = g.d_flow + kFlowHeader;
  fs.trace = nullptr;
  return fs;
}

// The block-size groups are independent (own pools, work vector, flags and
// persistent launches; each launch waits only on its own items), so they run
// concurrently, each on its own stream: fork after the work queued on the
// batch stream, join before the batch stream continues.
static int batch_fork(btc_batch_s *bt) {
  BTC_CUDA(cudaEventRecord(bt->fork_ev, bt->stream));
  for (BatchGroup &g : bt->groups) BTC_CUDA(cudaStreamWaitEvent(g.s, bt->fork_ev, 0));
  return BTC_OK;
}
static int batch_join(btc_batch_s *bt) {
  for (BatchGroup &g : bt->groups) {
    BTC_CUDA(cudaEventRecord(g.ev, g.s));
    BTC_CUDA(cudaStreamWaitEvent(bt->stream, g.ev, 0));
  }
  return BTC_OK;
}

static int group_solve(btc_batch_s *bt, BatchGroup &g) {
  const KernelSet &k = *g.ks;
  (void)bt;
  BTC_CUDA(cudaMemsetAsync(g.d_flow + 1, 0, sizeof(int), g.s));
  BTC_CUDA(cudaMemsetAsync(g.d_flow + kFlowHeader, 0, sizeof(int) * (size_t)g.n_solve, g.s));
  SolveArgs a;
  a.items = g.d_solve;
  a.count = g.n_solve;
  a.dpool = g.dpool;
  a.epool = g.epool;
  a.y = g.y;
  a.m = 1;
  return launch_n(k.solve_flow, std::min(g.solve_grid, g.n_solve), kSolveThreads, k.fwd_smem(1), g.s, a,
                  group_sync(g, 1));
}

static int batch_read_status(btc_batch_s *bt) {
  for (BatchGroup &g : bt->groups) {
    BTC_CUDA(cudaMemcpyAsync(bt->h_status, g.d_flow + 2, sizeof(int), cudaMemcpyDeviceToHost, bt->stream));
    BTC_CUDA(cudaStreamSynchronize(bt->stream));
    if (*bt->h_status) return fail(BTC_ERR_TIMEOUT, "a bounded device-side wait gave up");
  }
  return BTC_OK;
}

}  // namespace btc

extern "C" {

int btc_batch_plan(btc_batch_t *out, int count, const int *N, const int *n, int dtype, void *stream) {
  if (!out || count < 1 || !N || !n) return fail(BTC_ERR_ARG, "btc_batch_plan: invalid arguments");
  *out = nullptr;
  if (!dtype_ok(dtype)) return fail(BTC_ERR_ARG, "btc_batch_plan: unknown dtype %d", dtype);
  btc_batch_s *bt = new btc_batch_s();
  bt->count = count;
  bt->dtype = dtype;
  bt->stream = (cudaStream_t)stream;
  bt->N.assign(N, N + count);
  bt->n.assign(n, n + count);
  auto cleanup = [&](int code) {
    btc_batch_free(bt);
    return code;
  };
  std::map<int, std::vector<int>> by_np;
  for (int k = 0; k < count; ++k) {
    if (N[k] < 1 || n[k] < 1) return cleanup(fail(BTC_ERR_ARG, "instance %d: invalid sizes", k));
    const int np = padded_size(n[k], dtype);
    if (!np) return cleanup(fail(BTC_ERR_UNSUPPORTED, "instance %d: block size %d not compiled", k, n[k]));
    if (np > 128)
      return cleanup(fail(BTC_ERR_UNSUPPORTED, "instance %d: batches take block sizes up to 128 (n = %d)", k, n[k]));
    by_np[np].push_back(k);
  }
  int rc;
  for (auto &kv : by_np) {
    BatchGroup g;
    g.np = kv.first;
    g.ks = &kernels_for(dtype, g.np);
    if (!g.ks->valid) return cleanup(fail(BTC_ERR_UNSUPPORTED, "no kernels for np %d", g.np));
    g.inst = kv.second;
    bt->groups.push_back(g);
    if ((rc = build_group(bt, bt->groups.back()))) return cleanup(rc);
    bt->flops += bt->groups.back().flops;
  }
  int64_t *acc = &bt->device_bytes;
  bt->inst_host.assign(count, InstDesc{nullptr, nullptr, 0, 0});
  for (int k = 0; k < count; ++k) bt->inst_host[k] = InstDesc{nullptr, nullptr, N[k], n[k]};
  if ((rc = batch_alloc((void **)&bt->d_inst, count * sizeof(InstDesc), acc)) ||
      (rc = batch_alloc((void **)&bt->d_vec, count * sizeof(BatchVec), acc)) ||
      (rc = batch_alloc((void **)&bt->d_info, count * sizeof(unsigned long long), acc)) ||
      (rc = batch_alloc((void **)&bt->d_norms, 3 * count * sizeof(double), acc)))
    return cleanup(rc);
  if (cudaEventCreateWithFlags(&bt->fork_ev, cudaEventDisableTiming) != cudaSuccess)
    return cleanup(fail(BTC_ERR_CUDA, "btc_batch_plan: event creation failed"));
  for (BatchGroup &g : bt->groups)
    if (cudaStreamCreateWithFlags(&g.s, cudaStreamNonBlocking) != cudaSuccess ||
        cudaEventCreateWithFlags(&g.ev, cudaEventDisableTiming) != cudaSuccess)
      return cleanup(fail(BTC_ERR_CUDA, "btc_batch_plan: stream creation failed"));
  cudaError_t e;
  if ((e = cudaMallocHost(&bt->h_norms, 3 * count * sizeof(double))) != cudaSuccess ||
      (e = cudaMallocHost(&bt->h_info, count * sizeof(unsigned long long))) != cudaSuccess ||
      (e = cudaMallocHost(&bt->h_status, sizeof(int))) != cudaSuccess)
    return cleanup(fail(BTC_ERR_OOM, "btc_batch_plan: host staging: %s", cudaGetErrorString(e)));
  *out = bt;
  return BTC_OK;
}

int btc_batch_query(btc_batch_t bt, int *groups, double *factor_flops, int64_t *device_bytes) {
  if (!bt) return fail(BTC_ERR_ARG, "btc_batch_query: NULL batch");
  if (groups) *groups = (int)bt->groups.size();
  if (factor_flops) *factor_flops = bt->flops;
  if (device_bytes) *device_bytes = bt->device_bytes;
  return BTC_OK;
}

int btc_batch_factor(btc_batch_t bt, const void *const *D, const void *const *B) {
  if (!bt || !D || !B) return fail(BTC_ERR_ARG, "btc_batch_factor: NULL argument");
  for (int k = 0; k < bt->count; ++k) {
    if (!D[k] || (bt->N[k] > 1 && !B[k])) return fail(BTC_ERR_ARG, "btc_batch_factor: instance %d pointer", k);
    if (((uintptr_t)D[k] | (uintptr_t)B[k]) & 15) return fail(BTC_ERR_ARG, "instance %d: 16-byte alignment", k);
    bt->inst_host[k].D = D[k];
    bt->inst_host[k].B = B[k];
  }
  // pageable source: the copy is staged by the runtime before the call returns
  BTC_CUDA(cudaMemcpyAsync(bt->d_inst, bt->inst_host.data(), bt->count * sizeof(InstDesc), cudaMemcpyHostToDevice,
                           bt->stream));
  BTC_CUDA(cudaMemsetAsync(bt->d_info, 0xFF, bt->count * sizeof(unsigned long long), bt->stream));
  int rc = batch_fork(bt);
  for (BatchGroup &g : bt->groups) {
    if (rc) break;
    const KernelSet &k = *g.ks;
    FactorArgs a;
    a.dpool = g.dpool;
    a.epool = g.epool;
    a.inst = bt->d_inst;
    a.info = bt->d_info;
    a.status = g.d_flow + 2;
    InstDesc none{nullptr, nullptr, 0, 0};
    if (cudaMemsetAsync(g.d_flow, 0, 3 * sizeof(int), g.s) != cudaSuccess) {
      rc = fail(BTC_ERR_CUDA, "btc_batch_factor: memset");
      break;
    }
    if (g.n_fac > 0) {
      if (cudaMemsetAsync(g.d_flow + kFlowHeader, 0, sizeof(int) * (size_t)g.n_fac, g.s) != cudaSuccess) {
        rc = fail(BTC_ERR_CUDA, "btc_batch_factor: memset");
        break;
      }
      a.items = g.d_fac;
      a.count = g.n_fac;
      const int32_t *deps = g.d_fac_deps;
      if ((rc = launch_n(k.fac_flow, std::min(g.fac_grid, g.n_fac), k.fac_threads, k.fac_smem, g.s, a, none, deps,
                         g.n_first, group_sync(g, 0))))
        break;
    }
    if (g.n_roots_first > 0) {
      a.items = g.d_roots;
      a.count = g.n_roots_first;
      if ((rc = launch_n(k.root64_first, g.n_roots_first, k.root_threads, k.root_smem, g.s, a, none))) break;
    }
    if (g.n_roots_rest > 0) {
      a.items = g.d_roots + g.n_roots_first;
      a.count = g.n_roots_rest;
      if ((rc = launch_n(k.root64_rest, g.n_roots_rest, k.root_threads, k.root_smem, g.s, a, none))) break;
    }
  }
  const int rj = batch_join(bt);
  if (rc || (rc = rj)) return rc;
  bt->factored = true;
  bt->anorm_valid = false;
  return BTC_OK;
}

int btc_batch_info(btc_batch_t bt, int *failed_instance, int *block, int *col) {
  if (!bt) return fail(BTC_ERR_ARG, "btc_batch_info: NULL batch");
  int rc = batch_read_status(bt);
  if (rc) return rc;
  BTC_CUDA(cudaMemcpyAsync(bt->h_info, bt->d_info, bt->count * sizeof(unsigned long long), cudaMemcpyDeviceToHost,
                           bt->stream));
  BTC_CUDA(cudaStreamSynchronize(bt->stream));
  for (int k = 0; k < bt->count; ++k)
    if (bt->h_info[k] != ~0ull) {
      if (failed_instance) *failed_instance = k;
      if (block) *block = (int)(bt->h_info[k] >> 20);
      if (col) *col = (int)(bt->h_info[k] & 0xFFFFF);
      return fail(BTC_ERR_NOT_SPD, "instance %d: pivot not positive", k);
    }
  if (failed_instance) *failed_instance = -1;
  if (block) *block = -1;
  if (col) *col = -1;
  return BTC_OK;
}

static int batch_set_vec(btc_batch_t bt, const void *const *b, void *const *x) {
  std::vector<BatchVec> v(bt->count);
  for (int k = 0; k < bt->count; ++k) {
    if (!b[k] || !x[k]) return fail(BTC_ERR_ARG, "instance %d: NULL vector", k);
    v[k].b = b[k];
    v[k].x = x[k];
  }
  BTC_CUDA(cudaMemcpyAsync(bt->d_vec, v.data(), bt->count * sizeof(BatchVec), cudaMemcpyHostToDevice, bt->stream));
  return BTC_OK;
}

int btc_batch_solve(btc_batch_t bt, const void *const *b, void *const *x) {
  if (!bt || !b || !x) return fail(BTC_ERR_ARG, "btc_batch_solve: NULL argument");
  if (!bt->factored) return fail(BTC_ERR_NOT_FACTORED, "btc_batch_solve: no factorization");
  int rc = batch_set_vec(bt, b, x);
  if (rc || (rc = batch_fork(bt))) return rc;
  for (BatchGroup &g : bt->groups) {
    int assign = 0;
    if ((rc = launch_n(g.pack, g.n_nodes, 64, 0, g.s, g.y, (const BatchNode *)g.d_nodes, (const InstDesc *)bt->d_inst,
                       (const BatchVec *)bt->d_vec, g.np)) ||
        (rc = group_solve(bt, g)) ||
        (rc = launch_n(g.unpack, g.n_nodes, 64, 0, g.s, (const void *)g.y, (const BatchNode *)g.d_nodes,
                       (const InstDesc *)bt->d_inst, (const BatchVec *)bt->d_vec, g.np, assign)))
      break;
  }
  const int rj = batch_join(bt);
  return rc ? rc : rj;
}

int btc_batch_solve_refined(btc_batch_t bt, const double *const *b, double *const *x, double tol, int maxit,
                            int *iters, double *max_relres) {
  if (!bt || !b || !x || maxit < 0) return fail(BTC_ERR_ARG, "btc_batch_solve_refined: invalid arguments");
  if (bt->dtype == BTC_F32) return fail(BTC_ERR_ARG, "btc_batch_solve_refined needs an FP64 or mixed batch");
  if (!bt->factored) return fail(BTC_ERR_NOT_FACTORED, "btc_batch_solve_refined: no factorization");
  int rc = btc_batch_info(bt, nullptr, nullptr, nullptr);
  if (rc) return rc;
  if ((rc = btc_batch_solve(bt, (const void *const *)b, (void *const *)x))) return rc;
  if (!bt->anorm_valid) {
    BTC_CUDA(cudaMemsetAsync(bt->d_norms, 0, 3 * (size_t)bt->count * sizeof(double), bt->stream));
    if ((rc = batch_fork(bt))) return rc;
    for (BatchGroup &g : bt->groups)
      if ((rc = launch_n((const void *)&k_batch_anorm_lb, g.n_nodes, 64, 0, g.s, (const BatchNode *)g.d_nodes,
                         (const InstDesc *)bt->d_inst, bt->d_norms)))
        break;
    const int rj = batch_join(bt);
    if (rc || (rc = rj)) return rc;
    bt->anorm_valid = true;
  }
  int it = 0;
  double worst = 0.0;
  for (;;) {
    if ((rc = launch_n((const void *)&k_batch_clear_norms, (bt->count + 255) / 256, 256, 0, bt->stream, bt->d_norms,
                       bt->count)))
      return rc;
    if ((rc = batch_fork(bt))) return rc;
    for (BatchGroup &g : bt->groups)
      if ((rc = launch_n(g.resid, g.n_nodes, kResThreads, 0, g.s, g.y, (const BatchNode *)g.d_nodes,
                         (const InstDesc *)bt->d_inst, (const BatchVec *)bt->d_vec, g.np, bt->d_norms)))
        break;
    const int rj = batch_join(bt);
    if (rc || (rc = rj)) return rc;
    BTC_CUDA(cudaMemcpyAsync(bt->h_norms, bt->d_norms, 3 * bt->count * sizeof(double), cudaMemcpyDeviceToHost,
                             bt->stream));
    BTC_CUDA(cudaStreamSynchronize(bt->stream));
    worst = 0.0;
    bool nan = false;
    for (int k = 0; k < bt->count; ++k) {
      const double rn = bt->h_norms[3 * k], xn = bt->h_norms[3 * k + 1], an = bt->h_norms[3 * k + 2];
      const double rel = (an * xn > 0) ? rn / (an * xn) : rn;
      if (!(rel == rel)) nan = true;
      worst = std::max(worst, rel);
    }
    if (nan) worst = NAN;  // reported as such: a NaN residual never counts as converged
    if (nan || worst <= tol || it >= maxit) break;
    if ((rc = batch_fork(bt))) return rc;
    for (BatchGroup &g : bt->groups) {
      int accumulate = 1;
      if ((rc = group_solve(bt, g)) ||
          (rc = launch_n(g.unpack, g.n_nodes, 64, 0, g.s, (const void *)g.y, (const BatchNode *)g.d_nodes,
                         (const InstDesc *)bt->d_inst, (const BatchVec *)bt->d_vec, g.np, accumulate)))
        break;
    }
    const int rj2 = batch_join(bt);
    if (rc || (rc = rj2)) return rc;
    ++it;
  }
  if (iters) *iters = it;
  if (max_relres) *max_relres = worst;
  if ((rc = batch_read_status(bt))) return rc;
  if (!(worst <= tol)) return fail(BTC_ERR_NOT_CONVERGED, "batch refinement stopped at %.3e", worst);
  return BTC_OK;
}

int btc_batch_free(btc_batch_t bt) {
  if (!bt) return BTC_OK;
  cudaStreamSynchronize(bt->stream);
  for (BatchGroup &g : bt->groups) {
    if (g.s) {
      cudaStreamSynchronize(g.s);
      cudaStreamDestroy(g.s);
    }
    if (g.ev) cudaEventDestroy(g.ev);
    void *ptrs[] = {g.dpool, g.epool, g.y, g.d_fac, g.d_fac_deps, g.d_roots, g.d_solve, g.d_flow, g.d_nodes};
    for (void *q : ptrs)
      if (q) cudaFree(q);
  }
  void *ptrs[] = {bt->d_inst, bt->d_vec, bt->d_info, bt->d_norms};
  for (void *q : ptrs)
    if (q) cudaFree(q);
  if (bt->h_norms) cudaFreeHost(bt->h_norms);
  if (bt->h_info) cudaFreeHost(bt->h_info);
  if (bt->h_status) cudaFreeHost(bt->h_status);
  if (bt->fork_ev) cudaEventDestroy(bt->fork_ev);
  delete bt;
  return BTC_OK;
}

}  // extern "C"
