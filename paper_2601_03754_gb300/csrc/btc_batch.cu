// Batched plans: many independent block-tridiagonal systems of different
// (N, n) factored and solved together. Instances are grouped by padded block
// size; each group runs ONE persistent dataflow launch for the factor and one
// for the solve, whose work items are the (instance, node) eliminations of all
// instances in level order. Each item waits only for the producer nodes of its
// own instance (bounded waits), so short instances finish early and long ones
// keep the SMs busy. Each group's factor launch is autotuned (register budget
// x resident CTAs per SM, i.e. how many nodes one SM holds at once), the
// groups are launched largest first on their own streams, and the whole
// factor + refined solve can run as one captured graph with a device-side
// refinement loop (btc_batch_factor_solve_refined).
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
  grid_dep_enter();
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
  grid_dep_enter();
  const BatchNode nd = nodes[blockIdx.x];
  const int n = inst[nd.inst].n;
  S *x = reinterpret_cast<S *>(vec[nd.inst].x);
  for (int r = threadIdx.x; r < n; r += blockDim.x) {
    const S v = (S)y[(size_t)blockIdx.x * np + r];
    S *dst = x + (size_t)nd.row * n + r;
    *dst = accumulate ? *dst + v : v;
  }
}

// FP64 residual of block rows of the group (one RHS): r -> y (type T),
// max|r| and max|x| into norms[3*inst + 0/1], and with with_anorm also the
// lower bound of ||Psi_inst||_inf (each |a_ij| rounded toward zero to FP32,
// row sums with round-toward-zero additions) into norms[3*inst + 2]. One CTA
// covers NPC = max(1, kResThreads / (kResParts * np)) consecutive block rows
// of the group, so small blocks keep the CTA's threads busy. Each output's
// 3n-term dot product is split into kResParts column ranges, each with three
// independent FP64 chains (the D_i, B_{i-1} and B_i^T terms) added in a fixed
// order (deterministic).
template <typename T>
__global__ void __launch_bounds__(kResThreads) k_batch_residual(T *y, const BatchNode *nodes, int n_nodes,
                                                                const InstDesc *inst, const BatchVec *vec, int np,
                                                                double *norms, int with_anorm) {
  grid_dep_enter();
  constexpr int NMAX = 128;  // largest block size of a batch
  __shared__ double xs[3 * NMAX * 2];
  __shared__ double ps[kResParts * NMAX * 2];
  __shared__ float as[kResParts * NMAX * 2];
  __shared__ unsigned long long red[3 * 8];                 // per block row: max|r|, max|x|, norm bound
  const int npc = max(1, kResThreads / (kResParts * np));  // block rows per CTA (<= 8: np >= 8)
  const int slot_sz = np;                                   // per-row stride in the staging arrays
  const int r0 = blockIdx.x * npc;
  if (threadIdx.x < 3 * 8) red[threadIdx.x] = 0ull;  // +0.0
  // stage x_{i-1}, x_i, x_{i+1} of each block row of this CTA
  for (int q = threadIdx.x; q < npc * 3 * np; q += blockDim.x) {
    const int w = q / (3 * np), rem = q % (3 * np), which = rem / np, off = rem % np;
    if (r0 + w >= n_nodes) continue;
    const BatchNode nd = nodes[r0 + w];
    const InstDesc in = inst[nd.inst];
    const int row = nd.row - 1 + which;
    const double *x = reinterpret_cast<const double *>(vec[nd.inst].x);
    xs[(w * 3 + which) * slot_sz + off] = (off < in.n && row >= 0 && row < in.N) ? x[(size_t)row * in.n + off] : 0.0;
  }
  __syncthreads();
  for (int idx = threadIdx.x; idx < npc * kResParts * np; idx += blockDim.x) {
    const int w = idx / (kResParts * np), rem = idx % (kResParts * np), part = rem / np, r = rem % np;
    if (r0 + w >= n_nodes) continue;
    const BatchNode nd = nodes[r0 + w];
    const InstDesc in = inst[nd.inst];
    const int n = in.n, N = in.N, i = nd.row;
    if (r >= n) continue;
    const size_t bs = (size_t)n * n;
    const double *Di = reinterpret_cast<const double *>(in.D) + i * bs;
    const double *B = reinterpret_cast<const double *>(in.B);
    const bool has_l = i > 0, has_u = i + 1 < N;
    const double *Bl = has_l ? B + (i - 1) * bs : Di;  // a valid address when the block is absent
    const double *Br = has_u ? B + i * bs : Di;
    const int chunk = (n + kResParts - 1) / kResParts;
    const int c0 = part * chunk, c1 = min(n, c0 + chunk);
    const double *x0 = xs + (w * 3 + 0) * slot_sz, *x1 = x0 + slot_sz, *x2 = x1 + slot_sz;
    double vd = 0.0, vl = 0.0, vu = 0.0;
    float sabs = 0.0f;
    for (int c = c0; c < c1; ++c) {
      const double ad = __ldg(r >= c ? Di + r * n + c : Di + c * n + r);
      const double al = has_l ? __ldg(Bl + r * n + c) : 0.0;
      const double au = has_u ? __ldg(Br + c * n + r) : 0.0;
      vd = fma(ad, x1[c], vd);
      vl = fma(al, x0[c], vl);
      vu = fma(au, x2[c], vu);
      if (with_anorm)
        sabs = __fadd_rz(__fadd_rz(__fadd_rz(sabs, abs_lower_f32(ad)), abs_lower_f32(al)), abs_lower_f32(au));
    }
    ps[(w * kResParts + part) * slot_sz + r] = (vd + vl) + vu;
    if (with_anorm) as[(w * kResParts + part) * slot_sz + r] = sabs;
  }
  __syncthreads();
  for (int q = threadIdx.x; q < npc * np; q += blockDim.x) {
    const int w = q / np, r = q % np;
    if (r0 + w >= n_nodes) continue;
    const BatchNode nd = nodes[r0 + w];
    const InstDesc in = inst[nd.inst];
    const int n = in.n;
    T *yr = y + (size_t)(r0 + w) * np + r;
    if (r >= n) {
      *yr = T(0);
      continue;
    }
    double ax = 0.0;
    float rs = 0.0f;
#pragma unroll
    for (int k = 0; k < kResParts; ++k) {
      ax += ps[(w * kResParts + k) * slot_sz + r];
      if (with_anorm) rs = __fadd_rz(rs, as[(w * kResParts + k) * slot_sz + r]);
    }
    const double *b = reinterpret_cast<const double *>(vec[nd.inst].b);
    const double v = b[(size_t)nd.row * n + r] - ax;
    *yr = (T)v;
    // maxima of the block row in shared memory first (non-negative doubles order like their bits; fabs of a
    // NaN orders above +inf), then one global update per block row
    atomicMax(&red[3 * w + 0], (unsigned long long)__double_as_longlong(fabs(v)));
    atomicMax(&red[3 * w + 1], (unsigned long long)__double_as_longlong(fabs(xs[(w * 3 + 1) * slot_sz + r])));
    if (with_anorm) atomicMax(&red[3 * w + 2], (unsigned long long)__double_as_longlong((double)rs));
  }
  __syncthreads();
  if (threadIdx.x < 3 * npc) {
    const int w = threadIdx.x / 3, k = threadIdx.x % 3;
    if (r0 + w < n_nodes && (k < 2 || with_anorm))
      atomic_max_nonneg(norms + 3 * nodes[r0 + w].inst + k, __longlong_as_double((long long)red[threadIdx.x]));
  }
}

// Clears the residual and solution norm slots (norms[3k], norms[3k+1]) of every
// instance in one launch; the matrix-norm slot norms[3k+2] too when the next
// residual forms the matrix-norm bound.
__global__ void k_batch_clear_norms(double *norms, int count, int with_anorm) {
  grid_dep_enter();
  const int k = blockIdx.x * blockDim.x + threadIdx.x;
  if (k < count) {
    norms[3 * k] = 0.0;
    norms[3 * k + 1] = 0.0;
    if (with_anorm) norms[3 * k + 2] = 0.0;
  }
}

// Stopping test of the graph-resident batch refinement (one CTA): the worst
// relative residual over the instances (NaN if any is NaN); continue while it
// is above tol and fewer than maxit steps were taken.
__global__ void k_batch_decide(const double *norms, int count, double tol, int maxit, int first, void *rb_,
                               cudaGraphConditionalHandle h) {
  grid_dep_enter();
  __shared__ double red[32];
  double worst = 0.0;
  for (int k = threadIdx.x; k < count; k += blockDim.x) {
    const double rn = norms[3 * k], xn = norms[3 * k + 1], an = norms[3 * k + 2];
    worst = nan_max(worst, (an * xn > 0) ? rn / (an * xn) : rn);
  }
  for (int o = 16; o > 0; o >>= 1) worst = nan_max(worst, __shfl_xor_sync(0xffffffffu, worst, o));
  if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = worst;
  __syncthreads();
  if (threadIdx.x == 0) {
    for (int w = 1; w < (int)(blockDim.x >> 5); ++w) worst = nan_max(worst, red[w]);
    int *iters = reinterpret_cast<int *>(reinterpret_cast<char *>(rb_) + sizeof(double));
    double *wst = reinterpret_cast<double *>(rb_);
    if (first) *iters = 0;
    const bool more = !(worst <= tol) && worst == worst && *iters < maxit;
    if (more) *iters += 1;
    *wst = worst;
    cudaGraphSetConditional(h, more ? 1u : 0u);
  }
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
  // a group with a partition-order instance converts every instance's inputs in a batched packing
  // pass first (then no item reads the caller's arrays)
  bool packed = false;
  PackNode *d_pack = nullptr;
  const void *pack = nullptr, *unpack = nullptr, *resid = nullptr;
  double flops = 0;
  cudaStream_t s = nullptr;  // the group's own stream: groups run concurrently
  cudaEvent_t ev = nullptr;  // its join point
  // persistent factor launch configuration: residency variant and CTAs per SM (autotuned)
  int occ[kFlowVariants] = {};
  int var = 0, ctas = 0, sms = 1;
  bool tuned = false;
  double tuned_ms = 0.0;
};

// One readback block of the batch's graph-resident refinement: worst relative residual over the
// instances, refinement steps taken, and the launch status words of the groups.
struct BatchReadback {
  double worst;
  int iters;
  int status;
};

}  // namespace btc

using namespace btc;

struct btc_batch_s {
  int count = 0, dtype = 0;
  bool autotune = true, graphs = true;
  // captured factor + refined solve (btc_batch_factor_solve_refined)
  cudaStream_t gstream = nullptr, gstream2 = nullptr;
  cudaEvent_t gevent = nullptr;
  cudaGraphExec_t gexec = nullptr;
  double gtol = -1.0;
  int gmaxit = -1;
  BatchReadback *d_rb = nullptr, *h_rb = nullptr;
  cudaStream_t stream = nullptr;
  std::vector<int> N, n;
  std::vector<int> chunks;  // per instance: 0 = nested dissection, c >= 1 = partition order with c chunks
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
  std::vector<PackNode> pack;
  g.packed = false;
  for (size_t k = 0; k < g.inst.size(); ++k) g.packed = g.packed || bt->chunks[g.inst[k]] > 0;
  for (size_t k = 0; k < g.inst.size(); ++k) {
    const int id = g.inst[k];
    HostPlan &hp = hps[k];
    if (bt->chunks[id] > 0) {
      if (!build_partition_plan(bt->N[id], bt->n[id], g.np, bt->chunks[id], d_base, e_base, y_base, id, &hp))
        return fail(BTC_ERR_ARG, "instance %d: %d chunks do not fit in N = %d", id, bt->chunks[id], bt->N[id]);
    } else {
      build_host_plan(bt->N[id], bt->n[id], g.np, d_base, e_base, y_base, id, &hp);
    }
    if (g.packed)  // each node's coupling with the next one starts in the orientation of the node eliminated first
      for (int r = 0; r < bt->N[id]; ++r) {
        const int tr = r + 1 >= bt->N[id] ? 0 : hp.packed ? (int)hp.slot_transposed[r] : ((r + 1) & 1);
        pack.push_back({e_base + r, id, r, tr, 0});
      }
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
      (r.level == 1 && !g.packed ? roots_first : roots_rest).push_back(it);
      continue;
    }
    merged_of[r.k][r.local] = (int32_t)fac.size();
    fac.push_back(it);
    if (r.level == 1 && !g.packed) g.n_first = (int)fac.size();
  }
  deps.assign(3 * fac.size(), -1);
  for (const Ref &r : frefs) {
    const int32_t m = merged_of[r.k][r.local];
    if (m < 0) continue;
    for (int j = 0; j < 3; ++j) {
      const int32_t d = hps[r.k].fac_deps[3 * (size_t)r.local + j];
      deps[3 * (size_t)m + j] = d == -1 ? -1 : d >= 0 ? merged_of[r.k][d] : core_dep(merged_of[r.k][dep_item(d)]);
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
    if (hp.packed) {  // partition order: the planner's keys (level of the item's node, negated backward)
      for (size_t q = 0; q < hp.solve_flow.size(); ++q)
        sr.push_back({hp.solve_flow[q].kind, hp.solve_key[q], (int)k, (int)q});
      continue;
    }
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
      (rc = upload(&g.d_solve, solve, acc)) || (rc = upload(&g.d_nodes, nodes, acc)) ||
      (g.packed && (rc = upload(&g.d_pack, pack, acc))))
    return rc;
  const size_t nflags = kFlowHeader + (size_t)std::max(g.n_fac, g.n_solve);
  if ((rc = batch_alloc((void **)&g.d_flow, nflags * sizeof(int), acc))) return rc;
  BTC_CUDA(cudaMemset(g.d_flow, 0, nflags * sizeof(int)));
  if ((rc = set_smem(ks.fac_flow, ks.fac_smem)) || (rc = set_smem(ks.solve_flow, ks.fwd_smem(1))) ||
      (rc = set_smem(ks.root64_first, ks.root_smem)) || (rc = set_smem(ks.root64_rest, ks.root_smem)))
    return rc;
  int dev = 0, sms = 0, bsl = 0;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  g.sms = std::max(1, sms);
  for (int v = 0; v < ks.n_flow_v; ++v) {
    if ((rc = set_smem(ks.flow_v[v].fac, ks.fac_smem))) return rc;
    BTC_CUDA(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&g.occ[v], ks.flow_v[v].fac, ks.fac_threads, ks.fac_smem));
  }
  BTC_CUDA(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&bsl, ks.solve_flow, kSolveThreads, ks.fwd_smem(1)));
  g.var = ks.flow_default;
  g.ctas = std::max(1, g.occ[g.var]);
  g.fac_grid = g.ctas * g.sms;
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

// The group's persistent factorization (every level except the mixed path's top separators) with its
// configuration, then its top-separator roots (FP64 Cholesky) on the mixed path.
static int group_factor(btc_batch_s *bt, BatchGroup &g, bool roots) {
  const KernelSet &k = *g.ks;
  FactorArgs a;
  a.dpool = g.dpool;
  a.epool = g.epool;
  a.inst = bt->d_inst;
  a.info = bt->d_info;
  a.status = g.d_flow + 2;
  InstDesc none{nullptr, nullptr, 0, 0};
  int rc;
  BTC_CUDA(cudaMemsetAsync(g.d_flow, 0, 3 * sizeof(int), g.s));
  if (g.packed && (rc = k.pack_batch(g.dpool, g.epool, g.d_pack, bt->d_inst, g.n_nodes, g.s))) return rc;
  if (g.n_fac > 0) {
    BTC_CUDA(cudaMemsetAsync(g.d_flow + kFlowHeader, 0, sizeof(int) * (size_t)g.n_fac, g.s));
    a.items = g.d_fac;
    a.count = g.n_fac;
    const int32_t *deps = g.d_fac_deps;
    if ((rc = launch_n(k.flow_v[g.var].fac, std::min(g.fac_grid, g.n_fac), k.fac_threads, k.fac_smem, g.s, a, none,
                       deps, g.n_first, group_sync(g, 0))))
      return rc;
  }
  if (roots && g.n_roots_first > 0) {
    a.items = g.d_roots;
    a.count = g.n_roots_first;
    if ((rc = launch_n(k.root64_first, g.n_roots_first, k.root_threads, k.root_smem, g.s, a, none))) return rc;
  }
  if (roots && g.n_roots_rest > 0) {
    a.items = g.d_roots + g.n_roots_first;
    a.count = g.n_roots_rest;
    if ((rc = launch_n(k.root64_rest, g.n_roots_rest, k.root_threads, k.root_smem, g.s, a, none))) return rc;
  }
  return BTC_OK;
}

// Autotuner of a group's persistent factorization: every compiled residency variant (register
// budget) at 1, 2, 4, ... CTAs per SM up to what fits, three timed launches each on the batch's own
// inputs, the fastest median kept. The factor is the same in every configuration (only the schedule
// changes), so the last launch's result stands.
static int tune_group(btc_batch_s *bt, BatchGroup &g) {
  const KernelSet &k = *g.ks;
  cudaEvent_t e0, e1;
  BTC_CUDA(cudaEventCreate(&e0));
  BTC_CUDA(cudaEventCreate(&e1));
  float best = 1e30f;
  int best_v = g.var, best_c = g.ctas, rc = BTC_OK;
  for (int v = 0; v < k.n_flow_v && rc == BTC_OK; ++v)
    for (int c = 1; c <= g.occ[v] && rc == BTC_OK; c = next_ctas(c, g.occ[v])) {
      g.var = v;
      g.ctas = c;
      g.fac_grid = c * g.sms;
      float t[3];
      for (int r = 0; r < 3 && rc == BTC_OK; ++r) {
        cudaEventRecord(e0, g.s);
        rc = group_factor(bt, g, false);
        cudaEventRecord(e1, g.s);
        if (cudaEventSynchronize(e1) != cudaSuccess) rc = fail(BTC_ERR_CUDA, "batch autotune: synchronize failed");
        cudaEventElapsedTime(&t[r], e0, e1);
      }
      std::sort(t, t + 3);
      if (rc == BTC_OK && t[1] < best) {
        best = t[1];
        best_v = v;
        best_c = c;
      }
    }
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  g.var = best_v;
  g.ctas = best_c;
  g.fac_grid = best_c * g.sms;
  g.tuned = true;
  g.tuned_ms = best;
  return rc;
}

// Clear the norm slots and run every group's FP64 residual (forks onto the group streams and joins).
static int batch_residuals(btc_batch_s *bt, int with_anorm) {
  int rc;
  if ((rc = launch_n((const void *)&k_batch_clear_norms, (bt->count + 255) / 256, 256, 0, bt->stream, bt->d_norms,
                     bt->count, with_anorm)))
    return rc;
  if ((rc = batch_fork(bt))) return rc;
  for (BatchGroup &g : bt->groups) {
    const int npc = std::max(1, kResThreads / (kResParts * g.np));
    if ((rc = launch_n(g.resid, (g.n_nodes + npc - 1) / npc, kResThreads, 0, g.s, g.y, (const BatchNode *)g.d_nodes,
                       g.n_nodes, (const InstDesc *)bt->d_inst, (const BatchVec *)bt->d_vec, g.np, bt->d_norms,
                       with_anorm)))
      break;
  }
  const int rj = batch_join(bt);
  return rc ? rc : rj;
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
  return btc_batch_plan_orders(out, count, N, n, nullptr, dtype, stream);
}

int btc_batch_plan_orders(btc_batch_t *out, int count, const int *N, const int *n, const int *chunks, int dtype,
                          void *stream) {
  if (!out || count < 1 || !N || !n) return fail(BTC_ERR_ARG, "btc_batch_plan: invalid arguments");
  *out = nullptr;
  if (!dtype_ok(dtype)) return fail(BTC_ERR_ARG, "btc_batch_plan: unknown dtype %d", dtype);
  for (int k = 0; chunks && k < count; ++k)
    if (chunks[k] < 0) return fail(BTC_ERR_ARG, "btc_batch_plan_orders: instance %d: chunks %d", k, chunks[k]);
  btc_batch_s *bt = new btc_batch_s();
  bt->count = count;
  bt->dtype = dtype;
  bt->stream = (cudaStream_t)stream;
  bt->N.assign(N, N + count);
  bt->n.assign(n, n + count);
  bt->chunks.assign(count, 0);
  if (chunks) bt->chunks.assign(chunks, chunks + count);
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
  // launch order: the group with the most work first, so that its long tail of dependent upper
  // levels overlaps the smaller groups' launches
  std::stable_sort(bt->groups.begin(), bt->groups.end(),
                   [](const BatchGroup &a, const BatchGroup &b) { return a.flops > b.flops; });
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
  if ((rc = batch_alloc((void **)&bt->d_rb, sizeof(BatchReadback), acc))) return cleanup(rc);
  if ((e = cudaMallocHost(&bt->h_rb, sizeof(BatchReadback))) != cudaSuccess ||
      (e = cudaMallocHost(&bt->h_norms, 3 * count * sizeof(double))) != cudaSuccess ||
      (e = cudaMallocHost(&bt->h_info, count * sizeof(unsigned long long))) != cudaSuccess ||
      (e = cudaMallocHost(&bt->h_status, sizeof(int))) != cudaSuccess)
    return cleanup(fail(BTC_ERR_OOM, "btc_batch_plan: host staging: %s", cudaGetErrorString(e)));
  *out = bt;
  return BTC_OK;
}

int btc_dispatch_orders(int count, const int *N, const int *n, int dtype, int *chunks) {
  if (count < 1 || !N || !n || !chunks) return fail(BTC_ERR_ARG, "btc_dispatch_orders: invalid arguments");
  if (!dtype_ok(dtype)) return fail(BTC_ERR_ARG, "btc_dispatch_orders: unknown dtype %d", dtype);
  // time of one node step (us) of the one-CTA-per-node kernels by padded block size (measured on GB300 as
  // the per-node time of a lone partition chain, FP32 factor); a node with more work than a chain node's
  // potrf + trsm + syrk (7/3 n^3) takes t (0.7 + 0.3 r), r its flops over 7/3 n^3 (the dependent panel
  // chain of the Cholesky, not the products, dominates a node); one solve item takes 2 + n_p / 64 us
  auto t_node = [](int np) {
    static const int sz[] = {8, 16, 32, 48, 64, 96, 128};
    static const double us[] = {2.7, 3.5, 5.9, 9.0, 12.8, 20.0, 30.0};
    if (np <= sz[0]) return us[0];
    for (int i = 1; i < 7; ++i)
      if (np <= sz[i]) return us[i - 1] + (us[i] - us[i - 1]) * (np - sz[i - 1]) / (double)(sz[i] - sz[i - 1]);
    return us[6];
  };
  constexpr int kSolves = 2;  // a refined call: the first solve and one correction
  // every dependent launch level also waits for its producers' completion flags and stages its inputs
  // (about 1.5 us measured between a producer's end and its consumer's start, plus the input loads)
  constexpr double kLevelLatency = 2.0;
  int dev = 0, sms = 152;
  if (cudaGetDevice(&dev) == cudaSuccess) cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  cudaGetLastError();  // (no device: keep the default count)
  sms = std::max(sms, 1);
  // Per (instance, order): the persistent launches claim items level by level across the batch, so a
  // group's launch lasts about sum over levels of max(slowest item of the level, the level's work over
  // the resident CTAs); the same for the forward and backward solve levels.
  struct Profile {
    std::vector<double> fsum, fmax;  // factor work (us) and slowest item per launch level
    std::vector<int> fwd, bwd;       // solve items per level
    double work = 0.0;
  };
  auto profile = [&](int k, int c, Profile *pr) {
    const int np = padded_size(n[k], dtype);
    if (!np || np > 128) return false;
    HostPlan hp;
    if (c == 0) build_host_plan(N[k], n[k], np, 0, 0, 0, 0, &hp);
    else if (!build_partition_plan(N[k], n[k], np, c, 0, 0, 0, 0, &hp)) return false;
    const double n3 = (double)n[k] * n[k] * n[k], t = t_node(np);
    pr->fsum.assign(hp.levels, 0.0);
    pr->fmax.assign(hp.levels, 0.0);
    pr->fwd.assign(hp.levels + 1, 0);
    pr->bwd.assign(hp.levels + 1, 0);
    for (int l = 0; l < hp.levels; ++l)
      for (const FactorItem &it : hp.lv[l].fac) {
        double f = n3 / 3.0;
        if (it.p_a >= 0) f += n3;
        if (it.p_b >= 0) f += n3;
        if (it.r_down >= 0) f += 2 * n3;
        if (it.r_up >= 0) f += n3;
        if (it.fill >= 0) f += 2 * n3;
        const double us = t * (0.7 + 0.3 * f / (7.0 / 3.0 * n3));
        pr->fsum[l] += us;
        pr->fmax[l] = std::max(pr->fmax[l], us);
        pr->work += us;
      }
    if (hp.packed) {
      for (size_t q = 0; q < hp.solve_flow.size(); ++q) {
        const int key = hp.solve_key[q];
        (key > 0 ? pr->fwd : pr->bwd)[std::min(std::abs(key), hp.levels)]++;
      }
    } else {
      for (int l = 0; l < hp.levels; ++l) {
        pr->fwd[l + 1] += (int)hp.lv[l].fwd.size();
        pr->bwd[l + 1] += (int)hp.lv[l].bwd.size();
      }
    }
    return true;
  };
  // groups by padded block size, as the batch forms them
  std::map<int, std::vector<int>> groups;
  for (int k = 0; k < count; ++k) {
    const int np = N[k] >= 1 && n[k] >= 1 ? padded_size(n[k], dtype) : 0;
    if (!np || np > 128)
      return fail(BTC_ERR_UNSUPPORTED, "btc_dispatch_orders: instance %d (N = %d, n = %d)", k, N[k], n[k]);
    groups[np].push_back(k);
    chunks[k] = 0;
  }
  // profiles depend on (N, n_p, chunks) only (item times are relative to the node time)
  std::map<std::tuple<int, int, int>, Profile> cache;
  auto get = [&](int k, int c) -> const Profile * {
    const auto key = std::make_tuple(N[k], padded_size(n[k], dtype), c);
    auto it = cache.find(key);
    if (it != cache.end()) return &it->second;
    Profile pr;
    if (!profile(k, c, &pr)) return nullptr;
    return &cache.emplace(key, std::move(pr)).first->second;
  };
  double total = 0.0;
  for (int k = 0; k < count; ++k) total += get(k, 0)->work;
  static const int kChunks[] = {1, 2, 3, 4, 6, 8, 12, 16, 24, 32, 48, 64};
  // the groups run concurrently, so the batch lasts as long as its slowest group: only a group whose
  // nested-dissection makespan is the batch's may change orders, and only to shorten it
  struct Choice {
    double nd = 0.0, best = 0.0;
    int c = 0, thr = 0;
  };
  std::map<int, Choice> choice;
  for (auto &kv : groups) {
    const int np = kv.first;
    const std::vector<int> &ids = kv.second;
    const double ts = 2.0 + np / 64.0;
    double gwork = 0.0;
    for (int k : ids) gwork += get(k, 0)->work;
    // the group's share of the resident CTAs (two per SM in all), as its share of the batch's work
    const double C = std::max(0.5 * sms, 2.0 * sms * gwork / std::max(total, 1e-30));
    // makespan of a policy: systems with N <= nthr take the partition order with c chunks (when it fits),
    // the others nested dissection
    std::vector<double> fsum, fmax;
    std::vector<int> fwd, bwd;
    auto makespan = [&](int c, int nthr) {
      fsum.assign(0, 0.0);
      fmax.assign(0, 0.0);
      fwd.assign(0, 0);
      bwd.assign(0, 0);
      for (int k : ids) {
        const Profile *pr = (c > 0 && N[k] <= nthr) ? get(k, c) : nullptr;
        if (!pr) pr = get(k, 0);
        if (fsum.size() < pr->fsum.size()) {
          fsum.resize(pr->fsum.size(), 0.0);
          fmax.resize(pr->fsum.size(), 0.0);
        }
        if (fwd.size() < pr->fwd.size()) {
          fwd.resize(pr->fwd.size(), 0);
          bwd.resize(pr->fwd.size(), 0);
        }
        for (size_t l = 0; l < pr->fsum.size(); ++l) {
          fsum[l] += pr->fsum[l];
          fmax[l] = std::max(fmax[l], pr->fmax[l]);
        }
        for (size_t l = 0; l < pr->fwd.size(); ++l) {
          fwd[l] += pr->fwd[l];
          bwd[l] += pr->bwd[l];
        }
      }
      double m = 0.0;
      for (size_t l = 0; l < fsum.size(); ++l)
        if (fsum[l] > 1e-9) m += std::max(fmax[l], fsum[l] / C) + kLevelLatency;
      double sv = 0.0;
      for (size_t l = 0; l < fwd.size(); ++l) {
        if (fwd[l] > 0) sv += std::max(ts, fwd[l] * ts / C) + kLevelLatency;
        if (bwd[l] > 0) sv += std::max(ts, bwd[l] * ts / C) + kLevelLatency;
      }
      return m + kSolves * sv;
    };
    // thresholds: up to 16 quantiles of the group's sizes
    std::vector<int> sizes;
    for (int k : ids) sizes.push_back(N[k]);
    std::sort(sizes.begin(), sizes.end());
    std::vector<int> thr;
    for (int q = 1; q <= 16; ++q) thr.push_back(sizes[std::min(sizes.size() - 1, (sizes.size() * q) / 16)]);
    thr.erase(std::unique(thr.begin(), thr.end()), thr.end());
    Choice &ch = choice[np];
    ch.nd = ch.best = makespan(0, 0);
    for (int c : kChunks)
      for (int t : thr) {
        const double m = makespan(c, t);
        if (m < ch.best * (1.0 - 1e-6)) {
          ch.best = m;
          ch.c = c;
          ch.thr = t;
        }
      }
  }
  double slowest = 0.0;
  for (auto &kv : choice) slowest = std::max(slowest, kv.second.nd);
  for (auto &kv : groups) {
    const Choice &ch = choice[kv.first];
    if (ch.c == 0 || ch.nd < slowest * (1.0 - 1e-9)) continue;  // not the batch's slowest group
    for (int k : kv.second)
      if (N[k] <= ch.thr && get(k, ch.c)) chunks[k] = ch.c;
  }
  return BTC_OK;
}

int btc_batch_orders(btc_batch_t bt, int *chunks) {
  if (!bt || !chunks) return fail(BTC_ERR_ARG, "btc_batch_orders: NULL argument");
  std::copy(bt->chunks.begin(), bt->chunks.end(), chunks);
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
  for (BatchGroup &g : bt->groups) {  // largest group first: the small ones fill its tail
    if (rc) break;
    if (bt->autotune && !g.tuned && (rc = tune_group(bt, g))) break;
    rc = group_factor(bt, g, true);
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
  int it = 0;
  double worst = 0.0;
  for (;;) {
    // the first residual after a factorization also forms the matrix-norm bounds
    const int with_anorm = bt->anorm_valid ? 0 : 1;
    if ((rc = batch_residuals(bt, with_anorm))) return rc;
    bt->anorm_valid = true;
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

int btc_batch_set_autotune(btc_batch_t bt, int enable) {
  if (!bt) return fail(BTC_ERR_ARG, "btc_batch_set_autotune: NULL batch");
  bt->autotune = enable != 0;
  return BTC_OK;
}

int btc_batch_set_graphs(btc_batch_t bt, int enable) {
  if (!bt) return fail(BTC_ERR_ARG, "btc_batch_set_graphs: NULL batch");
  bt->graphs = enable != 0;
  if (bt->gexec) {
    cudaGraphExecDestroy(bt->gexec);
    bt->gexec = nullptr;
  }
  return BTC_OK;
}

int btc_batch_tuning(btc_batch_t bt, int group, int *np, int *resident_cap, int *ctas_per_sm, int *tuned,
                     double *factor_ms) {
  if (!bt || group < 0 || group >= (int)bt->groups.size()) return fail(BTC_ERR_ARG, "btc_batch_tuning: bad group");
  const BatchGroup &g = bt->groups[group];
  if (np) *np = g.np;
  if (resident_cap) *resident_cap = g.ks->flow_v[g.var].minb;
  if (ctas_per_sm) *ctas_per_sm = g.ctas;
  if (tuned) *tuned = g.tuned ? 1 : 0;
  if (factor_ms) *factor_ms = g.tuned ? g.tuned_ms : 0.0;
  return BTC_OK;
}

}  // extern "C"

namespace btc {

// Capture the batch's factor + refined solve as one executable graph: every group's persistent
// factorization and top-separator roots (forked onto the group streams), the packed first solve,
// the FP64 residuals with the matrix-norm bounds, the device-side stopping test, then a while node
// whose body (groups in turn on one stream) is one correction solve per group, the update, the
// residuals and the stopping test; finally one copy of the readback block. The instances' pointers
// are read from device arrays at run time, so the graph serves every call with the same tol and maxit.
static int build_batch_graph(btc_batch_s *bt, double tol, int maxit) {
  if (bt->gexec) {
    cudaGraphExecDestroy(bt->gexec);
    bt->gexec = nullptr;
  }
  if (!bt->gstream) {
    BTC_CUDA(cudaStreamCreateWithFlags(&bt->gstream, cudaStreamNonBlocking));
    BTC_CUDA(cudaStreamCreateWithFlags(&bt->gstream2, cudaStreamNonBlocking));
    BTC_CUDA(cudaEventCreateWithFlags(&bt->gevent, cudaEventDisableTiming));
  }
  cudaStream_t user = bt->stream;
  cudaGraph_t graph = nullptr;
  cudaGraphConditionalHandle h = 0;
  cudaError_t e = cudaStreamBeginCapture(bt->gstream, cudaStreamCaptureModeThreadLocal);
  if (e != cudaSuccess) return fail(BTC_ERR_CUDA, "batch graph capture: %s", cudaGetErrorString(e));
  bt->stream = bt->gstream;
  auto body = [&]() -> int {
    cudaStreamCaptureStatus st;
    cudaGraph_t cg = nullptr;
    BTC_CUDA(cudaStreamGetCaptureInfo(bt->gstream, &st, nullptr, &cg, nullptr, nullptr, nullptr));
    BTC_CUDA(cudaGraphConditionalHandleCreate(&h, cg, 1, cudaGraphCondAssignDefault));
    BTC_CUDA(cudaMemsetAsync(bt->d_info, 0xFF, bt->count * sizeof(unsigned long long), bt->stream));
    int rc = batch_fork(bt);
    for (BatchGroup &g : bt->groups)
      if (!rc) rc = group_factor(bt, g, true);
    const int rj = batch_join(bt);
    if (rc || (rc = rj)) return rc;
    if ((rc = batch_fork(bt))) return rc;
    for (BatchGroup &g : bt->groups) {
      int assign = 0;
      if ((rc = launch_n(g.pack, g.n_nodes, 64, 0, g.s, g.y, (const BatchNode *)g.d_nodes, (const InstDesc *)bt->d_inst,
                         (const BatchVec *)bt->d_vec, g.np)) ||
          (rc = group_solve(bt, g)) ||
          (rc = launch_n(g.unpack, g.n_nodes, 64, 0, g.s, (const void *)g.y, (const BatchNode *)g.d_nodes,
                         (const InstDesc *)bt->d_inst, (const BatchVec *)bt->d_vec, g.np, assign)))
        break;
    }
    const int rj2 = batch_join(bt);
    if (rc || (rc = rj2)) return rc;
    int one = 1, zero = 0;
    if ((rc = batch_residuals(bt, 1)) ||
        (rc = launch_n((const void *)&k_batch_decide, 1, 256, 0, bt->stream, (const double *)bt->d_norms, bt->count,
                       tol, maxit, one, (void *)bt->d_rb, h)))
      return rc;
    // the correction loop as a while node; its body runs the groups in turn on one stream
    const cudaGraphNode_t *deps = nullptr;
    const cudaGraphEdgeData *edata = nullptr;
    size_t ndeps = 0;
    BTC_CUDA(cudaStreamGetCaptureInfo(bt->gstream, &st, nullptr, &cg, &deps, &edata, &ndeps));
    alignas(cudaGraphNodeParams) unsigned char raw[sizeof(cudaGraphNodeParams)] = {};
    cudaGraphNodeParams &cp = *reinterpret_cast<cudaGraphNodeParams *>(raw);
    cp.type = cudaGraphNodeTypeConditional;
    cp.conditional.handle = h;
    cp.conditional.type = cudaGraphCondTypeWhile;
    cp.conditional.size = 1;
    cudaGraphNode_t wnode;
    BTC_CUDA(cudaGraphAddNode(&wnode, cg, deps, edata, ndeps, &cp));
    cudaGraph_t loop = cp.conditional.phGraph_out[0];
    BTC_CUDA(cudaStreamUpdateCaptureDependencies(bt->gstream, &wnode, nullptr, 1, cudaStreamSetCaptureDependencies));
    BTC_CUDA(cudaStreamBeginCaptureToGraph(bt->gstream2, loop, nullptr, nullptr, 0, cudaStreamCaptureModeThreadLocal));
    std::vector<cudaStream_t> saved;
    for (BatchGroup &g : bt->groups) {
      saved.push_back(g.s);
      g.s = bt->gstream2;
    }
    bt->stream = bt->gstream2;
    for (BatchGroup &g : bt->groups) {
      int accumulate = 1;
      if (!rc) rc = group_solve(bt, g);
      if (!rc)
        rc = launch_n(g.unpack, g.n_nodes, 64, 0, g.s, (const void *)g.y, (const BatchNode *)g.d_nodes,
                      (const InstDesc *)bt->d_inst, (const BatchVec *)bt->d_vec, g.np, accumulate);
    }
    if (!rc) {  // residuals of the groups in turn (no fork inside the loop body)
      rc = launch_n((const void *)&k_batch_clear_norms, (bt->count + 255) / 256, 256, 0, bt->stream, bt->d_norms,
                    bt->count, zero);
      for (BatchGroup &g : bt->groups) {
        const int npc = std::max(1, kResThreads / (kResParts * g.np));
        if (!rc)
          rc = launch_n(g.resid, (g.n_nodes + npc - 1) / npc, kResThreads, 0, g.s, g.y, (const BatchNode *)g.d_nodes,
                        g.n_nodes, (const InstDesc *)bt->d_inst, (const BatchVec *)bt->d_vec, g.np, bt->d_norms,
                        zero);
      }
    }
    if (!rc)
      rc = launch_n((const void *)&k_batch_decide, 1, 256, 0, bt->stream, (const double *)bt->d_norms, bt->count, tol,
                    maxit, zero, (void *)bt->d_rb, h);
    for (size_t q = 0; q < bt->groups.size(); ++q) bt->groups[q].s = saved[q];
    cudaGraph_t loop_out = nullptr;
    const cudaError_t e2 = cudaStreamEndCapture(bt->gstream2, &loop_out);
    bt->stream = bt->gstream;
    if (rc) return rc;
    if (e2 != cudaSuccess) return fail(BTC_ERR_CUDA, "batch graph capture (loop body): %s", cudaGetErrorString(e2));
    BTC_CUDA(cudaMemcpyAsync(bt->h_rb, bt->d_rb, sizeof(BatchReadback), cudaMemcpyDeviceToHost, bt->stream));
    return BTC_OK;
  };
  int rc = body();
  e = cudaStreamEndCapture(bt->gstream, &graph);
  bt->stream = user;
  if (rc == BTC_OK && e != cudaSuccess) rc = fail(BTC_ERR_CUDA, "batch graph capture: %s", cudaGetErrorString(e));
  if (rc == BTC_OK && (e = cudaGraphInstantiate(&bt->gexec, graph, 0)) != cudaSuccess)
    rc = fail(BTC_ERR_CUDA, "batch graph instantiate: %s", cudaGetErrorString(e));
  if (graph) cudaGraphDestroy(graph);
  if (rc) {
    bt->gexec = nullptr;
    cudaGetLastError();
    return rc;
  }
  bt->gtol = tol;
  bt->gmaxit = maxit;
  return BTC_OK;
}

}  // namespace btc

extern "C" {

int btc_batch_factor_solve_refined(btc_batch_t bt, const void *const *D, const void *const *B, const double *const *b,
                                   double *const *x, double tol, int maxit, int *iters, double *max_relres) {
  if (!bt || !D || !B || !b || !x || maxit < 0)
    return fail(BTC_ERR_ARG, "btc_batch_factor_solve_refined: invalid arguments");
  if (bt->dtype == BTC_F32) return fail(BTC_ERR_ARG, "btc_batch_factor_solve_refined needs an FP64 or mixed batch");
  bool settled = true;  // the groups' launch configurations are final (tuned, or tuning is off)
  if (bt->autotune)
    for (const BatchGroup &g : bt->groups) settled = settled && g.tuned;
  if (!bt->graphs || !settled) {  // plain launches (and, the first time, the tuning)
    int rc = btc_batch_factor(bt, D, B);
    return rc ? rc : btc_batch_solve_refined(bt, b, x, tol, maxit, iters, max_relres);
  }
  for (int k = 0; k < bt->count; ++k) {
    if (!D[k] || (bt->N[k] > 1 && !B[k])) return fail(BTC_ERR_ARG, "btc_batch_factor_solve_refined: instance %d", k);
    if (((uintptr_t)D[k] | (uintptr_t)B[k]) & 15) return fail(BTC_ERR_ARG, "instance %d: 16-byte alignment", k);
    bt->inst_host[k].D = D[k];
    bt->inst_host[k].B = B[k];
  }
  BTC_CUDA(cudaMemcpyAsync(bt->d_inst, bt->inst_host.data(), bt->count * sizeof(InstDesc), cudaMemcpyHostToDevice,
                           bt->stream));
  int rc = batch_set_vec(bt, (const void *const *)b, (void *const *)x);
  if (rc) return rc;
  if (!bt->gexec || bt->gtol != tol || bt->gmaxit != maxit) {
    if ((rc = build_batch_graph(bt, tol, maxit))) {
      if (rc != BTC_ERR_CUDA) return rc;
      bt->graphs = false;  // capture refused: plain launches from now on
      cudaGetLastError();
      rc = btc_batch_factor(bt, D, B);
      return rc ? rc : btc_batch_solve_refined(bt, b, x, tol, maxit, iters, max_relres);
    }
  }
  BTC_CUDA(cudaEventRecord(bt->gevent, bt->stream));
  BTC_CUDA(cudaStreamWaitEvent(bt->gstream, bt->gevent, 0));
  BTC_CUDA(cudaGraphLaunch(bt->gexec, bt->gstream));
  BTC_CUDA(cudaStreamSynchronize(bt->gstream));
  bt->factored = true;
  bt->anorm_valid = true;
  if ((rc = btc_batch_info(bt, nullptr, nullptr, nullptr))) return rc;
  if (iters) *iters = bt->h_rb->iters;
  if (max_relres) *max_relres = bt->h_rb->worst;
  if (!(bt->h_rb->worst <= tol))
    return fail(BTC_ERR_NOT_CONVERGED, "batch refinement stopped at %.3e", bt->h_rb->worst);
  return BTC_OK;
}

int btc_batch_free(btc_batch_t bt) {
  if (!bt) return BTC_OK;
  cudaStreamSynchronize(bt->stream);
  if (bt->gexec) cudaGraphExecDestroy(bt->gexec);
  if (bt->gstream) {
    cudaStreamSynchronize(bt->gstream);
    cudaStreamDestroy(bt->gstream);
    cudaStreamDestroy(bt->gstream2);
    cudaEventDestroy(bt->gevent);
  }
  if (bt->d_rb) cudaFree(bt->d_rb);
  if (bt->h_rb) cudaFreeHost(bt->h_rb);
  for (BatchGroup &g : bt->groups) {
    if (g.s) {
      cudaStreamSynchronize(g.s);
      cudaStreamDestroy(g.s);
    }
    if (g.ev) cudaEventDestroy(g.ev);
    void *ptrs[] = {g.dpool, g.epool, g.y, g.d_fac, g.d_fac_deps, g.d_roots, g.d_solve, g.d_flow, g.d_nodes,
                    g.d_pack};
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
