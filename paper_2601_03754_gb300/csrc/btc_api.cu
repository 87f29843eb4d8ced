// C ABI and runtime: plan objects, device pools, level launches and the
// refinement loop. See include/btc.h for the contract of every entry point.
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <cstdarg>
#include <cstdio>
#include <cstring>
#include <map>
#include <mutex>
#include <tuple>
#include <string>
#include <vector>

#include "../../include/btc.h"
#include "btc_factor.cuh"
#include "btc_internal.h"
#include "btc_kernels.h"
#include "btc_krylov.cuh"
#include "btc_solve.cuh"
#include "btc_runtime.h"

namespace btc {

static thread_local std::string g_err;

void set_error_message(const char *msg) { g_err = msg; }

int fail(int code, const char *fmt, ...) {
  char buf[512];
  va_list ap;
  va_start(ap, fmt);
  vsnprintf(buf, sizeof(buf), fmt, ap);
  va_end(ap);
  g_err = buf;
  return code;
}


// ------------------------------------------------------------ kernel table
static constexpr int kMaxSets = 12;
static constexpr int kDtypes = 5;
static KernelSet g_sets[kDtypes][kMaxSets];
static int g_nsets[kDtypes] = {0, 0, 0, 0, 0};
static std::once_flag g_once;

static void init_tables() {
  std::call_once(g_once, [] {
    const int code_f64 = BTC_F64, code_f32 = BTC_F32, code_mixed = BTC_MIXED_F32, code_tf32 = BTC_MIXED_TF32,
              code_bf16 = BTC_MIXED_BF16;
#define BTC_ADD_SET(dt, np) g_sets[code_##dt][g_nsets[code_##dt]++] = make_set_##dt##_##np();
    BTC_FOR_EACH_SET(BTC_ADD_SET)
#undef BTC_ADD_SET
    // below the tensor-core block size the TF32 and BF16 dtypes run the mixed FP32 sets
    for (int code : {code_tf32, code_bf16})
      for (int i = 0; i < g_nsets[code_mixed]; ++i)
        if (g_sets[code_mixed][i].np < 128) g_sets[code][g_nsets[code]++] = g_sets[code_mixed][i];
  });
}

const KernelSet &kernels_for(int dtype, int np) {
  static KernelSet none;
  init_tables();
  if (dtype < 0 || dtype >= kDtypes) return none;
  for (int i = 0; i < g_nsets[dtype]; ++i)
    if (g_sets[dtype][i].np == np) return g_sets[dtype][i];
  return none;
}

// ||Psi||_inf: max absolute row sum (lower triangles of D read), into norms[2].
__global__ void k_anorm(const double *D, const double *B, int N, int n, double *norms) {
  grid_dep_enter();
  const int i = blockIdx.x;
  const size_t bs = (size_t)n * n;
  double best = 0.0;
  for (int r = threadIdx.x; r < n; r += blockDim.x) {
    double s = 0.0;
    for (int c = 0; c < n; ++c) s += fabs(r >= c ? D[i * bs + r * n + c] : D[i * bs + c * n + r]);
    if (i > 0)
      for (int c = 0; c < n; ++c) s += fabs(B[(i - 1) * bs + r * n + c]);
    if (i + 1 < N)
      for (int c = 0; c < n; ++c) s += fabs(B[i * bs + c * n + r]);
    best = nan_max(best, s);
  }
  for (int o = 16; o > 0; o >>= 1) best = nan_max(best, __shfl_xor_sync(0xffffffffu, best, o));
  if ((threadIdx.x & 31) == 0) atomic_max_nonneg(norms + 2, best);
}

// One readback block: the norms, the pivot report, the flow status and the
// outcome of a graph-resident refinement come back to the host in one copy.
struct Readback {
  double norms[4];  // [0] max|r|, [1] max|x|, [2] ||Psi||_inf (lower bound)
  unsigned long long info;
  int status;
  int iters;   // refinement steps taken (graph-resident loop)
  double rel;  // last relative residual (graph-resident loop)
};

// Stopping test of the graph-resident refinement (one thread): relative
// residual from the norms of the residual kernel; continue while it is above
// tol, finite, and fewer than maxit steps were taken; the decision drives the
// graph's while node.
__global__ void k_refine_decide(Readback *rb, double tol, int maxit, int first, cudaGraphConditionalHandle h) {
  grid_dep_enter();
  const double rn = rb->norms[0], xn = rb->norms[1], an = rb->norms[2];
  const double rel = (an * xn > 0) ? rn / (an * xn) : rn;
  if (first) rb->iters = 0;
  const bool more = !(rel <= tol) && rel == rel && rb->iters < maxit;
  if (more) rb->iters += 1;
  rb->rel = rel;
  cudaGraphSetConditional(h, more ? 1u : 0u);
}

// The state of one persistent launch reset before it runs (its ticket and `count` completion flags),
// and optionally the launch status, the pivot report and the first `nnorms` residual norms: one small
// kernel in place of up to five memsets (fewer nodes in the captured graphs).
__global__ void k_flow_reset(int *ticket, int *flags, int count, int *status, unsigned long long *info,
                             double *norms, int nnorms) {
  grid_dep_enter();
  for (int q = blockIdx.x * blockDim.x + threadIdx.x; q < count; q += gridDim.x * blockDim.x) flags[q] = 0;
  if (blockIdx.x == 0) {
    if (threadIdx.x == 0) {
      *ticket = 0;
      if (status) *status = 0;
      if (info) *info = ~0ull;
    }
    if (threadIdx.x < nnorms) norms[threadIdx.x] = 0.0;
  }
}

// Diagonal entries of nblocks consecutive n x n FP64 blocks set to 1 (the pad blocks of a server's
// bucketed plans).
__global__ void k_set_unit_diagonal(double *D, int64_t nblocks, int n) {
  grid_dep_enter();
  const int64_t total = nblocks * n;
  for (int64_t q = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; q < total; q += (int64_t)gridDim.x * blockDim.x) {
    const int64_t b = q / n, i = q % n;
    D[(b * n + i) * n + i] = 1.0;
  }
}

int set_unit_diagonal(double *D, int64_t nblocks, int n, void *stream) {
  if (nblocks <= 0) return BTC_OK;
  return launch_n((const void *)&k_set_unit_diagonal, grid_for(nblocks * n), 256, 0, (cudaStream_t)stream, D,
                  nblocks, n);
}

bool dtype_ok(int dtype) {
  return dtype == BTC_F64 || dtype == BTC_F32 || dtype_mixed(dtype);
}
bool dtype_mixed(int dtype) { return dtype == BTC_MIXED_F32 || dtype == BTC_MIXED_TF32 || dtype == BTC_MIXED_BF16; }

}  // namespace btc

using namespace btc;

struct btc_plan_s {
  int N = 0, n = 0, np = 0, dtype = 0;
  cudaStream_t stream = nullptr;
  HostPlan hp;
  const KernelSet *ks = nullptr;
  // device memory
  void *dpool = nullptr, *epool = nullptr;
  FactorItem *d_fac = nullptr;
  FwdItem *d_fwd = nullptr;
  BwdItem *d_bwd = nullptr;
  std::vector<int64_t> fac_off, fwd_off, bwd_off;  // per level start index
  Readback *d_rb = nullptr, *h_rb = nullptr;
  unsigned long long *d_info = nullptr;  // &d_rb->info
  double *d_norms = nullptr;             // d_rb->norms
  int *d_status = nullptr;               // &d_rb->status
  void *d_y = nullptr;                   // work vector [N][np][kMaxCols]
  // persistent dataflow launches
  int sched = BTC_SCHED_FLOW;
  int variant = BTC_VARIANT_HYBRID;
  int32_t *d_fac_deps = nullptr, *d_fac_deps_rl = nullptr;
  SolveFlowItem *d_solve_flow = nullptr;
  int n_fac = 0, n_solve = 0;
  int *d_flow = nullptr;  // [0] factor ticket, [1] solve ticket, then done flags
  int fac_grid = 0, solve_grid = 0;
  // interlaced factorization + forward sweep, and the rest of the solve
  int32_t *d_inter_code = nullptr, *d_inter_deps = nullptr;
  SolveFlowItem *d_tail = nullptr;
  int n_inter = 0, n_tail = 0, inter_grid = 0;
  // small plans (KernelSet::solve_small): the solve's and the tail's items by dependency waves, for
  // the one-CTA solve; d_waves holds [solve order | solve wave offsets | tail order | tail offsets].
  // waves_* = 0: that launch stays on the persistent dataflow kernel
  int32_t *d_waves = nullptr;
  int waves_solve = 0, waves_tail = 0, small_threads_solve = 0, small_threads_tail = 0;
  int small_y_solve = 0, small_y_tail = 0;  // work-vector nodes the launch touches
  int64_t off_solve_waves = 0, off_tail_order = 0, off_tail_waves = 0;
  // persistent-kernel configuration: residency variant and CTAs per SM (autotuned)
  int sms = 0;
  int flow_var = 0, ctas_per_sm = 0;
  int inter_var = 0, inter_ctas = 0;  // the interlaced launch's own configuration
  int occ_fac[kFlowVariants] = {}, occ_fused[kFlowVariants] = {}, occ_rl[kFlowVariants] = {};
  bool autotune = true, tuned[3] = {false, false, false};  // hybrid, right-looking, interlaced launch
  bool tune_cached_only = false;  // autotune mode 2: a configuration remembered for the shape, no trials
  // executable graph of one refined factor + solve (btc_factor_solve_refined), for the pointers,
  // sizes and configuration it was captured with
  bool graphs = true;
  cudaStream_t gstream = nullptr, gstream2 = nullptr;
  cudaEvent_t gevent = nullptr;
  cudaGraphExec_t gexec = nullptr;
  std::vector<double> gkey;
  unsigned long long *trace_fac = nullptr, *trace_solve = nullptr;  // caller-owned trace buffers
  unsigned long long *phase = nullptr;                               // caller-owned per-node phase stamps
  // btc_factor_solve_host with host-resident D and B: the level-1 loads read them over the CPU-GPU link
  // and fill the staging copies s_D, s_B (which the factorization is given) for the residuals
  const void *ingD = nullptr, *ingB = nullptr;
  int root_prec = BTC_ROOT_FP64;  // top-separator Cholesky of the mixed path
  // failure-detection test hook (btc_plan_inject_stall): poll limit of the persistent launches' waits,
  // the factor item made to wait on a flag that no item sets (-1: none), that flag's index, and host
  // copies of the dependency lists to restore
  long long wait_limit = kMaxPolls;
  int stall_item = -1, stall_flag = 0;
  std::vector<int32_t> inter_code_h, inter_deps_h;
  // blocked nodes (padded n = 256): tile tasks in launch order and one completion counter per node
  TileTask *d_tiles = nullptr;
  int *d_tile_cnt = nullptr;
  int n_tiles = 0, tile_grid = 0;
  // partition orders (btc_plan_set_order): orientation of the original coupling slots for the packing pass
  int8_t *d_orient = nullptr;
  int64_t fixed_bytes = 0;  // device bytes that do not depend on the elimination order
  double *kry = nullptr;  // GMRES-IR workspace: basis, work and zero vectors, device scalars
  size_t kry_cap = 0;     // its size in doubles
  // optional per-kernel-class event timing (btc_plan_set_timing)
  bool timing = false;
  std::vector<std::pair<cudaEvent_t, cudaEvent_t>> timing_pending[BTC_TIMING_CLASSES];
  // host views of the readback block
  double *h_norms = nullptr;
  unsigned long long *h_info = nullptr;
  int *h_status = nullptr;
  // last factorization
  const void *D = nullptr, *B = nullptr;
  bool factored = false, anorm_valid = false;
  // end-to-end host path
  void *s_D = nullptr, *s_B = nullptr, *s_b = nullptr, *s_x = nullptr;
  size_t s_rhs_bytes = 0;
  int64_t device_bytes = 0;
};

namespace btc {

// Brackets the launches of one kernel class with CUDA events on the plan's
// stream when timing is enabled (resolved by btc_plan_timing).
struct KernelTimer {
  btc_plan_s *p;
  int cls;
  cudaEvent_t e0 = nullptr;
  KernelTimer(btc_plan_s *plan, int c) : p(plan), cls(c) {
    if (p->timing && cudaEventCreate(&e0) == cudaSuccess) cudaEventRecord(e0, p->stream);
  }
  ~KernelTimer() {
    cudaEvent_t e1 = nullptr;
    if (e0 && cudaEventCreate(&e1) == cudaSuccess) {
      cudaEventRecord(e1, p->stream);
      p->timing_pending[cls].push_back({e0, e1});
    } else if (e0) {
      cudaEventDestroy(e0);
    }
  }
};

static void fill_info(const HostPlan &hp, int dtype, btc_plan_info *info) {
  memset(info, 0, sizeof(*info));
  info->N = hp.N;
  info->n = hp.n;
  info->np = hp.np;
  info->levels = hp.levels;
  info->dtype = dtype;
  info->offdiag_blocks = hp.offdiag;
  info->fill_blocks = hp.fill;
  info->factor_flops = hp.factor_flops;
  info->seq_factor_flops = hp.seq_factor_flops;
  info->critical_path_flops = hp.crit_flops;
  info->critical_path_formula = hp.crit_formula;
  info->solve_flops_per_rhs = hp.solve_flops_per_rhs;
  const double w = dtype == BTC_F32 ? 4.0 : 8.0;   // caller's element size
  const double wf = dtype == BTC_F64 ? 8.0 : 4.0;  // factor element size
  const double n2 = (double)hp.n * hp.n;
  info->factor_bytes = (2.0 * hp.N - 1.0) * n2 * w + (hp.N + (double)hp.offdiag) * n2 * wf;
  info->solve_bytes = 2.0 * (hp.N + (double)hp.offdiag) * n2 * wf;
}

static int launch(const void *fn, int grid, int block, size_t smem, cudaStream_t s, void *arg) {
  if (grid <= 0) return BTC_OK;
  void *args[] = {arg};
  BTC_CUDA(launch_ex(fn, dim3(grid), dim3(block), args, smem, s));
  return BTC_OK;
}

// Allow `bytes` of dynamic shared memory for fn. The limit is per function and shared by every plan (and
// every copy of a template kernel a launcher may reach), so it is only ever raised: lowering it for a
// small plan would make a larger plan's launches fail.
int set_smem(const void *fn, size_t bytes) {
  if (!fn) return BTC_OK;
  cudaFuncAttributes fa;
  BTC_CUDA(cudaFuncGetAttributes(&fa, fn));
  if ((size_t)fa.maxDynamicSharedSizeBytes >= bytes) return BTC_OK;
  BTC_CUDA(cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)bytes));
  return BTC_OK;
}


static FlowSync flow_sync(btc_plan_s *p, int which) {
  FlowSync fs;
  fs.ticket = p->d_flow + which;
  fs.status = p->d_status;
  fs.done = p->d_flow + kFlowHeader;
  fs.trace = which == 0 ? p->trace_fac : p->trace_solve;
  fs.max_polls = p->wait_limit;
  return fs;
}

// Reset a launch's flow state (ticket `which`, `count` flags; optionally status, info, norms).
static int flow_reset(btc_plan_s *p, int which, int count, bool status, bool info, int nnorms) {
  const int grid = std::max(1, std::min((count + 255) / 256, 64));
  return launch_n((const void *)&k_flow_reset, grid, 256, 0, p->stream, p->d_flow + which, p->d_flow + kFlowHeader,
                  count, status ? p->d_status : (int *)nullptr, info ? p->d_info : (unsigned long long *)nullptr,
                  p->d_norms, nnorms);
}

// Forward + backward substitution of the work vector (m columns), Alg. 7. clear_norms: also zero the
// first clear_norms residual norms (the captured refinement folds that memset in here).
static int run_solve(btc_plan_s *p, int m, int clear_norms = 0) {
  const KernelSet &k = *p->ks;
  SolveArgs a;
  a.dpool = p->dpool;
  a.epool = p->epool;
  a.y = p->d_y;
  a.m = m;
  KernelTimer timer(p, BTC_TIME_SOLVE);
  if (m == 1 && p->waves_solve > 0 && !p->trace_solve && (p->sched == BTC_SCHED_FLOW || p->hp.packed)) {
    if (clear_norms) BTC_CUDA(cudaMemsetAsync(p->d_norms, 0, clear_norms * sizeof(double), p->stream));
    return k.solve_small(p->d_solve_flow, p->n_solve, p->dpool, p->epool, p->d_y, p->d_waves,
                         p->d_waves + p->off_solve_waves, p->waves_solve, p->small_y_solve, p->small_threads_solve,
                         p->stream);
  }
  if (p->sched == BTC_SCHED_FLOW || p->hp.packed) {  // partition orders have no per-level solve lists
    int rc = flow_reset(p, 1, p->n_solve, false, false, clear_norms);
    if (rc) return rc;
    a.items = p->d_solve_flow;
    a.count = p->n_solve;
    return launch_n(k.solve_flow, std::min(p->solve_grid, p->n_solve), kSolveThreads, k.fwd_smem(m), p->stream, a,
                    flow_sync(p, 1));
  }
  if (clear_norms) BTC_CUDA(cudaMemsetAsync(p->d_norms, 0, clear_norms * sizeof(double), p->stream));
  for (int l = 0; l < p->hp.levels; ++l) {
    a.items = p->d_fwd + p->fwd_off[l];
    a.count = (int)(p->fwd_off[l + 1] - p->fwd_off[l]);
    int rc = launch(k.fwd, a.count, kSolveThreads, k.fwd_smem(m), p->stream, &a);
    if (rc) return rc;
  }
  for (int l = p->hp.levels - 1; l >= 0; --l) {
    a.items = p->d_bwd + p->bwd_off[l];
    a.count = (int)(p->bwd_off[l + 1] - p->bwd_off[l]);
    int rc = launch(k.bwd, a.count, kSolveThreads, k.bwd_smem(m), p->stream, &a);
    if (rc) return rc;
  }
  return BTC_OK;
}

static int decode_info(btc_plan_s *p, int *block, int *col);

static int read_info(btc_plan_s *p, int *block, int *col) {
  BTC_CUDA(cudaMemcpyAsync(p->h_info, p->d_info, sizeof(unsigned long long) + sizeof(int), cudaMemcpyDeviceToHost,
                           p->stream));
  BTC_CUDA(cudaStreamSynchronize(p->stream));
  return decode_info(p, block, col);
}

// Pivot report and flow status as last copied to the host.
static int decode_info(btc_plan_s *p, int *block, int *col) {
  if (*p->h_status != 0) return BTC_ERR_TIMEOUT;
  unsigned long long v = *p->h_info;
  if (v == ~0ull) {
    if (block) *block = -1;
    if (col) *col = -1;
    return BTC_OK;
  }
  if (block) *block = (int)(v >> 20);
  if (col) *col = (int)(v & 0xFFFFF);
  return BTC_ERR_NOT_SPD;
}

// Persistent factor kernels of variant v with c CTAs per SM (0: as many as fit).
// Instance descriptor of a factorization of (D, B); while btc_factor_solve_host
// ingests host-resident inputs, the staging copies stand for them and the
// level-1 loads read the host arrays and fill the copies.
static InstDesc inst_desc(const btc_plan_s *p, const void *D, const void *B) {
  InstDesc d{D, B, p->N, p->n};
  if (p->ingD && D == p->s_D && B == p->s_B) {
    d.D = p->ingD;
    d.B = p->ingB;
    d.Dm = p->s_D;
    d.Bm = p->s_B;
  }
  return d;
}

// Configuration of the interlaced factor + forward launch: residency variant v,
// c CTAs per SM (0 or too many: as many as fit).
static void apply_inter_config(btc_plan_s *p, int v, int c) {
  const int occ = std::max(1, p->occ_fused[v]);
  c = (c <= 0 || c > occ) ? occ : c;
  p->inter_var = v;
  p->inter_ctas = c;
  p->inter_grid = c * p->sms;
}

// Configuration of the persistent factorization; the interlaced launch follows
// it until it is tuned on its own.
static void apply_flow_config(btc_plan_s *p, int v, int c) {
  const int occ = std::max(1, p->occ_fac[v]);
  c = (c <= 0 || c > occ) ? occ : c;
  p->flow_var = v;
  p->ctas_per_sm = c;
  p->fac_grid = c * p->sms;
  apply_inter_config(p, v, c);
}

// Suspends the plan's per-kernel event timing for its lifetime: tuning trial
// launches are not part of the caller's timing statistics.
struct TimingPause {
  btc_plan_s *p;
  bool was;
  explicit TimingPause(btc_plan_s *q) : p(q), was(q->timing) { q->timing = false; }
  ~TimingPause() { p->timing = was; }
};

// Process-wide memory of tuned configurations: (dtype, np, N, algorithm
// variant) -> (residency variant, CTAs per SM).
static std::mutex g_tune_mu;
static std::map<std::tuple<int, int, int, int>, std::pair<int, int>> g_tuned;

static int launch_factor_flow(btc_plan_s *p, const void *D, const void *B);

// Autotuner of the persistent factorization: times every compiled residency
// variant at every CTAs-per-SM count that fits on the caller's own D and B (the
// arithmetic does not depend on the configuration, only the schedule does) and
// keeps the fastest median of three; remembered per shape for the process.
static int autotune_flow(btc_plan_s *p, const void *D, const void *B) {
  // (the elimination order is part of the shape: chunks = 0 for nested dissection)
  const int alg = p->variant == BTC_VARIANT_RIGHT_LOOKING ? 1 : 0;
  const auto key = std::make_tuple(p->dtype, p->np, p->N, alg + 8 * p->hp.chunks);
  {
    std::lock_guard<std::mutex> lk(g_tune_mu);
    auto it = g_tuned.find(key);
    if (it != g_tuned.end()) {
      apply_flow_config(p, it->second.first, it->second.second);
      p->tuned[alg] = true;
      return BTC_OK;
    }
  }
  const KernelSet &k = *p->ks;
  if (p->tune_cached_only) {  // nothing remembered: the default configuration, no trial launches
    p->tuned[alg] = true;
    return BTC_OK;
  }
  TimingPause pause(p);
  cudaEvent_t e0, e1;
  BTC_CUDA(cudaEventCreate(&e0));
  BTC_CUDA(cudaEventCreate(&e1));
  float best = 1e30f;
  int best_v = k.flow_default, best_c = 0, rc = BTC_OK;
  for (int v = 0; v < k.n_flow_v && rc == BTC_OK; ++v) {
    const int occ = alg ? p->occ_rl[v] : p->occ_fac[v];
    for (int c = 1; c <= occ && rc == BTC_OK; c = next_ctas(c, occ)) {
      apply_flow_config(p, v, c);
      float t[3];
      for (int r = 0; r < 3 && rc == BTC_OK; ++r) {
        cudaEventRecord(e0, p->stream);
        rc = launch_factor_flow(p, D, B);
        cudaEventRecord(e1, p->stream);
        if (cudaEventSynchronize(e1) != cudaSuccess) rc = fail(BTC_ERR_CUDA, "autotune: synchronize failed");
        cudaEventElapsedTime(&t[r], e0, e1);
      }
      if (rc) break;
      std::sort(t, t + 3);
      if (t[1] < best) {
        best = t[1];
        best_v = v;
        best_c = c;
      }
    }
  }
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  if (rc) return rc;
  apply_flow_config(p, best_v, best_c);
  p->tuned[alg] = true;
  std::lock_guard<std::mutex> lk(g_tune_mu);
  g_tuned[key] = {best_v, best_c};
  return BTC_OK;
}

// Persistent factorization launch of every level except the FP64 (or double-FP32) top
// separator of the mixed path (hybrid Alg. 5, or Alg. 6 after its packing
// pass), with the plan's configuration.
static int launch_factor_flow(btc_plan_s *p, const void *D, const void *B) {
  const KernelSet &k = *p->ks;
  const FlowVariant &fv = k.flow_v[p->flow_var];
  const bool mixed_root = dtype_mixed(p->dtype);
  const int last = p->hp.levels - 1;
  const int nflow = mixed_root ? (int)p->fac_off[last] : p->n_fac;
  FactorArgs a;
  a.dpool = p->dpool;
  a.epool = p->epool;
  a.info = p->d_info;
  a.status = p->d_status;
  a.phase = p->phase;
  a.inst = nullptr;  // single instance: the descriptor travels by value in the kernel parameters
  a.items = p->d_fac;
  a.count = nflow;
  const InstDesc d = inst_desc(p, D, B);
  int rc = BTC_OK;
  const bool rl = p->variant == BTC_VARIANT_RIGHT_LOOKING;
  const int8_t *orient = p->d_orient;
  if ((rl || p->hp.packed) &&
      (rc = k.pack_pools(p->dpool, p->epool, D, B, p->N, p->n, orient, p->stream)))
    return rc;
  if ((rc = flow_reset(p, 0, nflow, true, true, 0))) return rc;
  if (nflow == 0) return BTC_OK;
  KernelTimer timer(p, BTC_TIME_FACTOR);
  if (rl) {
    int zero = 0;
    const int32_t *deps = p->d_fac_deps_rl;
    return launch_n(fv.fac_rl, std::min(p->fac_grid, nflow), k.fac_threads, k.fac_smem, p->stream, a, d, deps, zero,
                    flow_sync(p, 0));
  }
  const int nfirst = p->hp.packed ? 0 : (int)p->fac_off[1];  // items that read the caller's arrays
  const int32_t *deps = p->d_fac_deps;
  return launch_n(fv.fac, std::min(p->fac_grid, nflow), k.fac_threads, k.fac_smem, p->stream, a, d, deps, nfirst,
                  flow_sync(p, 0));
}

// The interlaced factor + forward launch over the first m columns of the packed
// work vector, with the plan's interlaced configuration.
static int launch_interlaced(btc_plan_s *p, const void *D, const void *B, int m) {
  const KernelSet &k = *p->ks;
  FactorArgs a;
  a.dpool = p->dpool;
  a.epool = p->epool;
  a.info = p->d_info;
  a.status = p->d_status;
  a.phase = p->phase;
  a.inst = nullptr;
  a.items = p->d_fac;
  a.count = p->n_inter;
  const InstDesc d = inst_desc(p, D, B);
  int rc = flow_reset(p, 0, p->n_inter, true, true, 0);
  if (rc) return rc;
  SolveArgs sa;
  sa.items = p->d_solve_flow;
  sa.count = p->hp.n_fwd;
  sa.dpool = p->dpool;
  sa.epool = p->epool;
  sa.y = p->d_y;
  sa.m = m;
  const int32_t *code = p->d_inter_code, *deps = p->d_inter_deps;
  const int nfirst = (int)p->fac_off[1];
  KernelTimer timer(p, BTC_TIME_FACTOR_FORWARD);
  return launch_n(k.flow_v[p->inter_var].fac_fwd, std::min(p->inter_grid, p->n_inter), k.fac_threads,
                  k.fused_smem(m), p->stream, a, d, sa, code, deps, nfirst, p->n_inter, flow_sync(p, 0));
}

// Autotuner of the interlaced launch, like autotune_flow but timing the fused
// kernel itself (its registers, shared memory and item mix differ from the
// plain factorization's, and so does its best residency). The launch runs the
// forward sweep in place, so the packed work vector is saved first and put back
// before every trial and at the end. Remembered per shape for the process.
static int autotune_inter(btc_plan_s *p, const void *D, const void *B, int m) {
  const auto key = std::make_tuple(p->dtype, p->np, p->N, 2);
  {
    std::lock_guard<std::mutex> lk(g_tune_mu);
    auto it = g_tuned.find(key);
    if (it != g_tuned.end()) {
      apply_inter_config(p, it->second.first, it->second.second);
      p->tuned[2] = true;
      return BTC_OK;
    }
  }
  const KernelSet &k = *p->ks;
  if (p->tune_cached_only) {
    p->tuned[2] = true;
    return BTC_OK;
  }
  TimingPause pause(p);
  const size_t ybytes = (size_t)p->N * p->np * m * k.elem;
  void *ysave = nullptr;
  BTC_CUDA(cudaMallocAsync(&ysave, ybytes, p->stream));
  int rc = BTC_OK;
  if (cudaMemcpyAsync(ysave, p->d_y, ybytes, cudaMemcpyDeviceToDevice, p->stream) != cudaSuccess)
    rc = fail(BTC_ERR_CUDA, "autotune: work vector copy failed");
  cudaEvent_t e0 = nullptr, e1 = nullptr;
  if (!rc && (cudaEventCreate(&e0) != cudaSuccess || cudaEventCreate(&e1) != cudaSuccess))
    rc = fail(BTC_ERR_CUDA, "autotune: event creation failed");
  float best = 1e30f;
  int best_v = p->inter_var, best_c = p->inter_ctas;
  for (int v = 0; v < k.n_flow_v && rc == BTC_OK; ++v) {
    for (int c = 1; c <= p->occ_fused[v] && rc == BTC_OK; c = next_ctas(c, p->occ_fused[v])) {
      apply_inter_config(p, v, c);
      float t[3];
      for (int r = 0; r < 3 && rc == BTC_OK; ++r) {
        if (cudaMemcpyAsync(p->d_y, ysave, ybytes, cudaMemcpyDeviceToDevice, p->stream) != cudaSuccess) {
          rc = fail(BTC_ERR_CUDA, "autotune: work vector copy failed");
          break;
        }
        cudaEventRecord(e0, p->stream);
        rc = launch_interlaced(p, D, B, m);
        cudaEventRecord(e1, p->stream);
        if (cudaEventSynchronize(e1) != cudaSuccess) rc = fail(BTC_ERR_CUDA, "autotune: synchronize failed");
        cudaEventElapsedTime(&t[r], e0, e1);
      }
      if (rc) break;
      std::sort(t, t + 3);
      if (t[1] < best) {
        best = t[1];
        best_v = v;
        best_c = c;
      }
    }
  }
  if (cudaMemcpyAsync(p->d_y, ysave, ybytes, cudaMemcpyDeviceToDevice, p->stream) != cudaSuccess && !rc)
    rc = fail(BTC_ERR_CUDA, "autotune: work vector copy failed");
  cudaFreeAsync(ysave, p->stream);
  if (e0) cudaEventDestroy(e0);
  if (e1) cudaEventDestroy(e1);
  if (rc) return rc;
  apply_inter_config(p, best_v, best_c);
  p->tuned[2] = true;
  std::lock_guard<std::mutex> lk(g_tune_mu);
  g_tuned[key] = {best_v, best_c};
  return BTC_OK;
}

// Factorization (Alg. 5, or Alg. 6 with the right-looking variant). m_inter > 0:
// the forward sweep over the first m_inter columns of the work vector (packed
// by the caller) is interlaced with the factorization in the same persistent
// launch (hybrid variant, persistent schedule); the caller then runs only the
// tail of the solve (run_solve_tail).
// Factorization of a plan with blocked 256 x 256 nodes: the packing pass
// (the caller's D and B, converted, into the pools in the orientation level 1
// eliminates), then one persistent launch of every node's tile tasks,
// including the top separator's.
static int tiled_factor(btc_plan_s *p, const void *D, const void *B) {
  const KernelSet &k = *p->ks;
  int rc;
  BTC_CUDA(cudaMemsetAsync(p->d_info, 0xFF, sizeof(unsigned long long), p->stream));
  BTC_CUDA(cudaMemsetAsync(p->d_status, 0, sizeof(int), p->stream));
  BTC_CUDA(cudaMemsetAsync(p->d_flow, 0, sizeof(int), p->stream));
  BTC_CUDA(cudaMemsetAsync(p->d_tile_cnt, 0, sizeof(int) * (size_t)p->n_fac, p->stream));
  if ((rc = k.pack_pools(p->dpool, p->epool, D, B, p->N, p->n, nullptr, p->stream))) return rc;
  TileArgs a;
  a.tasks = p->d_tiles;
  a.count = p->n_tiles;
  a.dpool = reinterpret_cast<float *>(p->dpool);
  a.epool = reinterpret_cast<float *>(p->epool);
  a.counters = p->d_tile_cnt;
  a.info = p->d_info;
  FlowSync fs = flow_sync(p, 0);
  fs.trace = nullptr;  // the trace buffers are sized for node items, not tile tasks
  {
    KernelTimer timer(p, BTC_TIME_FACTOR);
    if ((rc = launch_n(k.tile_flow, std::min(p->tile_grid, p->n_tiles), kTileThreads, k.tile_smem, p->stream, a,
                       fs)))
      return rc;
  }
  p->D = D;
  p->B = B;
  p->factored = true;
  p->anorm_valid = false;
  return BTC_OK;
}

static int factor_impl(btc_plan_s *p, const void *D, const void *B, int m_inter) {
  if (!p || !D || (p->N > 1 && !B)) return fail(BTC_ERR_ARG, "btc_factor: NULL argument");
  if (((uintptr_t)D | (uintptr_t)B) & 15) return fail(BTC_ERR_ARG, "btc_factor: D and B must be 16-byte aligned");
  const KernelSet &k = *p->ks;
  if (k.tiled) return tiled_factor(p, D, B);
  const bool rl = p->variant == BTC_VARIANT_RIGHT_LOOKING;
  int rc = BTC_OK;
  const bool inter = p->sched == BTC_SCHED_FLOW && !rl && m_inter > 0 && p->n_inter > 0;
  if (p->sched == BTC_SCHED_FLOW && p->autotune) {
    if (inter && !p->tuned[2] && (rc = autotune_inter(p, D, B, m_inter))) return rc;
    if (!inter && !p->tuned[rl ? 1 : 0] && (rc = autotune_flow(p, D, B))) return rc;
  }
  FactorArgs a;
  a.dpool = p->dpool;
  a.epool = p->epool;
  a.info = p->d_info;
  a.status = p->d_status;
  a.phase = p->phase;
  a.inst = nullptr;
  const InstDesc d = inst_desc(p, D, B);
  const bool mixed_root = dtype_mixed(p->dtype);
  const int last = p->hp.levels - 1;
  if (p->sched == BTC_SCHED_FLOW) {  // (the launch's reset kernel also clears the pivot report)
    if (inter) {
      rc = launch_interlaced(p, D, B, m_inter);
    } else {
      rc = launch_factor_flow(p, D, B);
    }
    if (rc) return rc;
  } else {
    // one launch per level (Alg. 5 or Alg. 6 level loops; the positions of a partition order)
    BTC_CUDA(cudaMemsetAsync(p->d_info, 0xFF, sizeof(unsigned long long), p->stream));
    BTC_CUDA(cudaMemsetAsync(p->d_status, 0, sizeof(int), p->stream));
    const int8_t *orient = p->d_orient;
    if ((rl || p->hp.packed) &&
        (rc = k.pack_pools(p->dpool, p->epool, D, B, p->N, p->n, orient, p->stream)))
      return rc;
    KernelTimer timer(p, BTC_TIME_FACTOR);
    for (int l = 0; l < p->hp.levels - (mixed_root ? 1 : 0); ++l) {
      a.items = p->d_fac + p->fac_off[l];
      a.count = (int)(p->fac_off[l + 1] - p->fac_off[l]);
      const void *fn = rl ? k.fac_rl : (l == 0 && !p->hp.packed ? k.fac_first : k.fac_rest);
      if ((rc = launch_n(fn, a.count, k.fac_threads, k.fac_smem, p->stream, a, d))) return rc;
    }
  }
  if (mixed_root) {
    a.items = p->d_fac + p->fac_off[last];
    a.count = 1;
    const bool f64 = p->root_prec == BTC_ROOT_FP64;
    const void *fn = rl ? (f64 ? k.root64_rl : k.root_rl)
                        : (last == 0 && !p->hp.packed ? (f64 ? k.root64_first : k.root_first)
                                                        : (f64 ? k.root64_rest : k.root_rest));
    KernelTimer timer(p, BTC_TIME_ROOT);
    if ((rc = launch_n(fn, 1, k.root_threads, k.root_smem, p->stream, a, d))) return rc;
  }
  p->D = D;
  p->B = B;
  p->factored = true;
  p->anorm_valid = false;
  return BTC_OK;
}

// GMRES-based iterative refinement (Carson and Higham, SIAM J. Sci. Comput.
// 2018): the correction equation Psi d = r is solved by GMRES (no restart
// within an outer step) on the left-preconditioned system M^{-1} Psi d = M^{-1} r, M = the plan's
// low-precision factor, with Psi applied in FP64 (the residual kernel with
// b = 0) and M^{-1} applied by the solve kernels in the factor's precision;
// classical Gram-Schmidt with one reorthogonalization, Givens rotations on the
// small Hessenberg matrix on the host. One right-hand side. Each outer step:
// r = b - Psi x in FP64, stop at ||r|| <= tol ||Psi|| ||x||, then at most
// `restart` Arnoldi steps until the preconditioned residual falls by
// `inner_tol`, x += V y.
static int gmres_ir_impl(btc_plan_s *p, const double *b, double *x, double tol, int max_outer, int restart,
                         double inner_tol, int *outer, int *inner, double *relres) {
  const KernelSet &k = *p->ks;
  const int64_t L = (int64_t)p->N * p->n;
  const size_t need = (size_t)(restart + 3) * L + 4 * (size_t)(restart + 2);
  if (p->kry_cap < need) {
    if (p->kry) cudaFree(p->kry);
    p->kry = nullptr;
    p->kry_cap = 0;
    BTC_CUDA(cudaMalloc(&p->kry, need * sizeof(double)));
    p->kry_cap = need;
  }
  double *V = p->kry;                        // restart + 1 basis vectors
  double *w = V + (int64_t)(restart + 1) * L;  // work vector
  double *zero = w + L;                       // b = 0 for products with Psi
  double *dh1 = zero + L, *dh2 = dh1 + (restart + 2), *dnrm = dh2 + (restart + 2), *dy = dnrm + (restart + 2);
  BTC_CUDA(cudaMemsetAsync(zero, 0, L * sizeof(double), p->stream));
  int64_t base = 0;
  int one = 1, c0 = 0, assign = 0, no_bound = 0;
  const int gv = grid_for(L);
  auto apply_precond = [&](const double *rhs_b, const double *xv, double *out, int with_anorm) -> int {
    // y = rhs_b - Psi xv (FP64, rounded to the factor precision), y <- M^{-1} y, out = y (FP64)
    int rc;
    if ((rc = k.residual(p->d_y, (const double *)p->D, (const double *)p->B, xv, rhs_b, p->N, p->n, p->np, one, base,
                         p->d_norms, with_anorm, p->stream)) ||
        (rc = run_solve(p, 1)) ||
        (rc = launch_n(k.unpack, grid_for(L), 256, 0, p->stream, (void *)out, (const void *)p->d_y, p->N, p->n, p->np,
                       one, one, c0, base, assign)))
      return rc;
    return BTC_OK;
  };
  // x0 = M^{-1} b
  int rc;
  if ((rc = launch_n(k.pack, grid_for((int64_t)p->N * p->np), 256, 0, p->stream, p->d_y, (const void *)b, p->N, p->n,
                     p->np, one, one, c0, base)) ||
      (rc = run_solve(p, 1)) ||
      (rc = launch_n(k.unpack, grid_for(L), 256, 0, p->stream, (void *)x, (const void *)p->d_y, p->N, p->n, p->np, one,
                     one, c0, base, assign)))
    return rc;
  std::vector<double> H((size_t)(restart + 1) * restart), cs(restart), sn(restart), g(restart + 1), y(restart);
  std::vector<double> hbuf(2 * (restart + 2) + 1);
  int it = 0, tot_inner = 0;
  double rel = 0.0;
  bool ok = false, info_checked = false;
  for (;;) {
    // r = b - Psi x (FP64) and z = M^{-1} r in V_0
    const int with_anorm = p->anorm_valid ? 0 : 1;
    BTC_CUDA(cudaMemsetAsync(p->d_norms, 0, (2 + with_anorm) * sizeof(double), p->stream));
    if ((rc = apply_precond(b, x, V, with_anorm))) return rc;
    if ((rc = launch_n((const void *)&k_mdot, 1, kKryThreads, 0, p->stream, (const double *)V, L, (const double *)V, L,
                       dnrm)))
      return rc;
    BTC_CUDA(cudaMemcpyAsync(p->h_rb, p->d_rb, sizeof(Readback), cudaMemcpyDeviceToHost, p->stream));
    BTC_CUDA(cudaMemcpyAsync(hbuf.data(), dnrm, sizeof(double), cudaMemcpyDeviceToHost, p->stream));
    BTC_CUDA(cudaStreamSynchronize(p->stream));
    p->anorm_valid = true;
    if (!info_checked) {
      int blk, col;
      rc = decode_info(p, &blk, &col);
      if (rc == BTC_ERR_TIMEOUT) return fail(rc, "factorization failed: a bounded device-side wait gave up");
      if (rc) return fail(rc, "factorization failed: pivot of block %d, column %d not positive", blk, col);
      info_checked = true;
    }
    const double rn = p->h_norms[0], xn = p->h_norms[1], an = p->h_norms[2];
    rel = (an * xn > 0) ? rn / (an * xn) : rn;
    if (!(rel == rel)) break;
    if (rel <= tol) {
      ok = true;
      break;
    }
    if (it >= max_outer) break;
    const double beta = std::sqrt(hbuf[0]);
    if (!(beta > 0.0)) break;
    if ((rc = launch_n((const void *)&k_vscale, gv, 256, 0, p->stream, V, (const double *)V, 1.0 / beta,
                       (const double *)nullptr, L)))
      return rc;
    std::fill(g.begin(), g.end(), 0.0);
    g[0] = beta;
    int kdim = 0;
    for (int j = 0; j < restart; ++j) {
      double *Vj = V + (int64_t)j * L, *Vn = V + (int64_t)(j + 1) * L;
      // w = M^{-1} Psi V_j: the residual kernel with b = 0 gives -Psi V_j
      if ((rc = apply_precond(zero, Vj, w, no_bound)) ||
          (rc = launch_n((const void *)&k_vscale, gv, 256, 0, p->stream, w, (const double *)w, -1.0,
                         (const double *)nullptr, L)))
        return rc;
      // classical Gram-Schmidt, twice
      const double *Vc = V;
      if ((rc = launch_n((const void *)&k_mdot, j + 1, kKryThreads, 0, p->stream, Vc, L, (const double *)w, L, dh1)) ||
          (rc = launch_n((const void *)&k_mupdate, gv, 256, 0, p->stream, w, Vc, L, (const double *)dh1, j + 1, L,
                         -1.0)) ||
          (rc = launch_n((const void *)&k_mdot, j + 1, kKryThreads, 0, p->stream, Vc, L, (const double *)w, L, dh2)) ||
          (rc = launch_n((const void *)&k_mupdate, gv, 256, 0, p->stream, w, Vc, L, (const double *)dh2, j + 1, L,
                         -1.0)) ||
          (rc = launch_n((const void *)&k_mdot, 1, kKryThreads, 0, p->stream, (const double *)w, L, (const double *)w,
                         L, dnrm)) ||
          (rc = launch_n((const void *)&k_vscale, gv, 256, 0, p->stream, Vn, (const double *)w, 0.0,
                         (const double *)dnrm, L)))
        return rc;
      BTC_CUDA(cudaMemcpyAsync(hbuf.data(), dh1, (2 * (restart + 2) + 1) * sizeof(double), cudaMemcpyDeviceToHost,
                               p->stream));
      BTC_CUDA(cudaStreamSynchronize(p->stream));
      const double *h1 = hbuf.data(), *h2 = h1 + (restart + 2);
      double *Hj = H.data() + (size_t)j * (restart + 1);  // column j
      for (int i = 0; i <= j; ++i) Hj[i] = h1[i] + h2[i];
      Hj[j + 1] = std::sqrt(std::max(h2[restart + 2], 0.0));
      // earlier rotations, then a new one that zeroes H[j+1][j]
      for (int i = 0; i < j; ++i) {
        const double a = Hj[i], c = Hj[i + 1];
        Hj[i] = cs[i] * a + sn[i] * c;
        Hj[i + 1] = -sn[i] * a + cs[i] * c;
      }
      const double a = Hj[j], c = Hj[j + 1], r = std::hypot(a, c);
      cs[j] = r > 0 ? a / r : 1.0;
      sn[j] = r > 0 ? c / r : 0.0;
      Hj[j] = r;
      Hj[j + 1] = 0.0;
      g[j + 1] = -sn[j] * g[j];
      g[j] = cs[j] * g[j];
      ++tot_inner;
      kdim = j + 1;
      if (std::fabs(g[j + 1]) <= inner_tol * beta || !(c > 0.0)) break;
    }
    // y = R^{-1} g (upper triangular kdim x kdim), x += V y
    for (int i = kdim - 1; i >= 0; --i) {
      double t = g[i];
      for (int q = i + 1; q < kdim; ++q) t -= H[(size_t)q * (restart + 1) + i] * y[q];
      const double d = H[(size_t)i * (restart + 1) + i];
      y[i] = d != 0.0 ? t / d : 0.0;
    }
    BTC_CUDA(cudaMemcpyAsync(dy, y.data(), kdim * sizeof(double), cudaMemcpyHostToDevice, p->stream));
    if ((rc = launch_n((const void *)&k_mupdate, gv, 256, 0, p->stream, x, (const double *)V, L, (const double *)dy,
                       kdim, L, 1.0)))
      return rc;
    BTC_CUDA(cudaStreamSynchronize(p->stream));  // y lives on the host stack frame
    ++it;
  }
  if (outer) *outer = it;
  if (inner) *inner = tot_inner;
  if (relres) *relres = rel;
  if (!ok) return fail(BTC_ERR_NOT_CONVERGED, "GMRES-IR stopped at relative residual %.3e", rel);
  return BTC_OK;
}

// The rest of the solve after an interlaced factorization: the top
// separator's forward item (mixed path) and the whole backward sweep, in one
// persistent launch.
static int run_solve_tail(btc_plan_s *p, int m, int clear_norms = 0) {
  const KernelSet &k = *p->ks;
  SolveArgs a;
  a.dpool = p->dpool;
  a.epool = p->epool;
  a.y = p->d_y;
  a.m = m;
  a.items = p->d_tail;
  a.count = p->n_tail;
  KernelTimer timer(p, BTC_TIME_SOLVE_TAIL);
  if (m == 1 && p->waves_tail > 0 && !p->trace_solve) {
    if (clear_norms) BTC_CUDA(cudaMemsetAsync(p->d_norms, 0, clear_norms * sizeof(double), p->stream));
    return k.solve_small(p->d_tail, p->n_tail, p->dpool, p->epool, p->d_y, p->d_waves + p->off_tail_order,
                         p->d_waves + p->off_tail_waves, p->waves_tail, p->small_y_tail, p->small_threads_tail,
                         p->stream);
  }
  int rc = flow_reset(p, 1, p->n_tail, false, false, clear_norms);
  if (rc) return rc;
  return launch_n(k.solve_flow, std::min(p->solve_grid, p->n_tail), kSolveThreads, k.fwd_smem(m), p->stream, a,
                  flow_sync(p, 1));
}

// The interlaced form needs the hybrid variant, the persistent schedule and
// right-hand sides that fit in one pass.
static bool can_interlace(const btc_plan_s *p, int m) {
  return p->variant == BTC_VARIANT_HYBRID && p->sched == BTC_SCHED_FLOW && p->ks->fac_fwd_flow && !p->hp.packed &&
         m >= 1 &&
         m <= std::min(kMaxCols, p->ks->max_cols);
}


// FP64 iterative refinement, chunk by chunk of at most max_cols columns:
// x = solve(b), then while ||b - Psi x|| > tol ||Psi|| ||x||: x += solve(r).
// first_done: the first chunk of x already holds its first solve (interlaced
// factorization). The first residual also forms the ||Psi|| bound when the
// factorization is new, and the norms, the pivot report and the flow status
// come back to the host in one copy per iteration.
static int refined_impl(btc_plan_s *p, const double *b, double *x, int nrhs, double tol, int maxit, int *iters,
                        double *relres, bool first_done) {
  const KernelSet &k = *p->ks;
  const int mc = std::min(kMaxCols, k.max_cols);
  int worst_it = 0, rc = BTC_OK;
  double worst_rel = 0.0;
  bool all_ok = true, info_checked = false;
  for (int c0 = 0; c0 < nrhs; c0 += mc) {
    const int m = std::min(mc, nrhs - c0);
    int64_t base = 0;
    int assign = 0, accumulate = 1;
    if (!(first_done && c0 == 0)) {
      if ((rc = launch_n(k.pack, grid_for((int64_t)p->N * p->np * m), 256, 0, p->stream, p->d_y, (const void *)b,
                         p->N, p->n, p->np, m, nrhs, c0, base)) ||
          (rc = run_solve(p, m)) ||
          (rc = launch_n(k.unpack, grid_for((int64_t)p->N * p->n * m), 256, 0, p->stream, (void *)x,
                         (const void *)p->d_y, p->N, p->n, p->np, m, nrhs, c0, base, assign)))
        return rc;
    }
    int it = 0;
    double rel = 0.0;
    bool ok = false;
    for (;;) {
      const int with_anorm = p->anorm_valid ? 0 : 1;
      BTC_CUDA(cudaMemsetAsync(p->d_norms, 0, (2 + with_anorm) * sizeof(double), p->stream));
      {
        KernelTimer timer(p, BTC_TIME_RESIDUAL);
        if ((rc = k.residual(p->d_y, (const double *)p->D, (const double *)p->B, (const double *)x, b, p->N, p->n,
                             p->np, m, base, p->d_norms, with_anorm, p->stream)))
          return rc;
      }
      BTC_CUDA(cudaMemcpyAsync(p->h_rb, p->d_rb, sizeof(Readback), cudaMemcpyDeviceToHost, p->stream));
      BTC_CUDA(cudaStreamSynchronize(p->stream));
      p->anorm_valid = true;
      if (!info_checked) {
        int blk, col;
        rc = decode_info(p, &blk, &col);
        if (rc == BTC_ERR_TIMEOUT) return fail(rc, "factorization failed: a bounded device-side wait gave up");
        if (rc) return fail(rc, "factorization failed: pivot of block %d, column %d not positive", blk, col);
        info_checked = true;
      }
      const double rn = p->h_norms[0], xn = p->h_norms[1], an = p->h_norms[2];
      rel = (an * xn > 0) ? rn / (an * xn) : rn;
      if (!(rel == rel)) break;  // NaN (in b, x or the factor): give up, not converged
      if (rel <= tol) {
        ok = true;
        break;
      }
      if (it >= maxit) break;
      if ((rc = run_solve(p, m))) return rc;
      if ((rc = launch_n(k.unpack, grid_for((int64_t)p->N * p->n * m), 256, 0, p->stream, (void *)x,
                         (const void *)p->d_y, p->N, p->n, p->np, m, nrhs, c0, base, accumulate)))
        return rc;
      ++it;
    }
    worst_it = std::max(worst_it, it);
    worst_rel = (rel == rel && worst_rel == worst_rel) ? std::max(worst_rel, rel) : NAN;
    all_ok = all_ok && ok;
  }
  if (iters) *iters = worst_it;
  if (relres) *relres = worst_rel;
  if (!all_ok) return fail(BTC_ERR_NOT_CONVERGED, "refinement stopped at relative residual %.3e", worst_rel);
  return BTC_OK;
}

// Key of a captured refinement graph: everything baked into it.
static std::vector<double> refine_graph_key(const btc_plan_s *p, const void *D, const void *B, const double *b,
                                            const double *x, int m, double tol, int maxit) {
  return {(double)(uintptr_t)D, (double)(uintptr_t)B, (double)(uintptr_t)b, (double)(uintptr_t)x, (double)m, tol,
          (double)maxit,        (double)p->flow_var,  (double)p->ctas_per_sm, (double)(uintptr_t)p->trace_fac,
          (double)(uintptr_t)p->trace_solve, (double)(uintptr_t)p->phase, (double)p->inter_var,
          (double)p->inter_ctas, (double)(uintptr_t)p->ingD, (double)(uintptr_t)p->ingB,
          (double)p->root_prec, (double)p->wait_limit};
}

// Capture one refined factor + solve of m <= max_cols columns as an executable
// graph: pack, interlaced factorization + forward sweep, top-separator root, solve
// tail, unpack, FP64 residual with the norm bound, stopping test; then a while
// node whose body is one correction (solve, update, residual, stopping test),
// repeated on the device until the test says stop; then one copy of the
// readback block to the host. The host synchronizes once per call.
static int build_refine_graph(btc_plan_s *p, const void *D, const void *B, const double *b, double *x, int m,
                              double tol, int maxit) {
  if (p->gexec) {
    cudaGraphExecDestroy(p->gexec);
    p->gexec = nullptr;
  }
  if (!p->gstream) {
    BTC_CUDA(cudaStreamCreateWithFlags(&p->gstream, cudaStreamNonBlocking));
    BTC_CUDA(cudaStreamCreateWithFlags(&p->gstream2, cudaStreamNonBlocking));
    BTC_CUDA(cudaEventCreateWithFlags(&p->gevent, cudaEventDisableTiming));
  }
  const KernelSet &k = *p->ks;
  cudaStream_t user = p->stream;
  cudaGraph_t g = nullptr;
  int rc = BTC_OK;
  int64_t base = 0;
  int c0 = 0, assign = 0, accumulate = 1, one = 1, zero = 0;
  cudaGraphConditionalHandle h = 0;
  cudaError_t e = cudaStreamBeginCapture(p->gstream, cudaStreamCaptureModeThreadLocal);
  if (e != cudaSuccess) return fail(BTC_ERR_CUDA, "graph capture: %s", cudaGetErrorString(e));
  p->stream = p->gstream;
  auto body_cuda = [&]() -> int {
    cudaStreamCaptureStatus st;
    cudaGraph_t cg = nullptr;
    BTC_CUDA(cudaStreamGetCaptureInfo(p->gstream, &st, nullptr, &cg, nullptr, nullptr, nullptr));
    BTC_CUDA(cudaGraphConditionalHandleCreate(&h, cg, 1, cudaGraphCondAssignDefault));
    int r;
    if ((r = launch_n(k.pack, grid_for((int64_t)p->N * p->np * m), 256, 0, p->stream, p->d_y, (const void *)b, p->N,
                      p->n, p->np, m, m, c0, base)) ||
        (r = factor_impl(p, D, B, m)) || (r = run_solve_tail(p, m, 3)) ||
        (r = launch_n(k.unpack, grid_for((int64_t)p->N * p->n * m), 256, 0, p->stream, (void *)x,
                      (const void *)p->d_y, p->N, p->n, p->np, m, m, c0, base, assign)))
      return r;
    if ((r = k.residual(p->d_y, (const double *)D, (const double *)B, (const double *)x, b, p->N, p->n, p->np, m,
                        base, p->d_norms, one, p->stream)) ||
        (r = launch_n((const void *)&k_refine_decide, 1, 1, 0, p->stream, p->d_rb, tol, maxit, one, h)))
      return r;
    // the correction loop as a while node
    const cudaGraphNode_t *deps = nullptr;
    const cudaGraphEdgeData *edata = nullptr;
    size_t ndeps = 0;
    BTC_CUDA(cudaStreamGetCaptureInfo(p->gstream, &st, nullptr, &cg, &deps, &edata, &ndeps));
    alignas(cudaGraphNodeParams) unsigned char raw[sizeof(cudaGraphNodeParams)] = {};  // zeroed, no constructor
    cudaGraphNodeParams &cp = *reinterpret_cast<cudaGraphNodeParams *>(raw);
    cp.type = cudaGraphNodeTypeConditional;
    cp.conditional.handle = h;
    cp.conditional.type = cudaGraphCondTypeWhile;
    cp.conditional.size = 1;
    cudaGraphNode_t wnode;
    BTC_CUDA(cudaGraphAddNode(&wnode, cg, deps, edata, ndeps, &cp));
    cudaGraph_t body = cp.conditional.phGraph_out[0];
    BTC_CUDA(cudaStreamUpdateCaptureDependencies(p->gstream, &wnode, nullptr, 1, cudaStreamSetCaptureDependencies));
    BTC_CUDA(cudaStreamBeginCaptureToGraph(p->gstream2, body, nullptr, nullptr, 0, cudaStreamCaptureModeThreadLocal));
    p->stream = p->gstream2;
    r = run_solve(p, m, 2);
    if (!r)
      r = launch_n(k.unpack, grid_for((int64_t)p->N * p->n * m), 256, 0, p->stream, (void *)x, (const void *)p->d_y,
                   p->N, p->n, p->np, m, m, c0, base, accumulate);
    if (!r)
      r = k.residual(p->d_y, (const double *)D, (const double *)B, (const double *)x, b, p->N, p->n, p->np, m, base,
                     p->d_norms, zero, p->stream);
    if (!r) r = launch_n((const void *)&k_refine_decide, 1, 1, 0, p->stream, p->d_rb, tol, maxit, zero, h);
    cudaGraph_t body_out = nullptr;
    cudaError_t e2 = cudaStreamEndCapture(p->gstream2, &body_out);
    p->stream = p->gstream;
    if (r) return r;
    if (e2 != cudaSuccess) return fail(BTC_ERR_CUDA, "graph capture (loop body): %s", cudaGetErrorString(e2));
    BTC_CUDA(cudaMemcpyAsync(p->h_rb, p->d_rb, sizeof(Readback), cudaMemcpyDeviceToHost, p->stream));
    return BTC_OK;
  };
  rc = body_cuda();
  e = cudaStreamEndCapture(p->gstream, &g);
  p->stream = user;
  if (rc == BTC_OK && e != cudaSuccess) rc = fail(BTC_ERR_CUDA, "graph capture: %s", cudaGetErrorString(e));
  if (rc == BTC_OK && (e = cudaGraphInstantiate(&p->gexec, g, 0)) != cudaSuccess)
    rc = fail(BTC_ERR_CUDA, "graph instantiate: %s", cudaGetErrorString(e));
  if (g) cudaGraphDestroy(g);
  if (rc) {
    p->gexec = nullptr;
    cudaGetLastError();
    return rc;
  }
  p->gkey = refine_graph_key(p, D, B, b, x, m, tol, maxit);
  return BTC_OK;
}

// The graph form applies to one column chunk with the interlaced form, once
// the persistent configuration is settled, and without per-kernel timing.
static bool can_graph(const btc_plan_s *p, int m) {
  return p->graphs && !p->timing && can_interlace(p, m) && (!p->autotune || p->tuned[2]);
}

// One refined factor + solve through the captured graph (re-captured when a
// pointer, size or configuration differs). Synchronous.
static int refine_graph_run(btc_plan_s *p, const void *D, const void *B, const double *b, double *x, int m,
                            double tol, int maxit, int *iters, double *relres) {
  if (!p->gexec || p->gkey != refine_graph_key(p, D, B, b, x, m, tol, maxit)) {
    int rc = build_refine_graph(p, D, B, b, x, m, tol, maxit);
    if (rc) return rc;
  }
  BTC_CUDA(cudaEventRecord(p->gevent, p->stream));
  BTC_CUDA(cudaStreamWaitEvent(p->gstream, p->gevent, 0));
  BTC_CUDA(cudaGraphLaunch(p->gexec, p->gstream));
  BTC_CUDA(cudaStreamSynchronize(p->gstream));
  p->D = D;
  p->B = B;
  p->factored = true;
  p->anorm_valid = true;
  int blk, col;
  int rc = decode_info(p, &blk, &col);
  if (rc == BTC_ERR_TIMEOUT) return fail(rc, "factorization failed: a bounded device-side wait gave up");
  if (rc) return fail(rc, "factorization failed: pivot of block %d, column %d not positive", blk, col);
  if (iters) *iters = p->h_rb->iters;
  if (relres) *relres = p->h_rb->rel;
  if (!(p->h_rb->rel <= tol))
    return fail(BTC_ERR_NOT_CONVERGED, "refinement stopped at relative residual %.3e", p->h_rb->rel);
  return BTC_OK;
}
}  // namespace btc

extern "C" {

int btc_version(void) { return 100; }

const char *btc_last_error(void) { return g_err.c_str(); }

int btc_describe(int N, int n, int dtype, btc_plan_info *info) {
  if (!info || N < 1 || n < 1) return fail(BTC_ERR_ARG, "btc_describe: invalid arguments");
  if (!dtype_ok(dtype)) return fail(BTC_ERR_ARG, "btc_describe: unknown dtype %d", dtype);
  int np = padded_size(n, dtype);
  if (!np) return fail(BTC_ERR_UNSUPPORTED, "block size %d exceeds the largest compiled size", n);
  HostPlan hp;
  build_host_plan(N, n, np, 0, 0, 0, 0, &hp);
  fill_info(hp, dtype, info);
  const double pe = dtype == BTC_F64 ? 8.0 : 4.0;
  info->device_bytes = (int64_t)(pe * (double)np * np * (N + std::max<int64_t>(hp.offdiag, 1)) +
                                 pe * (double)N * np * kMaxCols);
  return BTC_OK;
}

int btc_schedule(int N, int *order_out, int *levels_out) {
  if (N < 1 || !order_out) return fail(BTC_ERR_ARG, "btc_schedule: invalid arguments");
  HostPlan hp;
  build_host_plan(N, 1, 8, 0, 0, 0, 0, &hp);
  int t = 0;
  for (int l = 0; l < hp.levels; ++l)
    for (const FactorItem &it : hp.lv[l].fac) {
      order_out[t] = it.node;
      if (levels_out) levels_out[t] = l + 1;
      ++t;
    }
  return t == N ? BTC_OK : fail(BTC_ERR_ARG, "schedule covers %d of %d nodes", t, N);
}

int btc_describe_order(int N, int n, int dtype, int order, int chunks, btc_plan_info *info, int *order_out,
                       int *levels_out) {
  if (N < 1 || n < 1 || (order != BTC_ORDER_ND && order != BTC_ORDER_PARTITION) ||
      (order == BTC_ORDER_PARTITION && chunks < 1))
    return fail(BTC_ERR_ARG, "btc_describe_order: invalid arguments");
  if (!dtype_ok(dtype)) return fail(BTC_ERR_ARG, "btc_describe_order: unknown dtype %d", dtype);
  const int np = padded_size(n, dtype);
  if (!np) return fail(BTC_ERR_UNSUPPORTED, "block size %d exceeds the largest compiled size", n);
  if (order == BTC_ORDER_PARTITION && np > kTileT)
    return fail(BTC_ERR_UNSUPPORTED, "btc_describe_order: blocked 256 plans use the ND order only");
  HostPlan hp;
  if (order == BTC_ORDER_ND) build_host_plan(N, n, np, 0, 0, 0, 0, &hp);
  else if (!build_partition_plan(N, n, np, chunks, 0, 0, 0, 0, &hp))
    return fail(BTC_ERR_ARG, "btc_describe_order: %d chunks do not fit in N = %d", chunks, N);
  if (info) {
    fill_info(hp, dtype, info);
    const double pe = dtype == BTC_F64 ? 8.0 : 4.0;
    info->device_bytes = (int64_t)(pe * (double)np * np * (N + std::max<int64_t>(hp.offdiag, 1)) +
                                   pe * (double)N * np * kMaxCols);
  }
  int t = 0;
  for (int l = 0; l < hp.levels; ++l)
    for (const FactorItem &it : hp.lv[l].fac) {
      if (order_out) order_out[t] = it.node;
      if (levels_out) levels_out[t] = l + 1;
      ++t;
    }
  return t == N ? BTC_OK : fail(BTC_ERR_ARG, "schedule covers %d of %d nodes", t, N);
}

int btc_schedule_items(int N, int order, int chunks, int64_t *fac_rows, int *n_fac, int64_t *solve_rows,
                       int *n_solve, int *slot_rows, int *n_slots) {
  if (N < 1 || !n_fac || !n_solve || !n_slots || (order != BTC_ORDER_ND && order != BTC_ORDER_PARTITION))
    return fail(BTC_ERR_ARG, "btc_schedule_items: invalid arguments");
  HostPlan hp;
  if (order == BTC_ORDER_ND) build_host_plan(N, 1, 1, 0, 0, 0, 0, &hp);
  else if (chunks < 1 || !build_partition_plan(N, 1, 1, chunks, 0, 0, 0, 0, &hp))
    return fail(BTC_ERR_ARG, "btc_schedule_items: %d chunks do not fit in N = %d", chunks, N);
  int t = 0;
  for (int l = 0; l < hp.levels; ++l)
    for (const FactorItem &it : hp.lv[l].fac) {
      if (fac_rows && t < *n_fac) {
        const int64_t row[14] = {l + 1,   it.d_self, it.d_next, it.r_up,   it.r_down,           it.p_a,
                                 it.p_b,  it.fill,   it.d_prev, it.node,   it.flags,            hp.fac_deps[3 * t],
                                 hp.fac_deps[3 * t + 1], hp.fac_deps[3 * t + 2]};
        std::copy(row, row + 14, fac_rows + 14 * (size_t)t);
      }
      ++t;
    }
  *n_fac = t;
  const int ns = (int)hp.solve_flow.size();
  if (solve_rows)
    for (int q = 0; q < std::min(ns, *n_solve); ++q) {
      const SolveFlowItem &it = hp.solve_flow[q];
      const int64_t row[10] = {it.y_self, it.y_a, it.e_a, it.y_b, it.e_b, it.d_self, it.kind,
                               it.dep[0], it.dep[1], it.dep[2]};
      std::copy(row, row + 10, solve_rows + 10 * (size_t)q);
    }
  *n_solve = ns;
  const int nsl = (int)hp.offdiag;
  if (slot_rows)
    for (int q = 0; q < std::min(nsl, *n_slots); ++q) {
      slot_rows[3 * q] = hp.slot_e[q];
      slot_rows[3 * q + 1] = hp.slot_o[q];
      slot_rows[3 * q + 2] = q + 1 < N ? (hp.packed ? hp.slot_transposed[q] : ((q + 1) & 1)) : -1;
    }
  *n_slots = nsl;
  return BTC_OK;
}

int btc_schedule_interlaced(int N, int root_separate, int *kind, int *node, int *level, int *deps, int *count,
                            int *tail_count) {
  if (N < 1 || !count) return fail(BTC_ERR_ARG, "btc_schedule_interlaced: invalid arguments");
  HostPlan hp;
  build_host_plan(N, 1, 8, 0, 0, 0, 0, &hp);
  std::vector<int32_t> code, dp;
  std::vector<SolveFlowItem> tail;
  build_interlaced(hp, root_separate != 0, &code, &dp, &tail);
  std::vector<int32_t> fnode, flevel;
  for (int l = 1; l <= hp.levels; ++l)
    for (const FactorItem &it : hp.lv[l - 1].fac) {
      fnode.push_back(it.node + 1);
      flevel.push_back(l);
    }
  const int c = (int)code.size();
  if (kind && node && level && deps)
    for (int t = 0; t < std::min(c, *count); ++t) {
      const int32_t q = code[t];
      kind[t] = q >= 0 ? 0 : 1;
      node[t] = q >= 0 ? fnode[q] : hp.fwd_node[-1 - q];
      level[t] = q >= 0 ? flevel[q] : hp.fwd_level[-1 - q];
      for (int k = 0; k < kInterDeps; ++k) deps[kInterDeps * t + k] = dp[(size_t)kInterDeps * t + k];
    }
  *count = c;
  if (tail_count) *tail_count = (int)tail.size();
  return BTC_OK;
}

// Device state that depends on the plan's elimination order (p->hp): the off-diagonal pool, the
// per-level and persistent schedules, the interlaced schedule, the tile tasks, the flags, the packing
// orientation, and the launch configurations. Called by btc_plan and again by btc_plan_set_order.
static int plan_schedule(btc_plan_s *p) {
  const KernelSet &ks = *p->ks;
  const int N = p->N, n = p->n, np = p->np;
  const size_t bs = (size_t)np * np * ks.elem;
  const size_t ebytes = bs * std::max<int64_t>(p->hp.offdiag, 1);
  int rc = BTC_OK;
  cudaError_t e;
  auto cleanup = [](int code) { return code; };
  if ((e = cudaMalloc(&p->epool, ebytes)) != cudaSuccess)
    return fail(e == cudaErrorMemoryAllocation ? BTC_ERR_OOM : BTC_ERR_CUDA, "btc_plan: allocation: %s",
                cudaGetErrorString(e));
  p->device_bytes = p->fixed_bytes + (int64_t)ebytes;
  if (p->hp.packed && N > 1) {
    if ((e = cudaMalloc(&p->d_orient, p->hp.slot_transposed.size())) != cudaSuccess ||
        (e = cudaMemcpy(p->d_orient, p->hp.slot_transposed.data(), p->hp.slot_transposed.size(),
                        cudaMemcpyHostToDevice)) != cudaSuccess)
      return fail(BTC_ERR_CUDA, "btc_plan: orientation upload: %s", cudaGetErrorString(e));
  }
  // flatten the per-level schedules and upload them
  p->fac_off.clear();
  p->fwd_off.clear();
  p->bwd_off.clear();
  std::vector<FactorItem> fac;
  std::vector<FwdItem> fwd;
  std::vector<BwdItem> bwd;
  p->fac_off.push_back(0);
  p->fwd_off.push_back(0);
  p->bwd_off.push_back(0);
  for (const LevelSchedule &L : p->hp.lv) {
    fac.insert(fac.end(), L.fac.begin(), L.fac.end());
    fwd.insert(fwd.end(), L.fwd.begin(), L.fwd.end());
    bwd.insert(bwd.end(), L.bwd.begin(), L.bwd.end());
    p->fac_off.push_back((int64_t)fac.size());
    p->fwd_off.push_back((int64_t)fwd.size());
    p->bwd_off.push_back((int64_t)bwd.size());
  }
  if ((e = cudaMalloc(&p->d_fac, fac.size() * sizeof(FactorItem))) != cudaSuccess ||
      (e = cudaMalloc(&p->d_fwd, fwd.size() * sizeof(FwdItem))) != cudaSuccess ||
      (e = cudaMalloc(&p->d_bwd, bwd.size() * sizeof(BwdItem))) != cudaSuccess)
    return cleanup(fail(BTC_ERR_OOM, "btc_plan: schedule allocation: %s", cudaGetErrorString(e)));
  if ((e = cudaMemcpy(p->d_fac, fac.data(), fac.size() * sizeof(FactorItem), cudaMemcpyHostToDevice)) !=
          cudaSuccess ||
      (e = cudaMemcpy(p->d_fwd, fwd.data(), fwd.size() * sizeof(FwdItem), cudaMemcpyHostToDevice)) != cudaSuccess ||
      (e = cudaMemcpy(p->d_bwd, bwd.data(), bwd.size() * sizeof(BwdItem), cudaMemcpyHostToDevice)) != cudaSuccess)
    return cleanup(fail(BTC_ERR_CUDA, "btc_plan: schedule upload: %s", cudaGetErrorString(e)));
  p->device_bytes += (int64_t)(fac.size() * sizeof(FactorItem) + fwd.size() * sizeof(FwdItem) +
                               bwd.size() * sizeof(BwdItem));
  // dataflow form
  p->n_fac = (int)fac.size();
  p->n_solve = (int)p->hp.solve_flow.size();
  std::vector<int32_t> icode, ideps;
  std::vector<SolveFlowItem> tail;
  if (!p->hp.packed) build_interlaced(p->hp, dtype_mixed(p->dtype), &icode, &ideps, &tail);
  p->n_inter = (int)icode.size();
  p->n_tail = (int)tail.size();
  if ((e = cudaMalloc(&p->d_inter_code, std::max<size_t>(icode.size(), 1) * sizeof(int32_t))) != cudaSuccess ||
      (e = cudaMalloc(&p->d_inter_deps, std::max<size_t>(ideps.size(), 1) * sizeof(int32_t))) != cudaSuccess ||
      (e = cudaMalloc(&p->d_tail, std::max<size_t>(tail.size(), 1) * sizeof(SolveFlowItem))) != cudaSuccess)
    return cleanup(fail(BTC_ERR_OOM, "btc_plan: interlaced schedule allocation: %s", cudaGetErrorString(e)));
  if ((!icode.empty() && (e = cudaMemcpy(p->d_inter_code, icode.data(), icode.size() * sizeof(int32_t),
                                         cudaMemcpyHostToDevice)) != cudaSuccess) ||
      (!ideps.empty() && (e = cudaMemcpy(p->d_inter_deps, ideps.data(), ideps.size() * sizeof(int32_t),
                                         cudaMemcpyHostToDevice)) != cudaSuccess) ||
      (!tail.empty() && (e = cudaMemcpy(p->d_tail, tail.data(), tail.size() * sizeof(SolveFlowItem),
                                        cudaMemcpyHostToDevice)) != cudaSuccess))
    return cleanup(fail(BTC_ERR_CUDA, "btc_plan: interlaced schedule upload: %s", cudaGetErrorString(e)));
  p->device_bytes += (int64_t)((icode.size() + ideps.size()) * sizeof(int32_t) + tail.size() * sizeof(SolveFlowItem));
  p->waves_solve = p->waves_tail = 0;
  if (ks.solve_small) {  // small plans: the one-CTA solve when no wave is wider than two rounds of its warps
    std::vector<int32_t> so, sw, to, tw;
    const int ws = build_solve_waves(p->hp.solve_flow, &so, &sw);
    const int wt = tail.empty() ? -1 : build_solve_waves(tail, &to, &tw);
    auto nodes = [](const std::vector<SolveFlowItem> &v) {
      int64_t top = 0;
      for (const SolveFlowItem &it : v) top = std::max({top, it.y_self + 1, it.y_a + 1, it.y_b + 1});
      return (int)top;
    };
    p->small_y_solve = nodes(p->hp.solve_flow);
    p->small_y_tail = nodes(tail);
    auto fits = [&](int width, size_t count, int ycount, size_t nwaves) {  // shared memory within 48 KB
      return width >= 1 && width <= kSmallSolveWidth &&
             small_solve_smem((int)count, ycount, (int)nwaves, ks.np, ks.elem) <= (size_t)48 * 1024;
    };
    const bool use_s = fits(ws, p->hp.solve_flow.size(), p->small_y_solve, sw.size()),
               use_t = fits(wt, tail.size(), p->small_y_tail, tw.size());
    if (use_s || use_t) {
      std::vector<int32_t> all;
      if (use_s) all.insert(all.end(), so.begin(), so.end());
      p->off_solve_waves = (int64_t)all.size();
      if (use_s) all.insert(all.end(), sw.begin(), sw.end());
      p->off_tail_order = (int64_t)all.size();
      if (use_t) all.insert(all.end(), to.begin(), to.end());
      p->off_tail_waves = (int64_t)all.size();
      if (use_t) all.insert(all.end(), tw.begin(), tw.end());
      if ((e = cudaMalloc(&p->d_waves, all.size() * sizeof(int32_t))) != cudaSuccess)
        return cleanup(fail(BTC_ERR_OOM, "btc_plan: wave list allocation: %s", cudaGetErrorString(e)));
      if ((e = cudaMemcpy(p->d_waves, all.data(), all.size() * sizeof(int32_t), cudaMemcpyHostToDevice)) !=
          cudaSuccess)
        return cleanup(fail(BTC_ERR_CUDA, "btc_plan: wave list upload: %s", cudaGetErrorString(e)));
      p->device_bytes += (int64_t)(all.size() * sizeof(int32_t));
      const int g = std::max(1, 32 / ks.np);  // items per warp (lane groups of np lanes)
      if (use_s) {
        p->waves_solve = (int)sw.size() - 1;
        p->small_threads_solve = 32 * std::min((ws + g - 1) / g, 32);
      }
      if (use_t) {
        p->waves_tail = (int)tw.size() - 1;
        p->small_threads_tail = 32 * std::min((wt + g - 1) / g, 32);
      }
    }
  }
  if (ks.tiled) {
    std::vector<TileTask> tiles;
    std::vector<int32_t> totals;
    build_tile_tasks(p->hp, &tiles, &totals);
    p->n_tiles = (int)tiles.size();
    if ((e = cudaMalloc(&p->d_tiles, tiles.size() * sizeof(TileTask))) != cudaSuccess ||
        (e = cudaMalloc(&p->d_tile_cnt, std::max<size_t>(totals.size(), 1) * sizeof(int))) != cudaSuccess)
      return cleanup(fail(BTC_ERR_OOM, "btc_plan: tile task allocation: %s", cudaGetErrorString(e)));
    if ((e = cudaMemcpy(p->d_tiles, tiles.data(), tiles.size() * sizeof(TileTask), cudaMemcpyHostToDevice)) !=
        cudaSuccess)
      return cleanup(fail(BTC_ERR_CUDA, "btc_plan: tile task upload: %s", cudaGetErrorString(e)));
    p->device_bytes += (int64_t)(tiles.size() * sizeof(TileTask) + totals.size() * sizeof(int));
    int occ = 0;
    if ((rc = set_smem(ks.tile_flow, ks.tile_smem)) ||
        (e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, ks.tile_flow, kTileThreads, ks.tile_smem)) !=
            cudaSuccess)
      return cleanup(rc ? rc : fail(BTC_ERR_CUDA, "btc_plan: tile occupancy: %s", cudaGetErrorString(e)));
    int dev = 0, sms = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    p->tile_grid = std::max(1, occ) * std::max(1, sms);
  }
  // one flag per item of the largest launch, and one more that no item ever sets (the target of
  // btc_plan_inject_stall)
  const size_t nflags =
      kFlowHeader + (size_t)std::max(std::max(p->n_fac, p->n_solve), std::max(p->n_inter, p->n_tail)) + 1;
  p->stall_flag = (int)(nflags - 1 - kFlowHeader);
  p->inter_code_h = icode;
  p->inter_deps_h = ideps;
  if ((e = cudaMalloc(&p->d_fac_deps, p->hp.fac_deps.size() * sizeof(int32_t))) != cudaSuccess ||
      (e = cudaMalloc(&p->d_fac_deps_rl, p->hp.fac_deps_rl.size() * sizeof(int32_t))) != cudaSuccess ||
      (e = cudaMalloc(&p->d_solve_flow, p->hp.solve_flow.size() * sizeof(SolveFlowItem))) != cudaSuccess ||
      (e = cudaMalloc(&p->d_flow, nflags * sizeof(int))) != cudaSuccess)
    return cleanup(fail(BTC_ERR_OOM, "btc_plan: flow allocation: %s", cudaGetErrorString(e)));
  if ((e = cudaMemcpy(p->d_fac_deps, p->hp.fac_deps.data(), p->hp.fac_deps.size() * sizeof(int32_t),
                      cudaMemcpyHostToDevice)) != cudaSuccess ||
      (e = cudaMemcpy(p->d_fac_deps_rl, p->hp.fac_deps_rl.data(), p->hp.fac_deps_rl.size() * sizeof(int32_t),
                      cudaMemcpyHostToDevice)) != cudaSuccess ||
      (e = cudaMemcpy(p->d_solve_flow, p->hp.solve_flow.data(), p->hp.solve_flow.size() * sizeof(SolveFlowItem),
                      cudaMemcpyHostToDevice)) != cudaSuccess ||
      (e = cudaMemset(p->d_flow, 0, nflags * sizeof(int))) != cudaSuccess)
    return cleanup(fail(BTC_ERR_CUDA, "btc_plan: flow upload: %s", cudaGetErrorString(e)));
  // allow the large dynamic shared memory the kernels use
  if ((rc = set_smem(ks.fac_first, ks.fac_smem)) || (rc = set_smem(ks.fac_rest, ks.fac_smem)) ||
      (rc = set_smem(ks.root_first, ks.root_smem)) || (rc = set_smem(ks.root_rest, ks.root_smem)) ||
      (rc = set_smem(ks.root64_first, ks.root_smem)) || (rc = set_smem(ks.root64_rest, ks.root_smem)) ||
      (rc = set_smem(ks.root64_rl, ks.root_smem)) ||
      (rc = set_smem(ks.fwd, ks.fwd_smem(std::min(kMaxCols, ks.max_cols)))) ||
      (rc = set_smem(ks.bwd, ks.bwd_smem(std::min(kMaxCols, ks.max_cols)))) ||
      (rc = set_smem(ks.resid, residual_smem_bytes(n, std::min(kMaxCols, ks.max_cols)))) ||
      (rc = set_smem(ks.fac_flow, ks.fac_smem)) || (rc = set_smem(ks.fac_flow_rl, ks.fac_smem)) ||
      (rc = set_smem(ks.fac_rl, ks.fac_smem)) || (rc = set_smem(ks.root_rl, ks.root_smem)) ||
      (rc = set_smem(ks.solve_flow, ks.fwd_smem(std::min(kMaxCols, ks.max_cols)))) ||
      (rc = set_smem(ks.fac_fwd_flow, ks.fused_smem(std::min(kMaxCols, ks.max_cols)))))
    return cleanup(rc);
  {
    int dev = 0, sms = 0, bs_ = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    p->sms = std::max(1, sms);
    if ((e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&bs_, ks.solve_flow, kSolveThreads, ks.fwd_smem(1))) !=
        cudaSuccess)
      return cleanup(fail(BTC_ERR_CUDA, "btc_plan: occupancy: %s", cudaGetErrorString(e)));
    for (int v = 0; v < ks.n_flow_v; ++v) {
      const FlowVariant &fv = ks.flow_v[v];
      if ((rc = set_smem(fv.fac, ks.fac_smem)) || (rc = set_smem(fv.fac_rl, ks.fac_smem)) ||
          (rc = set_smem(fv.fac_fwd, ks.fused_smem(std::min(kMaxCols, ks.max_cols)))))
        return cleanup(rc);
      if ((e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&p->occ_fac[v], fv.fac, ks.fac_threads, ks.fac_smem)) !=
              cudaSuccess ||
          (e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&p->occ_fused[v], fv.fac_fwd, ks.fac_threads,
                                                             ks.fused_smem(1))) != cudaSuccess ||
          (e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&p->occ_rl[v], fv.fac_rl, ks.fac_threads, ks.fac_smem)) !=
              cudaSuccess)
        return cleanup(fail(BTC_ERR_CUDA, "btc_plan: occupancy: %s", cudaGetErrorString(e)));
    }
    p->solve_grid = std::max(1, bs_ * sms);
    apply_flow_config(p, ks.flow_default, 0);
  }
  return BTC_OK;
}

// Release what plan_schedule allocated (before a new elimination order is planned).
static void plan_unschedule(btc_plan_s *p) {
  if (p->stream || p->dpool) cudaStreamSynchronize(p->stream);
  if (p->gexec) {
    cudaGraphExecDestroy(p->gexec);
    p->gexec = nullptr;
  }
  void *dev[] = {p->epool,        p->d_fac,        p->d_fwd,      p->d_bwd,     p->d_fac_deps, p->d_fac_deps_rl,
                 p->d_solve_flow, p->d_flow,       p->d_inter_code, p->d_inter_deps, p->d_tail, p->d_tiles,
                 p->d_tile_cnt,   p->d_orient,     p->d_waves};
  for (void *q : dev)
    if (q) cudaFree(q);
  p->epool = nullptr;
  p->d_fac = nullptr;
  p->d_fwd = nullptr;
  p->d_bwd = nullptr;
  p->d_fac_deps = p->d_fac_deps_rl = nullptr;
  p->d_solve_flow = nullptr;
  p->d_flow = nullptr;
  p->d_inter_code = p->d_inter_deps = nullptr;
  p->d_tail = nullptr;
  p->d_tiles = nullptr;
  p->d_tile_cnt = nullptr;
  p->d_orient = nullptr;
  p->d_waves = nullptr;
  p->waves_solve = p->waves_tail = 0;
}

int btc_plan(btc_plan_t *out, int N, int n, int dtype, void *stream) {
  if (!out || N < 1 || n < 1) return fail(BTC_ERR_ARG, "btc_plan: invalid arguments (N=%d, n=%d)", N, n);
  *out = nullptr;
  if (!dtype_ok(dtype)) return fail(BTC_ERR_ARG, "btc_plan: unknown dtype %d", dtype);
  int np = padded_size(n, dtype);
  if (!np) return fail(BTC_ERR_UNSUPPORTED, "block size %d exceeds the largest compiled size", n);
  const KernelSet &ks = kernels_for(dtype, np);
  if (!ks.valid) return fail(BTC_ERR_UNSUPPORTED, "no kernels for dtype %d, np %d", dtype, np);
  btc_plan_s *p = new btc_plan_s();
  p->N = N;
  p->n = n;
  p->np = np;
  p->dtype = dtype;
  p->stream = (cudaStream_t)stream;
  p->ks = &ks;
  build_host_plan(N, n, np, 0, 0, 0, 0, &p->hp);
  int rc = BTC_OK;
  auto cleanup = [&](int code) {
    btc_free(p);
    return code;
  };
  const size_t bs = (size_t)np * np * ks.elem;
  size_t dbytes = bs * N;
  cudaError_t e;
  if ((e = cudaMalloc(&p->dpool, dbytes)) != cudaSuccess ||
      (e = cudaMalloc(&p->d_y, (size_t)N * np * kMaxCols * ks.elem)) != cudaSuccess ||
      (e = cudaMalloc(&p->d_rb, sizeof(Readback))) != cudaSuccess ||
      (e = cudaMallocHost(&p->h_rb, sizeof(Readback))) != cudaSuccess)
    return cleanup(fail(e == cudaErrorMemoryAllocation ? BTC_ERR_OOM : BTC_ERR_CUDA, "btc_plan: allocation: %s",
                        cudaGetErrorString(e)));
  p->d_norms = p->d_rb->norms;
  p->d_info = &p->d_rb->info;
  p->d_status = &p->d_rb->status;
  p->h_norms = p->h_rb->norms;
  p->h_info = &p->h_rb->info;
  p->h_status = &p->h_rb->status;
  if ((e = cudaMemset(p->d_rb, 0, sizeof(Readback))) != cudaSuccess)
    return cleanup(fail(BTC_ERR_CUDA, "btc_plan: %s", cudaGetErrorString(e)));
  p->fixed_bytes = (int64_t)(dbytes + (size_t)N * np * kMaxCols * ks.elem);
  if ((rc = plan_schedule(p))) return cleanup(rc);
  *out = p;
  return BTC_OK;
}

int btc_plan_set_trace(btc_plan_t p, void *factor_trace, void *solve_trace) {
  if (!p) return fail(BTC_ERR_ARG, "btc_plan_set_trace: NULL plan");
  p->trace_fac = (unsigned long long *)factor_trace;
  p->trace_solve = (unsigned long long *)solve_trace;
  return BTC_OK;
}

int btc_plan_set_phase_trace(btc_plan_t p, void *phase) {
  if (!p) return fail(BTC_ERR_ARG, "btc_plan_set_phase_trace: NULL plan");
  p->phase = (unsigned long long *)phase;
  return BTC_OK;
}

int btc_plan_inject_stall(btc_plan_t p, int item, int64_t max_polls) {
  if (!p) return fail(BTC_ERR_ARG, "btc_plan_inject_stall: NULL plan");
  if (p->ks->tiled) return fail(BTC_ERR_UNSUPPORTED, "btc_plan_inject_stall: not for plans of blocked 256 nodes");
  const int nflow = dtype_mixed(p->dtype) ? (int)p->fac_off[p->hp.levels - 1] : p->n_fac;
  if (item >= nflow || (item >= 0 && max_polls < 64))
    return fail(BTC_ERR_ARG, "btc_plan_inject_stall: item %d outside 0..%d or poll limit below 64", item, nflow - 1);
  BTC_CUDA(cudaStreamSynchronize(p->stream));
  // first dependency slot of `it` in the plain and in the interlaced lists (or -1)
  auto inter_slot = [&](int it) {
    for (size_t t = 0; t < p->inter_code_h.size(); ++t)
      if (p->inter_code_h[t] == it) return (int64_t)t * kInterDeps;
    return (int64_t)-1;
  };
  auto put = [&](int32_t *dst, int64_t off, int32_t v) -> int {
    if (off < 0) return BTC_OK;
    BTC_CUDA(cudaMemcpy(dst + off, &v, sizeof(int32_t), cudaMemcpyHostToDevice));
    return BTC_OK;
  };
  int rc;
  if (p->stall_item >= 0) {  // restore the planner's dependency lists
    const int it = p->stall_item;
    const int64_t si = inter_slot(it);
    if ((rc = put(p->d_fac_deps, 3 * (int64_t)it, p->hp.fac_deps[3 * (size_t)it])) ||
        (rc = put(p->d_inter_deps, si, si >= 0 ? p->inter_deps_h[si] : -1)))
      return rc;
    p->stall_item = -1;
  }
  p->wait_limit = kMaxPolls;
  if (item < 0) return BTC_OK;
  if ((rc = put(p->d_fac_deps, 3 * (int64_t)item, p->stall_flag)) ||
      (rc = put(p->d_inter_deps, inter_slot(item), p->stall_flag)))
    return rc;
  p->stall_item = item;
  p->wait_limit = max_polls;
  return BTC_OK;
}

int btc_plan_set_order(btc_plan_t p, int order, int chunks) {
  if (!p || (order != BTC_ORDER_ND && order != BTC_ORDER_PARTITION) || (order == BTC_ORDER_PARTITION && chunks < 1))
    return fail(BTC_ERR_ARG, "btc_plan_set_order: invalid arguments");
  if (p->ks->tiled) return fail(BTC_ERR_UNSUPPORTED, "btc_plan_set_order: blocked 256 plans use the ND order only");
  if (order == BTC_ORDER_PARTITION && p->variant == BTC_VARIANT_RIGHT_LOOKING)
    return fail(BTC_ERR_UNSUPPORTED, "btc_plan_set_order: the right-looking variant needs the nested-dissection order");
  HostPlan hp;
  if (order == BTC_ORDER_ND) {
    build_host_plan(p->N, p->n, p->np, 0, 0, 0, 0, &hp);
  } else if (!build_partition_plan(p->N, p->n, p->np, chunks, 0, 0, 0, 0, &hp)) {
    return fail(BTC_ERR_ARG, "btc_plan_set_order: %d chunks do not fit in N = %d", chunks, p->N);
  }
  plan_unschedule(p);
  p->hp = std::move(hp);
  p->stall_item = -1;
  p->wait_limit = kMaxPolls;
  p->factored = false;
  p->anorm_valid = false;
  p->tuned[0] = p->tuned[1] = p->tuned[2] = false;
  return plan_schedule(p);
}

int btc_plan_set_root_precision(btc_plan_t p, int precision) {
  if (!p || (precision != BTC_ROOT_DOUBLE_FP32 && precision != BTC_ROOT_FP64))
    return fail(BTC_ERR_ARG, "btc_plan_set_root_precision: invalid arguments");
  p->root_prec = precision;
  return BTC_OK;
}

int btc_plan_set_variant(btc_plan_t p, int variant) {
  if (!p || (variant != BTC_VARIANT_HYBRID && variant != BTC_VARIANT_RIGHT_LOOKING))
    return fail(BTC_ERR_ARG, "btc_plan_set_variant: invalid arguments");
  if (variant == BTC_VARIANT_RIGHT_LOOKING && p->hp.packed)
    return fail(BTC_ERR_UNSUPPORTED, "btc_plan_set_variant: the right-looking variant needs the nested-dissection order");
  p->variant = variant;
  return BTC_OK;
}

int btc_plan_set_stream(btc_plan_t p, void *stream) {
  if (!p) return fail(BTC_ERR_ARG, "btc_plan_set_stream: NULL plan");
  p->stream = (cudaStream_t)stream;
  return BTC_OK;
}

int btc_plan_set_schedule(btc_plan_t p, int mode) {
  if (!p || (mode != BTC_SCHED_LEVELS && mode != BTC_SCHED_FLOW))
    return fail(BTC_ERR_ARG, "btc_plan_set_schedule: invalid arguments");
  p->sched = mode;
  return BTC_OK;
}

int btc_plan_query(btc_plan_t p, btc_plan_info *info) {
  if (!p || !info) return fail(BTC_ERR_ARG, "btc_plan_query: NULL argument");
  fill_info(p->hp, p->dtype, info);
  info->device_bytes = p->device_bytes;
  return BTC_OK;
}

int btc_factor(btc_plan_t p, const void *D, const void *B) { return factor_impl(p, D, B, 0); }

int btc_solve(btc_plan_t p, void *rhs, int nrhs) {
  if (!p || !rhs || nrhs < 1) return fail(BTC_ERR_ARG, "btc_solve: invalid arguments");
  if (!p->factored) return fail(BTC_ERR_NOT_FACTORED, "btc_solve: no factorization");
  const KernelSet &k = *p->ks;
  const int mc = std::min(kMaxCols, k.max_cols);
  for (int c0 = 0; c0 < nrhs; c0 += mc) {
    const int m = std::min(mc, nrhs - c0);
    int64_t base = 0;
    int rc = launch_n(k.pack, grid_for((int64_t)p->N * p->np * m), 256, 0, p->stream, p->d_y, (const void *)rhs,
                      p->N, p->n, p->np, m, nrhs, c0, base);
    if (rc) return rc;
    if ((rc = run_solve(p, m))) return rc;
    int acc = 0;
    rc = launch_n(k.unpack, grid_for((int64_t)p->N * p->n * m), 256, 0, p->stream, rhs, (const void *)p->d_y, p->N,
                  p->n, p->np, m, nrhs, c0, base, acc);
    if (rc) return rc;
  }
  return BTC_OK;
}

int btc_solve_refined(btc_plan_t p, const double *b, double *x, int nrhs, double tol, int maxit, int *iters,
                      double *relres) {
  if (!p || !b || !x || nrhs < 1 || maxit < 0) return fail(BTC_ERR_ARG, "btc_solve_refined: invalid arguments");
  if (p->dtype == BTC_F32) return fail(BTC_ERR_ARG, "btc_solve_refined needs an FP64 or mixed plan");
  const int mc = std::min(kMaxCols, p->ks->max_cols);
  if (nrhs > mc) return fail(BTC_ERR_UNSUPPORTED, "btc_solve_refined: at most %d right-hand sides for this plan", mc);
  if (!p->factored) return fail(BTC_ERR_NOT_FACTORED, "btc_solve_refined: no factorization");
  return refined_impl(p, b, x, nrhs, tol, maxit, iters, relres, false);
}

int btc_solve_gmres_ir(btc_plan_t p, const double *b, double *x, double tol, int max_outer, int restart,
                       double inner_tol, int *outer, int *inner, double *relres) {
  if (!p || !b || !x || max_outer < 0 || restart < 1 || restart > 200 || !(inner_tol > 0.0) || !(inner_tol < 1.0))
    return fail(BTC_ERR_ARG, "btc_solve_gmres_ir: invalid arguments");
  if (p->dtype == BTC_F32) return fail(BTC_ERR_ARG, "btc_solve_gmres_ir needs an FP64 or mixed plan");
  if (!p->factored) return fail(BTC_ERR_NOT_FACTORED, "btc_solve_gmres_ir: no factorization");
  return gmres_ir_impl(p, b, x, tol, max_outer, restart, inner_tol, outer, inner, relres);
}

int btc_factor_solve(btc_plan_t p, const void *D, const void *B, void *rhs, int nrhs) {
  if (!p || !rhs || nrhs < 1) return fail(BTC_ERR_ARG, "btc_factor_solve: invalid arguments");
  if (!can_interlace(p, nrhs)) {
    int rc = btc_factor(p, D, B);
    return rc ? rc : btc_solve(p, rhs, nrhs);
  }
  const KernelSet &k = *p->ks;
  int64_t base = 0;
  int c0 = 0, assign = 0;
  int rc = launch_n(k.pack, grid_for((int64_t)p->N * p->np * nrhs), 256, 0, p->stream, p->d_y, (const void *)rhs,
                    p->N, p->n, p->np, nrhs, nrhs, c0, base);
  if (rc || (rc = factor_impl(p, D, B, nrhs)) || (rc = run_solve_tail(p, nrhs))) return rc;
  return launch_n(k.unpack, grid_for((int64_t)p->N * p->n * nrhs), 256, 0, p->stream, rhs, (const void *)p->d_y,
                  p->N, p->n, p->np, nrhs, nrhs, c0, base, assign);
}

int btc_factor_solve_refined(btc_plan_t p, const void *D, const void *B, const double *b, double *x, int nrhs,
                             double tol, int maxit, int *iters, double *relres) {
  if (!p || !b || !x || nrhs < 1 || maxit < 0) return fail(BTC_ERR_ARG, "btc_factor_solve_refined: invalid arguments");
  if (p->dtype == BTC_F32) return fail(BTC_ERR_ARG, "btc_factor_solve_refined needs an FP64 or mixed plan");
  const int mc = std::min(kMaxCols, p->ks->max_cols);
  if (nrhs > mc)
    return fail(BTC_ERR_UNSUPPORTED, "btc_factor_solve_refined: at most %d right-hand sides for this plan", mc);
  if (!can_interlace(p, nrhs)) {
    int rc = btc_factor(p, D, B);
    return rc ? rc : btc_solve_refined(p, b, x, nrhs, tol, maxit, iters, relres);
  }
  if (!D || (p->N > 1 && !B)) return fail(BTC_ERR_ARG, "btc_factor_solve_refined: NULL argument");
  if (can_graph(p, nrhs)) {
    int rc = refine_graph_run(p, D, B, b, x, nrhs, tol, maxit, iters, relres);
    if (rc != BTC_ERR_CUDA) return rc;
    p->graphs = false;  // capture or launch refused: continue without graphs for this plan
    cudaGetLastError();
  }
  const KernelSet &k = *p->ks;
  int64_t base = 0;
  int c0 = 0, assign = 0;
  int rc = launch_n(k.pack, grid_for((int64_t)p->N * p->np * nrhs), 256, 0, p->stream, p->d_y, (const void *)b, p->N,
                    p->n, p->np, nrhs, nrhs, c0, base);
  if (rc || (rc = factor_impl(p, D, B, nrhs)) || (rc = run_solve_tail(p, nrhs))) return rc;
  if ((rc = launch_n(k.unpack, grid_for((int64_t)p->N * p->n * nrhs), 256, 0, p->stream, (void *)x,
                     (const void *)p->d_y, p->N, p->n, p->np, nrhs, nrhs, c0, base, assign)))
    return rc;
  return refined_impl(p, b, x, nrhs, tol, maxit, iters, relres, true);
}

// Device address of page-locked host memory (registered or allocated through CUDA), or null.
static const void *device_view_of_host(const void *h) {
  if (!h) return nullptr;
  cudaPointerAttributes a;
  if (cudaPointerGetAttributes(&a, h) != cudaSuccess) {
    cudaGetLastError();
    return nullptr;
  }
  return a.type == cudaMemoryTypeHost ? a.devicePointer : nullptr;
}

int btc_factor_solve_host(btc_plan_t p, const void *D, const void *B, const void *b, void *x, int nrhs, double tol,
                          int maxit, int *iters, double *relres) {
  if (!p || !D || (p->N > 1 && !B) || !b || !x || nrhs < 1) return fail(BTC_ERR_ARG, "btc_factor_solve_host: args");
  const size_t w = p->ks->src_elem;
  const size_t nb = (size_t)p->n * p->n * w;
  const size_t rbytes = (size_t)p->N * p->n * nrhs * w;
  if (!p->s_D) {
    BTC_CUDA(cudaMalloc(&p->s_D, nb * p->N));
    BTC_CUDA(cudaMalloc(&p->s_B, nb * std::max(p->N - 1, 1)));
  }
  if (p->s_rhs_bytes < rbytes) {
    if (p->s_b) cudaFree(p->s_b);
    if (p->s_x) cudaFree(p->s_x);
    p->s_b = p->s_x = nullptr;
    BTC_CUDA(cudaMalloc(&p->s_b, rbytes));
    BTC_CUDA(cudaMalloc(&p->s_x, rbytes));
    p->s_rhs_bytes = rbytes;
  }
  // D and B in page-locked host memory that the GPU addresses: the level-1 loads read them over the
  // CPU-GPU link (D's lower triangles only) while the factorization runs, and fill s_D, s_B for the
  // residuals; otherwise both are copied first
  const void *hD = device_view_of_host(D), *hB = p->N > 1 ? device_view_of_host(B) : nullptr;
  const bool ingest = p->dtype != BTC_F32 && p->N > 1 && hD && hB && !((((uintptr_t)hD) | ((uintptr_t)hB)) & 7) &&
                      p->variant == BTC_VARIANT_HYBRID && p->sched == BTC_SCHED_FLOW && !p->ks->tensor_cores &&
                      !p->hp.packed;  // (a packing pass, not the level-1 loads, reads a partition plan's inputs)
  struct IngestGuard {
    btc_plan_s *p;
    ~IngestGuard() { p->ingD = p->ingB = nullptr; }
  } guard{p};
  if (ingest) {
    p->ingD = hD;
    p->ingB = hB;
  } else {
    BTC_CUDA(cudaMemcpyAsync(p->s_D, D, nb * p->N, cudaMemcpyHostToDevice, p->stream));
    if (p->N > 1) BTC_CUDA(cudaMemcpyAsync(p->s_B, B, nb * (p->N - 1), cudaMemcpyHostToDevice, p->stream));
  }
  BTC_CUDA(cudaMemcpyAsync(p->s_b, b, rbytes, cudaMemcpyHostToDevice, p->stream));
  int rc = BTC_OK;
  if (p->dtype == BTC_F32) {
    BTC_CUDA(cudaMemcpyAsync(p->s_x, p->s_b, rbytes, cudaMemcpyDeviceToDevice, p->stream));
    if ((rc = btc_factor_solve(p, p->s_D, p->s_B, p->s_x, nrhs))) return rc;
    int blk, col;
    if ((rc = read_info(p, &blk, &col))) return fail(rc, "pivot of block %d, column %d not positive", blk, col);
    if (iters) *iters = 0;
    if (relres) *relres = -1.0;
  } else {
    rc = btc_factor_solve_refined(p, p->s_D, p->s_B, (const double *)p->s_b, (double *)p->s_x, nrhs, tol, maxit, iters,
                                  relres);
    if (rc && rc != BTC_ERR_NOT_CONVERGED) return rc;
    if (rc) {
      std::string keep = g_err;
      BTC_CUDA(cudaMemcpyAsync(x, p->s_x, rbytes, cudaMemcpyDeviceToHost, p->stream));
      BTC_CUDA(cudaStreamSynchronize(p->stream));
      g_err = keep;
      return rc;
    }
  }
  BTC_CUDA(cudaMemcpyAsync(x, p->s_x, rbytes, cudaMemcpyDeviceToHost, p->stream));
  BTC_CUDA(cudaStreamSynchronize(p->stream));
  return BTC_OK;
}

int btc_info(btc_plan_t p, int *block, int *col) {
  if (!p) return fail(BTC_ERR_ARG, "btc_info: NULL plan");
  if (!p->factored) {
    if (block) *block = -1;
    if (col) *col = -1;
    return BTC_OK;
  }
  int rc = read_info(p, block, col);
  if (rc == BTC_ERR_NOT_SPD) return fail(rc, "pivot not positive");
  if (rc == BTC_ERR_TIMEOUT) return fail(rc, "a bounded device-side wait gave up");
  return rc;
}

int btc_get_factor(btc_plan_t p, void *Dhat, void *U, int *pairs) {
  if (!p) return fail(BTC_ERR_ARG, "btc_get_factor: NULL plan");
  BTC_CUDA(cudaStreamSynchronize(p->stream));
  const size_t w = p->ks->elem, np = p->np, n = p->n;
  const size_t bs = np * np * w;
  if (Dhat) {
    std::vector<char> buf(bs * p->N);
    BTC_CUDA(cudaMemcpy(buf.data(), p->dpool, buf.size(), cudaMemcpyDeviceToHost));
    // the pool holds the upper factor U_e = L(e,e)^T: transpose on the way out
    for (int i = 0; i < p->N; ++i)
      for (size_t r = 0; r < n; ++r)
        for (size_t c = 0; c < n; ++c)
          memcpy((char *)Dhat + ((size_t)i * n * n + r * n + c) * w, buf.data() + i * bs + (c * np + r) * w, w);
  }
  if (U && p->hp.offdiag > 0) {
    std::vector<char> buf(bs * p->hp.offdiag);
    BTC_CUDA(cudaMemcpy(buf.data(), p->epool, buf.size(), cudaMemcpyDeviceToHost));
    for (int64_t s = 0; s < p->hp.offdiag; ++s)
      for (size_t r = 0; r < n; ++r)
        memcpy((char *)U + ((size_t)s * n * n + r * n) * w, buf.data() + s * bs + r * np * w, n * w);
  }
  if (pairs)
    for (int64_t s = 0; s < p->hp.offdiag; ++s) {
      pairs[2 * s] = p->hp.slot_e[s];
      pairs[2 * s + 1] = p->hp.slot_o[s];
    }
  return BTC_OK;
}

int btc_residual(int N, int n, int nrhs, const double *D, const double *B, const double *x, const double *b,
                 double *out3, void *stream) {
  if (N < 1 || n < 1 || nrhs < 1 || !D || (N > 1 && !B) || !x || !b || !out3)
    return fail(BTC_ERR_ARG, "btc_residual: invalid arguments");
  cudaStream_t s = (cudaStream_t)stream;
  double *d = nullptr;
  BTC_CUDA(cudaMallocAsync((void **)&d, 3 * sizeof(double), s));
  int rc = BTC_OK;
  cudaError_t e = cudaMemsetAsync(d, 0, 3 * sizeof(double), s);
  const size_t rsm = residual_smem_bytes(n, nrhs);
  if (rsm > 220 * 1024) return fail(BTC_ERR_UNSUPPORTED, "btc_residual: n * nrhs too large for one block row");
  const void *rk = (const void *)&k_residual<double>;
  if (e == cudaSuccess && (rc = set_smem(rk, rsm))) e = cudaErrorInvalidValue;
  if (e == cudaSuccess) {
    rc = launch_n((const void *)&k_anorm, N, 64, 0, s, D, B, N, n, d);
    if (!rc) rc = launch_residual<double>(nullptr, D, B, x, b, N, n, n, nrhs, 0, d, 0, s);
  }
  double h[3] = {0, 0, 0};
  if (e == cudaSuccess && !rc) e = cudaMemcpyAsync(h, d, sizeof(h), cudaMemcpyDeviceToHost, s);
  cudaFreeAsync(d, s);
  cudaError_t e2 = cudaStreamSynchronize(s);
  if (e != cudaSuccess) return fail(BTC_ERR_CUDA, "btc_residual: %s", cudaGetErrorString(e));
  if (rc) return rc;
  if (e2 != cudaSuccess) return fail(BTC_ERR_CUDA, "btc_residual: %s", cudaGetErrorString(e2));
  out3[0] = h[0];
  out3[1] = h[2];
  out3[2] = h[1];
  return BTC_OK;
}

int btc_plan_set_autotune(btc_plan_t p, int enable) {
  if (!p || enable < 0 || enable > 2) return fail(BTC_ERR_ARG, "btc_plan_set_autotune: invalid arguments");
  p->autotune = enable != 0;
  p->tune_cached_only = enable == 2;
  p->tuned[0] = p->tuned[1] = p->tuned[2] = false;
  if (!p->autotune) {
    apply_flow_config(p, p->ks->flow_default, 0);
    p->tuned[0] = p->tuned[1] = p->tuned[2] = false;
  }
  return BTC_OK;
}

int btc_plan_set_flow_config(btc_plan_t p, int resident_cap, int ctas_per_sm) {
  if (!p) return fail(BTC_ERR_ARG, "btc_plan_set_flow_config: NULL plan");
  for (int v = 0; v < p->ks->n_flow_v; ++v)
    if (p->ks->flow_v[v].minb == resident_cap) {
      if (ctas_per_sm < 0 || ctas_per_sm > p->occ_fac[v])
        return fail(BTC_ERR_ARG, "btc_plan_set_flow_config: %d CTAs per SM do not fit (at most %d)", ctas_per_sm,
                    p->occ_fac[v]);
      p->autotune = false;
      p->tuned[0] = p->tuned[1] = p->tuned[2] = false;
      apply_flow_config(p, v, ctas_per_sm);
      return BTC_OK;
    }
  return fail(BTC_ERR_UNSUPPORTED, "btc_plan_set_flow_config: no variant compiled for a cap of %d", resident_cap);
}

int btc_plan_flow_configs(btc_plan_t p, int *caps, int *max_ctas, int *count) {
  if (!p || !count) return fail(BTC_ERR_ARG, "btc_plan_flow_configs: NULL argument");
  const int n = std::min(*count, p->ks->n_flow_v);
  for (int v = 0; v < n; ++v) {
    if (caps) caps[v] = p->ks->flow_v[v].minb;
    if (max_ctas) max_ctas[v] = p->occ_fac[v];
  }
  *count = p->ks->n_flow_v;
  return BTC_OK;
}

int btc_plan_tuning(btc_plan_t p, int *resident_cap, int *ctas_per_sm, int *tuned) {
  if (!p) return fail(BTC_ERR_ARG, "btc_plan_tuning: NULL plan");
  if (resident_cap) *resident_cap = p->ks->flow_v[p->flow_var].minb;
  if (ctas_per_sm) *ctas_per_sm = p->ctas_per_sm;
  if (tuned) *tuned = p->tuned[p->variant == BTC_VARIANT_RIGHT_LOOKING ? 1 : 0] ? 1 : 0;
  return BTC_OK;
}

int btc_plan_tuning_interlaced(btc_plan_t p, int *resident_cap, int *ctas_per_sm, int *tuned) {
  if (!p) return fail(BTC_ERR_ARG, "btc_plan_tuning_interlaced: NULL plan");
  if (resident_cap) *resident_cap = p->ks->flow_v[p->inter_var].minb;
  if (ctas_per_sm) *ctas_per_sm = p->inter_ctas;
  if (tuned) *tuned = p->tuned[2] ? 1 : 0;
  return BTC_OK;
}

int btc_plan_set_graphs(btc_plan_t p, int enable) {
  if (!p) return fail(BTC_ERR_ARG, "btc_plan_set_graphs: NULL plan");
  p->graphs = enable != 0;
  if (p->gexec) {
    cudaGraphExecDestroy(p->gexec);
    p->gexec = nullptr;
  }
  return BTC_OK;
}

int btc_plan_set_timing(btc_plan_t p, int enable) {
  if (!p) return fail(BTC_ERR_ARG, "btc_plan_set_timing: NULL plan");
  double ms[BTC_TIMING_CLASSES];
  int n[BTC_TIMING_CLASSES];
  int rc = btc_plan_timing(p, ms, n);  // drop what is pending
  p->timing = enable != 0;
  return rc;
}

int btc_plan_timing(btc_plan_t p, double *ms, int *launches) {
  if (!p || !ms || !launches) return fail(BTC_ERR_ARG, "btc_plan_timing: NULL argument");
  cudaError_t e = cudaStreamSynchronize(p->stream);
  for (int c = 0; c < BTC_TIMING_CLASSES; ++c) {
    ms[c] = 0.0;
    launches[c] = 0;
    for (auto &ev : p->timing_pending[c]) {
      float t = 0.0f;
      if (e == cudaSuccess) e = cudaEventElapsedTime(&t, ev.first, ev.second);
      ms[c] += t;
      ++launches[c];
      cudaEventDestroy(ev.first);
      cudaEventDestroy(ev.second);
    }
    p->timing_pending[c].clear();
  }
  if (e != cudaSuccess) return fail(BTC_ERR_CUDA, "btc_plan_timing: %s", cudaGetErrorString(e));
  return BTC_OK;
}

int btc_free(btc_plan_t p) {
  if (!p) return BTC_OK;
  if (p->stream || p->dpool) cudaStreamSynchronize(p->stream);
  for (auto &v : p->timing_pending)
    for (auto &ev : v) {
      cudaEventDestroy(ev.first);
      cudaEventDestroy(ev.second);
    }
  if (p->gexec) cudaGraphExecDestroy(p->gexec);
  if (p->gstream) {
    cudaStreamSynchronize(p->gstream);
    cudaStreamDestroy(p->gstream);
    cudaStreamDestroy(p->gstream2);
    cudaEventDestroy(p->gevent);
  }

  void *dev[] = {p->dpool,        p->epool,        p->d_fac,    p->d_fwd,  p->d_bwd,     p->d_rb,
                 p->d_y,          p->s_D,          p->d_fac_deps, p->d_solve_flow, p->d_flow, p->s_B,
                 p->s_b,          p->s_x,          p->d_fac_deps_rl, p->d_inter_code, p->d_inter_deps, p->d_tail,
                 p->kry,          p->d_tiles,      p->d_tile_cnt, p->d_orient, p->d_waves};
  for (void *q : dev)
    if (q) cudaFree(q);
  if (p->h_rb) cudaFreeHost(p->h_rb);
  delete p;
  return BTC_OK;
}

}  // extern "C"
