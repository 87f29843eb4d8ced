// Level-elimination kernel: one CTA per eliminated node of one dissection
// level (Alg. 5, one iteration of its parallel loop). The whole elimination of
// node e is fused in one CTA, its blocks staged in shared memory:
//   S_e      -= P_a^T P_a                          deferred syrk (level > 1)
//   S_e       = U_e^T U_e                          potrf (blocked, upper form)
//   U(e,e-s)  = U_e^{-T} S(e,e-s)                  trsm (up)
//   U(e,e+s)  = U_e^{-T} S(e,e+s)                  trsm (down)
//   S_{e+s}  -= P_b^T P_b + U(e,e+s)^T U(e,e+s)    deferred + immediate syrk
//   S'(e-s,e+s) or S'(e+s,e-s) = -U^T U            fill gemm for level l+1
// Level 1 reads the caller's D and B directly (with conversion and padding),
// so no separate packing pass is needed.
//
// Pool contents: a diagonal slot holds the symmetric Schur complement S (upper
// triangle valid) until its node is eliminated, then the upper factor U_e
// (zeros below the diagonal). Off-diagonal slots: see btc_internal.h.
#pragma once
#include "btc_internal.h"
#include "btc_runtime.h"
#include "btc_tile.cuh"

namespace btc {

struct InstDesc {
  const void *D;  // user D [N][n][n] (source type)
  const void *B;  // user B [N-1][n][n]
  int N, n;
  // optional: device copies that the level-1 loads fill with what they read (the lower triangles of
  // D, all of B), when D and B are host memory read over the CPU-GPU link
  void *Dm = nullptr;
  void *Bm = nullptr;
};

struct FactorArgs {
  const FactorItem *items;
  int count;
  void *dpool;
  void *epool;
  const InstDesc *inst;      // per-instance descriptors (batched); NULL: use the by-value one
  unsigned long long *info;  // one word per instance
  int *status = nullptr;     // launch status word (a bounded wait that gives up sets kFlowTimeout)
  unsigned long long *phase = nullptr;  // optional per-node phase stamps (phase_stamp), or null
};

// Dataflow control of a factor item inside a persistent launch (null elsewhere): the kernel has
// waited for the factor blocks of every dependency; factor_node applies the deferred products
// (which read only those blocks), then waits for the dependencies that must be complete (the
// diagonal block and the fill blocks it reads), and publishes its own factor blocks as soon as
// they are stored, before its trailing products.
struct FlowCtl {
  const FlowSync *fs;
  const int32_t *deps;
  int ndeps;
  int t;
  int *s_ok;
};

// Optional phase stamps of one node e (8 words per node): the global timer
// (ns) at entry (0), when its operands and deferred updates are in place (1),
// after the Cholesky and its two triangular solves (2), after U_e, U(e,e-s),
// U(e,e+s) are stored (3), after the update of the next diagonal block (4)
// and at the end, after the fill block (5); word 6 = SM id. Each stamp
// follows a CTA barrier; ph is uniform across the CTA.
__device__ __forceinline__ void phase_stamp(unsigned long long *ph, int e, int k) {
  if (!ph) return;
  __syncthreads();
  if (threadIdx.x == 0) {
    ph[(size_t)e * 8 + k] = global_ns();
    if (k == 0) ph[(size_t)e * 8 + 6] = sm_id();
  }
}

template <typename T, int NP, int R>
constexpr size_t factor_smem_bytes() {
  using C = TileCfg<T, NP, R>;
  return sizeof(T) * (3 * (size_t)C::BLK + NP);
}

// T: arithmetic type; P: element type of the pools; S: element type of the
// caller's D and B (read at level 1 only). The double-FP32 top-separator Cholesky of
// the mixed-precision path is the instantiation T = double, P = float.
//
// Three shared-memory blocks: sS holds S_e -> U_e; sA and sB first hold the
// deferred blocks P_a, P_b (both deferred updates are applied before the
// Cholesky, the one onto S_{e+s} in registers), then receive S(e,e-s) and
// S(e,e+s) by asynchronous copies that overlap the Cholesky, and finally hold
// U(e,e-s), U(e,e+s) for the syrk and the fill.
// Atomic a -= X^T Y into a pool block (Alg. 6: two nodes of one level may
// update the same diagonal block; floating-point atomics, contention <= 2).
template <class C, typename T, typename P>
__device__ __forceinline__ void tile_atomic_sub_xty(P *g, const T *X, const T *Y, int r0, int c0) {
  T a[C::R][C::R];
  tile_zero<C>(a);
  tile_sub_xty<C, C::NP>(a, X, Y, r0, c0);
#pragma unroll
  for (int r = 0; r < C::R; ++r)
#pragma unroll
    for (int c = 0; c < C::R; ++c) atomicAdd(g + (size_t)(r0 + r) * C::NP + c0 + c, (P)a[r][c]);
}

// RL = true: the fully right-looking form of Alg. 6 — no deferred updates;
// after its trsm the node subtracts U(e,e-s)^T U(e,e-s) from Dhat_{e-s} and
// U(e,e+s)^T U(e,e+s) from Dhat_{e+s} with atomics. Every level reads the
// pools, which a packing pass has initialized (FIRST must be false).
// Returns false when a bounded wait of fc gave up (the node is then abandoned; the caller publishes it).
template <typename T, typename P, typename S, int NP, int R, bool FIRST, bool RL = false>
__device__ __forceinline__ bool factor_node(const FactorItem &it, const FactorArgs &args, const InstDesc &single,
                                            unsigned char *smem_raw, const FlowCtl *fc = nullptr) {
  static_assert(!(FIRST && RL), "the right-looking form reads packed pools at every level");
  using C = TileCfg<T, NP, R>;
  T *sS = reinterpret_cast<T *>(smem_raw);  // S_e -> U_e
  T *sA = sS + C::BLK;                      // P_a, then S(e,e-s) -> U(e,e-s)
  T *sB = sA + C::BLK;                      // P_b, then S(e,e+s) -> U(e,e+s)
  T *dinv = sB + C::BLK;                    // 1 / U_kk

  P *dpool = reinterpret_cast<P *>(args.dpool);
  P *epool = reinterpret_cast<P *>(args.epool);
  const int tid = threadIdx.x;
  const int ty = tid / C::TXN, tx = tid % C::TXN;
  const int r0 = ty * R, c0 = tx * R;
  const bool upper_tile = c0 >= r0;
  unsigned long long *info = args.info + it.inst;
  const InstDesc ins = args.inst ? args.inst[it.inst] : single;
  const int e = it.node;
  const S *uD = reinterpret_cast<const S *>(ins.D);
  const S *uB = reinterpret_cast<const S *>(ins.B);
  const size_t ubs = (size_t)ins.n * ins.n;
  const bool has_up = it.r_up >= 0, has_dn = it.r_down >= 0, has_next = it.d_next >= 0;
  constexpr bool ASYNC = sizeof(T) == sizeof(P);
  T d[R][R];  // the tile of S_{e+s} owned by this thread (upper tiles only)
  phase_stamp(args.phase, e, 0);

  if constexpr (FIRST) {
    // level 1: the caller's blocks, converted and padded on the way in (of D_e only its lower
    // triangle, the upper triangle of S)
    S *mD = reinterpret_cast<S *>(ins.Dm), *mB = reinterpret_cast<S *>(ins.Bm);
    user_to_smem<C>(sS, uD + e * ubs, ins.n, true, T(1), true, mD ? mD + e * ubs : nullptr);  // S[i][j] = D_e[j][i]
    if (has_up)  // S(e, e-1) = B_{e-1}
      user_to_smem<C>(sA, uB + (e - 1) * ubs, ins.n, false, T(0), false, mB ? mB + (e - 1) * ubs : nullptr);
    if (has_dn)  // S(e, e+1) = B_e^T
      user_to_smem<C>(sB, uB + e * ubs, ins.n, true, T(0), false, mB ? mB + e * ubs : nullptr);
    if (has_next && upper_tile)
      tile_from_user<C>(d, uD + (e + 1) * ubs, ins.n, r0, c0, true, T(1), mD ? mD + (e + 1) * ubs : nullptr);
    __syncthreads();
  } else if constexpr (RL) {
    if constexpr (ASYNC) {
      block_to_smem_async<C>(sS, dpool + it.d_self);
      cp_async_commit_wait_all();
    } else {
      block_to_smem<C>(sS, dpool + it.d_self);
    }
    __syncthreads();
    // the off-diagonal operands arrive while the Cholesky runs
    if constexpr (ASYNC) {
      if (has_up) block_to_smem_async<C>(sA, epool + it.r_up);
      if (has_dn) block_to_smem_async<C>(sB, epool + it.r_down);
    } else {
      if (has_up) block_to_smem<C>(sA, epool + it.r_up);
      if (has_dn) block_to_smem<C>(sB, epool + it.r_down);
    }
  } else {
    // deferred updates of level l-1, -P_a^T P_a for S_e and -P_b^T P_b for S_{e+s}: they read only the
    // factor blocks of the previous level, so they run before the diagonal blocks are complete
    const bool pa = it.p_a >= 0, pb = it.p_b >= 0;
    if constexpr (ASYNC) {
      if (pa) block_to_smem_async<C>(sA, epool + it.p_a);
      if (pb) block_to_smem_async<C>(sB, epool + it.p_b);
      cp_async_commit_wait_all();
    } else {
      if (pa) block_to_smem<C>(sA, epool + it.p_a);
      if (pb) block_to_smem<C>(sB, epool + it.p_b);
    }
    __syncthreads();
    T acc[R][R];
    tile_zero<C>(acc);
    tile_zero<C>(d);
    if (upper_tile) {
      if (pa) tile_sub_xty<C, NP>(acc, sA, sA, r0, c0);
      if (pb && has_next) tile_sub_xty<C, NP>(d, sB, sB, r0, c0);
    }
    // then the blocks that must be complete: S_e and S_{e+s} (the fill blocks follow below)
    if (fc) {
      if (!flow_wait(*fc->fs, fc->deps, fc->ndeps, fc->s_ok, kWaitFullOnly)) return false;
    } else {
      __syncthreads();
    }
    if constexpr (ASYNC) {
      block_to_smem_async<C>(sS, dpool + it.d_self);
    }
    if (has_next && upper_tile) {
      T dn[R][R];
      tile_from_pool<C>(dn, dpool + it.d_next, r0, c0);
#pragma unroll
      for (int r = 0; r < R; ++r)
#pragma unroll
        for (int c = 0; c < R; ++c) d[r][c] = dn[r][c] + d[r][c];
    }
    if constexpr (ASYNC) {
      cp_async_commit_wait_all();
    } else {
      block_to_smem<C>(sS, dpool + it.d_self);
    }
    __syncthreads();
    if (pa && upper_tile) {
      T a[R][R];
      tile_from_smem<C>(a, sS, r0, c0);
#pragma unroll
      for (int r = 0; r < R; ++r)
#pragma unroll
        for (int c = 0; c < R; ++c) a[r][c] = a[r][c] + acc[r][c];
      tile_to_smem<C>(sS, a, r0, c0);
    }
    __syncthreads();
    // the off-diagonal operands arrive while the Cholesky runs
    if constexpr (ASYNC) {
      if (has_up) block_to_smem_async<C>(sA, epool + it.r_up);
      if (has_dn) block_to_smem_async<C>(sB, epool + it.r_down);
    } else {
      if (has_up) block_to_smem<C>(sA, epool + it.r_up);
      if (has_dn) block_to_smem<C>(sB, epool + it.r_down);
    }
  }

  phase_stamp(args.phase, e, 1);
  // ---- potrf with the two trsm of the same node, pipelined by panels
  block_potrf_trsm<C>(sS, dinv, has_up ? sA : nullptr, has_dn ? sB : nullptr, info, e, [] {
    if constexpr (!FIRST && ASYNC) cp_async_commit_wait_all();
  });
  phase_stamp(args.phase, e, 2);
  smem_to_block<C>(dpool + it.d_self, sS, true);
  if (has_up) smem_to_block<C>(epool + it.r_up, sA, false);
  if (has_dn) smem_to_block<C>(epool + it.r_down, sB, false);
  if (fc) flow_publish_core(*fc->fs, fc->t);  // the factor blocks are in the pools

  phase_stamp(args.phase, e, 3);
  // ---- S_{e+s} -= U_dn^T U_dn (and, right-looking, S_{e-s} -= U_up^T U_up)
  if constexpr (RL) {
    if (upper_tile) {
      if (has_next) tile_atomic_sub_xty<C>(dpool + it.d_next, sB, sB, r0, c0);
      if (it.d_prev >= 0) tile_atomic_sub_xty<C>(dpool + it.d_prev, sA, sA, r0, c0);
    }
  } else if (has_next && upper_tile) {
    tile_sub_xty<C, NP>(d, sB, sB, r0, c0);
    tile_to_pool<C>(dpool + it.d_next, d, r0, c0);
  }
  phase_stamp(args.phase, e, 4);
  // ---- fill block for level l+1
  if (it.fill >= 0) {
    T f[R][R];
    tile_zero<C>(f);
    if (it.flags & FI_FILL_UPFIRST) tile_sub_xty<C, NP>(f, sA, sB, r0, c0);  // S'(e-s, e+s) = -U_up^T U_dn
    else tile_sub_xty<C, NP>(f, sB, sA, r0, c0);                             // S'(e+s, e-s) = -U_dn^T U_up
    tile_to_pool<C>(epool + it.fill, f, r0, c0);
  }
  phase_stamp(args.phase, e, 5);
  return true;
}

// One launch per dissection level: CTA b eliminates item b of the level.
template <typename T, typename P, typename S, int NP, int R, bool FIRST, bool RL = false>
__global__ void __launch_bounds__(TileCfg<T, NP, R>::NT) k_factor_level(FactorArgs args, InstDesc single) {
  grid_dep_enter();
  extern __shared__ __align__(16) unsigned char smem_raw[];
  const FactorItem it = args.items[blockIdx.x];
  factor_node<T, P, S, NP, R, FIRST, RL>(it, args, single, smem_raw);
}

// Persistent dataflow form: all levels in one launch. CTAs claim items in
// level order and wait only for the (<= 3) items of the previous level that
// produce their inputs (deps, 3 per item). The first `nfirst` items are
// level 1 and read the caller's arrays. MINB: resident CTAs per SM the
// register budget is set for (one compiled variant per value).
template <typename T, int NP, int R>
struct FlowFit {  // resident CTAs per SM that shared memory and threads allow
  static constexpr size_t smem = factor_smem_bytes<T, NP, R>();
  static constexpr int by_smem = (int)((226 * 1024) / smem);
  static constexpr int by_threads = 2048 / TileCfg<T, NP, R>::NT;
  static constexpr int value = by_smem < by_threads ? (by_smem < 1 ? 1 : by_smem) : by_threads;
};

template <typename T, typename P, typename S, int NP, int R, int MINB>
__global__ void __launch_bounds__(TileCfg<T, NP, R>::NT, MINB)
    k_factor_flow(FactorArgs args, InstDesc single, const int32_t *deps, int nfirst, FlowSync fs) {
  grid_dep_enter();
  extern __shared__ __align__(16) unsigned char smem_raw[];
  __shared__ int s_slot, s_ok;
  for (;;) {
    const int t = flow_claim(fs, args.count, &s_slot);
    if (t < 0) break;
    const FactorItem it = args.items[t];
    flow_trace(fs, t, 0);
    // first the factor blocks of every dependency; factor_node waits for the rest itself
    if (flow_wait(fs, deps + 3 * t, 3, &s_ok, kWaitCoreOnly)) {
      flow_trace(fs, t, 1);
      const FlowCtl fc{&fs, deps + 3 * t, 3, t, &s_ok};
      if (t < nfirst) factor_node<T, P, S, NP, R, true>(it, args, single, smem_raw, &fc);
      else factor_node<T, P, S, NP, R, false>(it, args, single, smem_raw, &fc);
    }
    __syncthreads();
    flow_trace(fs, t, 2);
    flow_publish(fs, t);
  }
}

// Persistent dataflow form of Alg. 6 (right-looking, atomics): every level
// reads the packed pools; each item waits for the two nodes of the previous
// level that last update its diagonal block and write its two fill blocks.
template <typename T, typename P, typename S, int NP, int R, int MINB>
__global__ void __launch_bounds__(TileCfg<T, NP, R>::NT, MINB)
    k_factor_flow_rl(FactorArgs args, InstDesc single, const int32_t *deps, int nfirst, FlowSync fs) {
  grid_dep_enter();
  extern __shared__ __align__(16) unsigned char smem_raw[];
  __shared__ int s_slot, s_ok;
  (void)nfirst;
  for (;;) {
    const int t = flow_claim(fs, args.count, &s_slot);
    if (t < 0) break;
    const FactorItem it = args.items[t];
    if (flow_wait(fs, deps + 3 * t, 3, &s_ok)) factor_node<T, P, S, NP, R, false, true>(it, args, single, smem_raw);
    flow_publish(fs, t);
  }
}

// ------------------------------------------ double-FP32 top-separator Cholesky
// Double-FP32 numbers: unevaluated pairs hi + lo of FP32 values with
// |lo| <= ulp(hi) / 2 (about 48 significant bits), built from the error-free
// transformations of the double-double literature (Knuth's two-sum, the
// FMA-based exact product; Hida, Li and Bailey 2001). The rounded intrinsics
// keep the compiler from contracting the steps into FMAs, which would break
// their exactness.
struct F2 {
  float hi, lo;
};
__device__ __forceinline__ F2 f2_fast_two_sum(float a, float b) {  // |a| >= |b|
  const float s = __fadd_rn(a, b);
  return {s, __fsub_rn(b, __fsub_rn(s, a))};
}
__device__ __forceinline__ F2 f2_two_sum(float a, float b) {
  const float s = __fadd_rn(a, b), bb = __fsub_rn(s, a);
  return {s, __fadd_rn(__fsub_rn(a, __fsub_rn(s, bb)), __fsub_rn(b, bb))};
}
// u * v; the lo * lo term is below the format's precision
__device__ __forceinline__ F2 f2_mul(F2 u, F2 v) {
  const float p = __fmul_rn(u.hi, v.hi);
  float e = fmaf(u.hi, v.hi, -p);  // exact error of p
  e = fmaf(u.hi, v.lo, e);
  e = fmaf(u.lo, v.hi, e);
  return f2_fast_two_sum(p, e);
}
// a - u * v
__device__ __forceinline__ F2 f2_sub_mul(F2 a, F2 u, F2 v) {
  const float p = __fmul_rn(u.hi, v.hi);
  float e = fmaf(u.hi, v.hi, -p);
  e = fmaf(u.hi, v.lo, e);
  e = fmaf(u.lo, v.hi, e);
  const F2 t = f2_two_sum(a.hi, -p);
  return f2_fast_two_sum(t.hi, __fadd_rn(t.lo, __fsub_rn(a.lo, e)));
}
// 1 / sqrt(d), d > 0: the FP32 estimate x and one Newton step x + x (1 - d x^2) / 2, with 1 - d x^2
// formed from the exact square of x and the double-FP32 product (the difference from 1 is exact there)
__device__ __forceinline__ F2 f2_rsqrt(F2 d) {
  const float x = rsqrtf(d.hi);
  const float x2 = __fmul_rn(x, x);
  const F2 dx2 = f2_mul(d, F2{x2, fmaf(x, x, -x2)});
  const float r = __fsub_rn(__fsub_rn(1.0f, dx2.hi), dx2.lo);
  return f2_fast_two_sum(x, __fmul_rn(x, __fmul_rn(0.5f, r)));
}

// Mixed path: the top separator's Schur complement S (FP32 pool, upper
// triangle valid) is factored in double-FP32 arithmetic by one CTA and the
// factor is rounded to the FP32 pool, so the Cholesky adds no FP32 rounding of
// its own (the pool value is the rounded double-FP32 result, as an FP64
// factorization rounded to FP32 would give up to ties). The deferred update
// S -= P_a^T P_a (Alg. 5, level L-1 block) is applied first in FP32 register
// tiles, like every other Schur update of this path. Everything runs on the
// FP32 pipe: the FP64 pipe of this GPU issues two lanes per clock per SM and
// its square root is a software sequence, which made an FP64 form of this
// kernel (same structure) about four times slower.
//
// The factorization is the unblocked right-looking form over a dense list of
// the upper-triangle elements (no masked lanes): at step k every element
// (i, j) with k+2 <= i <= j is updated, S_ij -= U_ki U_kj, by the threads of
// warps 1.., in list order (row-major, so the elements still active form a
// suffix); warp 0 meanwhile updates row k+1 and factors it (pivot, 1/sqrt,
// row scaling), so that one barrier per column suffices.
template <int NP>
struct RootCfg {
  static constexpr int LD = NP + 1;                // leading dimension of the (hi, lo) array
  static constexpr int NE = NP * (NP + 1) / 2;     // upper-triangle elements
  __host__ __device__ static constexpr int row_off(int i) { return i * NP - i * (i - 1) / 2; }
};

template <int NP, int R>
constexpr size_t root_smem_bytes() {
  using C = TileCfg<float, NP, R>;
  constexpr size_t f2 = 2 * sizeof(float) * ((size_t)NP * RootCfg<NP>::LD + NP);
  constexpr size_t tab = sizeof(unsigned short) * (size_t)RootCfg<NP>::NE;
  constexpr size_t stage = sizeof(float) * (size_t)C::BLK;  // P_a, before the element list is built
  return f2 + (tab > stage ? tab : stage);
}

template <typename P, typename S, int NP, int R, bool FIRST, bool RL>
__global__ void __launch_bounds__(TileCfg<float, NP, R>::NT) k_root_chol(FactorArgs args, InstDesc single) {
  grid_dep_enter();
  static_assert(sizeof(P) == 4, "the double-FP32 top-separator kernel serves FP32 pools");
  using C = TileCfg<float, NP, R>;
  using RC = RootCfg<NP>;
  constexpr int NT = C::NT, LD = RC::LD, NE = RC::NE;
  static_assert(NT >= 64, "a full look-ahead warp and at least one update warp");
  extern __shared__ __align__(16) unsigned char smem_raw[];
  float2 *S2 = reinterpret_cast<float2 *>(smem_raw);  // NP x LD (hi, lo) pairs, upper triangle used
  float2 *dinv = S2 + NP * LD;                         // 1 / U_kk
  unsigned short *tab = reinterpret_cast<unsigned short *>(dinv + NP);  // element list (i | j << 7)
  float *sA = reinterpret_cast<float *>(dinv + NP);                      // P_a (aliases the list)
  auto ld = [&](int q) {
    const float2 v = S2[q];
    return F2{v.x, v.y};
  };
  auto st = [&](int q, F2 v) { S2[q] = make_float2(v.hi, v.lo); };

  const FactorItem it = args.items[blockIdx.x];
  P *dpool = reinterpret_cast<P *>(args.dpool);
  const P *epool = reinterpret_cast<const P *>(args.epool);
  const InstDesc ins = args.inst ? args.inst[it.inst] : single;
  unsigned long long *info = args.info + it.inst;
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;

  // ---- S in double-FP32
  if constexpr (FIRST) {  // a single-node problem: the caller's D_1 (lower triangle valid)
    const S *uD = reinterpret_cast<const S *>(ins.D) + (size_t)it.node * ins.n * ins.n;
    for (int q = tid; q < NP * NP; q += NT) {
      const int i = q / NP, j = q % NP;
      if (i > j) continue;
      if (j < ins.n) {
        const S v = uD[(size_t)j * ins.n + i];
        const float h = convert_in<float, S>(v);
        float l = 0.0f;
        if constexpr (sizeof(S) == 8) l = f64_to_f32_rn(v - f32_to_f64(h));
        st(i * LD + j, F2{h, l});
      } else {
        st(i * LD + j, F2{i == j ? 1.0f : 0.0f, 0.0f});
      }
    }
  } else if (!RL && it.p_a >= 0) {
    block_to_smem_async<C>(sA, epool + it.p_a);
    const int r0 = (tid / C::TXN) * R, c0 = (tid % C::TXN) * R;
    float a[R][R];
    if (c0 >= r0) tile_from_pool<C>(a, dpool + it.d_self, r0, c0);
    cp_async_commit_wait_all();
    __syncthreads();
    if (c0 >= r0) {
      tile_sub_xty<C, NP>(a, sA, sA, r0, c0);
#pragma unroll
      for (int r = 0; r < R; ++r)
#pragma unroll
        for (int c = 0; c < R; ++c) st((r0 + r) * LD + c0 + c, F2{a[r][c], 0.0f});
    }
  } else {
    const P *g = dpool + it.d_self;
    for (int q = tid; q < NP * NP; q += NT) {
      const int i = q / NP, j = q % NP;
      if (i <= j) st(i * LD + j, F2{__ldcg(g + q), 0.0f});
    }
  }
  __syncthreads();  // sA is dead from here on
  for (int q = tid; q < NP * NP; q += NT) {
    const int i = q / NP, j = q % NP;
    if (i <= j) tab[RC::row_off(i) + j - i] = (unsigned short)(i | (j << 7));
  }

  // pivot of row r (already updated by every earlier row): U_rr = sqrt(d), row r scaled by 1/sqrt(d)
  auto factor_row = [&](int r) {
    F2 d = ld(r * LD + r);
    if (!(d.hi > 0.0f)) {
      if (lane == 0 && info) atomicMin(info, pack_info(it.node, r));
      d = F2{1.0f, 0.0f};
    }
    const F2 rs = f2_rsqrt(d);
    __syncwarp();
    for (int j = r + 1 + lane; j < NP; j += 32) st(r * LD + j, f2_mul(ld(r * LD + j), rs));
    if (lane == 0) {
      st(r * LD + r, f2_mul(d, rs));
      dinv[r] = make_float2(rs.hi, rs.lo);
    }
  };

  // ---- row 0
  if (warp == 0) factor_row(0);
  __syncthreads();

  // ---- steps k = 0 .. NP-2: row k is final at the start of step k
#pragma unroll 1
  for (int k = 0; k + 1 < NP; ++k) {
    const int uk = k * LD;
    if (warp == 0) {
      const int r1 = (k + 1) * LD;
      const F2 ukk1 = ld(uk + k + 1);
      for (int j = k + 1 + lane; j < NP; j += 32) st(r1 + j, f2_sub_mul(ld(r1 + j), ukk1, ld(uk + j)));
      __syncwarp();
      factor_row(k + 1);
    } else {
      const int base = RC::row_off(k + 2);
#pragma unroll 4
      for (int q = base + tid - 32; q < NE; q += NT - 32) {
        const unsigned e = tab[q];
        const int i = e & 127, j = e >> 7;
        st(i * LD + j, f2_sub_mul(ld(i * LD + j), ld(uk + i), ld(uk + j)));
      }
    }
    __syncthreads();
  }

  // ---- U (zeros below the diagonal) -> FP32 pool
  P *g = dpool + it.d_self;
  for (int q = tid; q < NP * NP; q += NT) {
    const int i = q / NP, j = q % NP;
    const float2 v = S2[i * LD + j];
    g[q] = i <= j ? __fadd_rn(v.x, v.y) : P(0);
  }
}

// The same top-separator factorization in FP64 (btc_plan_set_root_precision):
// S from the FP32 pool (or the caller's FP64 block when the problem is one
// node) in FP64 shared memory, the same dense-list right-looking Cholesky with
// a look-ahead warp, FP64 square roots, the result rounded to the FP32 pool.
// On this GPU the FP64 pipe issues two lanes per clock per SM and a masked
// lane costs as much as an active one, which is why the list form avoids
// single-warp panels and tile masks here too.
template <typename P, typename S, int NP, int R, bool FIRST, bool RL>
__global__ void __launch_bounds__(TileCfg<float, NP, R>::NT) k_root_chol_f64(FactorArgs args, InstDesc single) {
  grid_dep_enter();
  static_assert(sizeof(P) == 4, "the FP64 top-separator kernel serves FP32 pools");
  using C = TileCfg<float, NP, R>;
  using RC = RootCfg<NP>;
  constexpr int NT = C::NT, LD = RC::LD, NE = RC::NE;
  static_assert(NT >= 64, "a full look-ahead warp and at least one update warp");
  extern __shared__ __align__(16) unsigned char smem_raw[];
  double *Sd = reinterpret_cast<double *>(smem_raw);  // NP x LD, upper triangle used
  double *dinv = Sd + NP * LD;                         // 1 / U_kk
  unsigned short *tab = reinterpret_cast<unsigned short *>(dinv + NP);  // element list (i | j << 7)
  float *sA = reinterpret_cast<float *>(dinv + NP);                     // P_a (aliases the list)

  const FactorItem it = args.items[blockIdx.x];
  P *dpool = reinterpret_cast<P *>(args.dpool);
  const P *epool = reinterpret_cast<const P *>(args.epool);
  const InstDesc ins = args.inst ? args.inst[it.inst] : single;
  unsigned long long *info = args.info + it.inst;
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;

  // ---- S in FP64
  if constexpr (FIRST) {  // a single-node problem: the caller's D_1 (lower triangle valid)
    const S *uD = reinterpret_cast<const S *>(ins.D) + (size_t)it.node * ins.n * ins.n;
    for (int q = tid; q < NP * NP; q += NT) {
      const int i = q / NP, j = q % NP;
      if (i > j) continue;
      Sd[i * LD + j] = (j < ins.n) ? (double)uD[(size_t)j * ins.n + i] : (i == j ? 1.0 : 0.0);
    }
  } else if (!RL && it.p_a >= 0) {
    block_to_smem_async<C>(sA, epool + it.p_a);
    const int r0 = (tid / C::TXN) * R, c0 = (tid % C::TXN) * R;
    float a[R][R];
    if (c0 >= r0) tile_from_pool<C>(a, dpool + it.d_self, r0, c0);
    cp_async_commit_wait_all();
    __syncthreads();
    if (c0 >= r0) {
      tile_sub_xty<C, NP>(a, sA, sA, r0, c0);
#pragma unroll
      for (int r = 0; r < R; ++r)
#pragma unroll
        for (int c = 0; c < R; ++c) Sd[(r0 + r) * LD + c0 + c] = f32_to_f64(a[r][c]);
    }
  } else {
    const P *g = dpool + it.d_self;
    for (int q = tid; q < NP * NP; q += NT) {
      const int i = q / NP, j = q % NP;
      if (i <= j) Sd[i * LD + j] = f32_to_f64(__ldcg(g + q));
    }
  }
  __syncthreads();  // sA is dead from here on
  for (int q = tid; q < NP * NP; q += NT) {
    const int i = q / NP, j = q % NP;
    if (i <= j) tab[RC::row_off(i) + j - i] = (unsigned short)(i | (j << 7));
  }

  // ---- row 0
  if (warp == 0) {
    double d = Sd[0];
    if (!(d > 0.0)) {
      if (lane == 0 && info) atomicMin(info, pack_info(it.node, 0));
      d = 1.0;
    }
    const double rs = rsqrt(d);
    __syncwarp();
    for (int j = 1 + lane; j < NP; j += 32) Sd[j] *= rs;
    if (lane == 0) {
      Sd[0] = d * rs;
      dinv[0] = rs;
    }
  }
  __syncthreads();

  // ---- steps k = 0 .. NP-2: row k is final at the start of step k
#pragma unroll 1
  for (int k = 0; k + 1 < NP; ++k) {
    const double *Uk = Sd + k * LD;
    if (warp == 0) {
      double *row = Sd + (k + 1) * LD;
      const double ukk1 = Uk[k + 1];
      for (int j = k + 1 + lane; j < NP; j += 32) row[j] = fma(-ukk1, Uk[j], row[j]);
      __syncwarp();
      double d = row[k + 1];
      if (!(d > 0.0)) {
        if (lane == 0 && info) atomicMin(info, pack_info(it.node, k + 1));
        d = 1.0;
      }
      const double rs = rsqrt(d);
      __syncwarp();
      for (int j = k + 2 + lane; j < NP; j += 32) row[j] *= rs;
      if (lane == 0) {
        row[k + 1] = d * rs;
        dinv[k + 1] = rs;
      }
    } else {
      const int base = RC::row_off(k + 2);
#pragma unroll 4
      for (int q = base + tid - 32; q < NE; q += NT - 32) {
        const unsigned e = tab[q];
        const int i = e & 127, j = e >> 7;
        Sd[i * LD + j] = fma(-Uk[i], Uk[j], Sd[i * LD + j]);
      }
    }
    __syncthreads();
  }

  // ---- U (zeros below the diagonal) -> FP32 pool
  P *g = dpool + it.d_self;
  for (int q = tid; q < NP * NP; q += NT) {
    const int i = q / NP, j = q % NP;
    g[q] = i <= j ? f64_to_f32_rn(Sd[i * LD + j]) : P(0);
  }
}

// Packing pass of Alg. 6 (its first parallel loop) and of the partition
// orders: Dhat_v <- D_v for every node (upper-form copy of the caller's lower
// triangle, identity padding) and the slot of B_v (coupling nodes v, v+1) in
// the orientation of the node eliminated first: with `transposed` null, the
// nested-dissection level 1 (slot k, 1-based, holds S(k, k+1) = B_k^T when k
// is odd, else S(k+1, k) = B_k); otherwise B_v^T where transposed[v] != 0,
// else B_v. One CTA per node.
template <typename P, typename S, int NP>
__global__ void k_pack_matrix(P *dpool, P *epool, const S *D, const S *B, int N, int n,
                              const int8_t *transposed) {
  grid_dep_enter();
  const int v = blockIdx.x;  // 0-based node
  const size_t ubs = (size_t)n * n, bs = (size_t)NP * NP;
  for (int q = threadIdx.x; q < NP * NP; q += blockDim.x) {
    const int i = q / NP, j = q % NP;
    P val;
    if (i < n && j < n) val = convert_in<P, S>(i <= j ? D[v * ubs + (size_t)j * n + i] : D[v * ubs + (size_t)i * n + j]);
    else val = (i == j) ? P(1) : P(0);
    dpool[v * bs + q] = val;
    if (v + 1 < N) {
      const bool odd = transposed ? transposed[v] != 0 : ((v + 1) & 1) != 0;  // (ND: 1-based slot k = v + 1)
      P b;
      if (i < n && j < n) b = convert_in<P, S>(odd ? B[v * ubs + (size_t)j * n + i] : B[v * ubs + (size_t)i * n + j]);
      else b = P(0);
      epool[v * bs + q] = b;
    }
  }
}

// One node of a batched packing pass: its diagonal block goes to dpool slot
// `blockIdx.x` (the group's nodes are numbered instance by instance) and its
// coupling with the next node of its instance to epool slot `slot`, as B^T
// when `transposed` (the node is eliminated first), else as B.
struct PackNode {
  int64_t slot;
  int32_t inst, row;
  int32_t transposed, pad;
};

template <typename P, typename S, int NP>
__global__ void k_pack_batch(P *dpool, P *epool, const PackNode *nodes, const InstDesc *inst) {
  grid_dep_enter();
  const PackNode nd = nodes[blockIdx.x];
  const InstDesc in = inst[nd.inst];
  const int n = in.n;
  const size_t ubs = (size_t)n * n, bs = (size_t)NP * NP;
  const S *D = reinterpret_cast<const S *>(in.D) + nd.row * ubs;
  const S *B = reinterpret_cast<const S *>(in.B) + nd.row * ubs;
  const bool has_b = nd.row + 1 < in.N;
  for (int q = threadIdx.x; q < NP * NP; q += blockDim.x) {
    const int i = q / NP, j = q % NP;
    P val;
    if (i < n && j < n) val = convert_in<P, S>(i <= j ? D[(size_t)j * n + i] : D[(size_t)i * n + j]);
    else val = (i == j) ? P(1) : P(0);
    dpool[blockIdx.x * bs + q] = val;
    if (has_b) {
      P b;
      if (i < n && j < n) b = convert_in<P, S>(nd.transposed ? B[(size_t)j * n + i] : B[(size_t)i * n + j]);
      else b = P(0);
      epool[nd.slot * bs + q] = b;
    }
  }
}

template <typename P, typename S, int NP>
int launch_pack_batch(void *dpool, void *epool, const void *nodes, const void *inst, int count, cudaStream_t s) {
  if (count <= 0) return BTC_OK;
  k_pack_batch<P, S, NP><<<count, 256, 0, s>>>(static_cast<P *>(dpool), static_cast<P *>(epool),
                                                static_cast<const PackNode *>(nodes),
                                                static_cast<const InstDesc *>(inst));
  const cudaError_t e = cudaGetLastError();
  return e == cudaSuccess ? BTC_OK : fail(BTC_ERR_CUDA, "batched packing pass launch: %s", cudaGetErrorString(e));
}

// Typed launch of the packing pass (argument types checked at compile time).
template <typename P, typename S, int NP>
int launch_pack(void *dpool, void *epool, const void *D, const void *B, int N, int n, const int8_t *orient,
                cudaStream_t s) {
  if (N <= 0) return BTC_OK;
  k_pack_matrix<P, S, NP><<<N, 256, 0, s>>>(static_cast<P *>(dpool), static_cast<P *>(epool),
                                             static_cast<const S *>(D), static_cast<const S *>(B), N, n, orient);
  const cudaError_t e = cudaGetLastError();
  return e == cudaSuccess ? BTC_OK : fail(BTC_ERR_CUDA, "packing pass launch: %s", cudaGetErrorString(e));
}

}  // namespace btc
