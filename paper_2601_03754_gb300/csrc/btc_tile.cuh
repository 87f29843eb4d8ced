// Block operations on padded np x np blocks held in shared memory, for one
// CTA per node elimination.
//
// Thread layout for the dense products: the CTA's NT = (NP/R)^2 threads form a
// (NP/R) x (NP/R) grid; thread (ty, tx) owns the R x R register tile of rows
// [ty*R, ty*R+R) and columns [tx*R, tx*R+R). Every product of the elimination
// is written as C -= X^T Y (row reads of X and Y only), which is the
// bank-conflict-free access pattern for row-major blocks with the padded
// leading dimension LD.
//
// The Cholesky factor is kept in UPPER form, S = U^T U (U = L^T), so that the
// blocked factorization and the triangular solves are also X^T Y products:
//   panel row:      U[p, j>p] = U_pp^{-T} S[p, j]        (column-wise substitution)
//   trailing:       S[i, j]  -= U[p, i]^T U[p, j]        (X^T Y, K = panel width)
//   solve:          Z = U^{-T} R                          (same two steps on R)
#pragma once
#include <cuda_runtime.h>
#include <stdint.h>

namespace btc {

template <typename T, int NP_, int R_>
struct TileCfg {
  static constexpr int NP = NP_;
  static constexpr int R = R_;
  static constexpr int TXN = NP / R;
  static constexpr int NT = TXN * TXN;
  static constexpr int PAD = sizeof(T) == 4 ? 4 : 2;
  static constexpr int LD = NP + PAD;
  static constexpr int BLK = NP * LD;            // elements of one shared-memory block
  static constexpr int PB = NP >= 16 ? 16 : NP;  // panel width of the blocked factorization
  static constexpr int NPAN = NP / PB;
  static_assert(NP % R == 0, "tile must divide the block");
  static_assert(NP % PB == 0 && PB % R == 0, "panels must align with tiles");
};

// ---------------------------------------------------------------- vector io
template <typename T, int R>
__device__ __forceinline__ void vload(const T *p, T (&v)[R]) {
  if constexpr (sizeof(T) * R == 16) {
    const float4 q = *reinterpret_cast<const float4 *>(p);
    const T *s = reinterpret_cast<const T *>(&q);
#pragma unroll
    for (int i = 0; i < R; ++i) v[i] = s[i];
  } else if constexpr (sizeof(T) * R == 32) {
    const float4 q0 = reinterpret_cast<const float4 *>(p)[0];
    const float4 q1 = reinterpret_cast<const float4 *>(p)[1];
    const T *s0 = reinterpret_cast<const T *>(&q0);
    const T *s1 = reinterpret_cast<const T *>(&q1);
#pragma unroll
    for (int i = 0; i < R / 2; ++i) {
      v[i] = s0[i];
      v[i + R / 2] = s1[i];
    }
  } else if constexpr (sizeof(T) * R == 8) {
    const float2 q = *reinterpret_cast<const float2 *>(p);
    const T *s = reinterpret_cast<const T *>(&q);
#pragma unroll
    for (int i = 0; i < R; ++i) v[i] = s[i];
  } else {
#pragma unroll
    for (int i = 0; i < R; ++i) v[i] = p[i];
  }
}

template <typename T, int R>
__device__ __forceinline__ void vstore(T *p, const T (&v)[R]) {
  if constexpr (sizeof(T) * R == 16) {
    float4 q;
    T *s = reinterpret_cast<T *>(&q);
#pragma unroll
    for (int i = 0; i < R; ++i) s[i] = v[i];
    *reinterpret_cast<float4 *>(p) = q;
  } else if constexpr (sizeof(T) * R == 32) {
    float4 q0, q1;
    T *s0 = reinterpret_cast<T *>(&q0);
    T *s1 = reinterpret_cast<T *>(&q1);
#pragma unroll
    for (int i = 0; i < R / 2; ++i) {
      s0[i] = v[i];
      s1[i] = v[i + R / 2];
    }
    reinterpret_cast<float4 *>(p)[0] = q0;
    reinterpret_cast<float4 *>(p)[1] = q1;
  } else if constexpr (sizeof(T) * R == 8) {
    float2 q;
    T *s = reinterpret_cast<T *>(&q);
#pragma unroll
    for (int i = 0; i < R; ++i) s[i] = v[i];
    *reinterpret_cast<float2 *>(p) = q;
  } else {
#pragma unroll
    for (int i = 0; i < R; ++i) p[i] = v[i];
  }
}

// ------------------------------------------------------------ conversions
// FP64 -> FP32 with round-to-nearest-even using integer operations only: on
// this GPU the conversion instruction runs on the FP64 pipe, which is 1/64 of
// the FP32 rate. Exact (IEEE) for results in the FP32 normal range, for
// zeros, infinities and NaNs; results below the normal range fall back to the
// hardware conversion.
__device__ __forceinline__ float f64_to_f32_rn(double a) {
  const unsigned hi = (unsigned)__double2hiint(a), lo = (unsigned)__double2loint(a);
  const unsigned sign = hi & 0x80000000u;
  const int e = (int)((hi >> 20) & 0x7ffu);
  if (e == 0x7ff) return __uint_as_float(sign | 0x7f800000u | (((hi & 0xfffffu) | lo) ? 0x400000u : 0u));
  if (e == 0) return __uint_as_float(sign);  // zero / FP64 subnormal -> signed zero
  const int ef = e - 1023 + 127;
  if (ef >= 255) return __uint_as_float(sign | 0x7f800000u);
  if (ef <= 0) return (float)a;
  const unsigned mant = ((hi & 0xfffffu) << 3) | (lo >> 29);  // top 23 of the 52 fraction bits
  const unsigned rem = lo & 0x1fffffffu, half = 0x10000000u;   // the 29 dropped bits
  unsigned bits = ((unsigned)ef << 23) | mant;
  if (rem > half || (rem == half && (mant & 1u))) bits += 1u;  // a carry moves to the next binade
  return __uint_as_float(sign | bits);
}

// FP32 -> FP64 (exact) with integer operations; subnormal, infinite and NaN
// inputs use the hardware conversion.
__device__ __forceinline__ double f32_to_f64(float f) {
  const unsigned u = __float_as_uint(f);
  const unsigned long long sign = (unsigned long long)(u >> 31) << 63;
  if ((u & 0x7fffffffu) == 0) return __longlong_as_double((long long)sign);
  const unsigned e = (u >> 23) & 0xffu;
  if (e == 0 || e == 0xffu) return (double)f;
  const unsigned long long bits = sign | ((unsigned long long)(e + 896u) << 52) | ((unsigned long long)(u & 0x7fffffu) << 29);
  return __longlong_as_double((long long)bits);
}

// Element conversion between the caller's, the pools' and the arithmetic
// types (identity when they agree).
template <typename T, typename S>
__device__ __forceinline__ T convert_in(S v) {
  if constexpr (sizeof(T) == 4 && sizeof(S) == 8) return f64_to_f32_rn(v);
  else if constexpr (sizeof(T) == 8 && sizeof(S) == 4) return f32_to_f64(v);
  else return (T)v;
}

// ------------------------------------------------------------ async copies
// 16-byte global -> shared copy that bypasses registers (cp.async, L2 only).
__device__ __forceinline__ void cp_async16(void *smem, const void *gmem) {
  const unsigned s = (unsigned)__cvta_generic_to_shared(smem);
  asm volatile("cp.async.cg.shared.global [%0], [%1], 16;\n" ::"r"(s), "l"(gmem) : "memory");
}
__device__ __forceinline__ void cp_async_commit_wait_all() {
  asm volatile("cp.async.commit_group;\ncp.async.wait_all;\n" ::: "memory");
}

// ------------------------------------------------------------ block transfer
// Pool block (np x np, type T, row stride ldg) -> padded shared memory (same
// type) with cp.async; completes at cp_async_commit_wait_all() + __syncthreads().
template <class C, typename T>
__device__ __forceinline__ void block_to_smem_async(T *s, const T *g, int ldg = C::NP) {
  constexpr int V = 16 / sizeof(T);
  constexpr int CPR = C::NP / V;
  constexpr int TOTAL = C::NP * CPR;
#pragma unroll
  for (int q = threadIdx.x; q < TOTAL; q += C::NT) {
    const int row = q / CPR, col = (q % CPR) * V;
    cp_async16(s + row * C::LD + col, g + (size_t)row * ldg + col);
  }
}

// Pool block (np x np, row-major, element type P) -> padded shared memory (type T),
// cooperative 16-byte loads, all issued before any store.
template <class C, typename T, typename P>
__device__ __forceinline__ void block_to_smem(T *s, const P *g) {
  constexpr int V = 16 / sizeof(P);  // source elements per 16-byte chunk
  constexpr int CPR = C::NP / V;     // chunks per row
  constexpr int TOTAL = C::NP * CPR;
  constexpr int ITER = (TOTAL + C::NT - 1) / C::NT;
  float4 raw[ITER];
#pragma unroll
  for (int it = 0; it < ITER; ++it) {
    const int q = threadIdx.x + it * C::NT;
    if (q < TOTAL) {
      const int row = q / CPR, col = (q % CPR) * V;
      raw[it] = __ldcg(reinterpret_cast<const float4 *>(g + (size_t)row * C::NP + col));
    }
  }
#pragma unroll
  for (int it = 0; it < ITER; ++it) {
    const int q = threadIdx.x + it * C::NT;
    if (q < TOTAL) {
      const int row = q / CPR, col = (q % CPR) * V;
      const P *src = reinterpret_cast<const P *>(&raw[it]);
      if constexpr (sizeof(T) == sizeof(P)) {
        *reinterpret_cast<float4 *>(s + row * C::LD + col) = raw[it];
      } else {
#pragma unroll
        for (int i = 0; i < V; ++i) s[row * C::LD + col + i] = convert_in<T, P>(src[i]);
      }
    }
  }
}

// Padded shared memory (type T) -> pool block (type P, row stride ldg), cooperative.
// lower_zero: write zeros below the diagonal (the final U factor).
template <class C, typename T, typename P>
__device__ __forceinline__ void smem_to_block(P *g, const T *s, bool lower_zero, int ldg = C::NP) {
  constexpr int V = 16 / sizeof(P);
  constexpr int CPR = C::NP / V;
  constexpr int TOTAL = C::NP * CPR;
  for (int q = threadIdx.x; q < TOTAL; q += C::NT) {
    const int row = q / CPR, col = (q % CPR) * V;
    float4 raw;
    P *dst = reinterpret_cast<P *>(&raw);
#pragma unroll
    for (int i = 0; i < V; ++i) dst[i] = (lower_zero && col + i < row) ? P(0) : convert_in<P, T>(s[row * C::LD + col + i]);
    *reinterpret_cast<float4 *>(g + (size_t)row * ldg + col) = raw;
  }
}


// Caller's block (n x n row-major, type S) -> padded shared memory (type T).
// trans: element (i, k) of the result is src(k, i). Padding: `diag` on the
// padded diagonal, 0 elsewhere. lower: read only the source's lower triangle
// (row >= column; the rest of the result is 0). mirror (optional): every
// element read is also stored there at its source offset. Each thread issues
// a chunk of loads before converting any of them, so their latencies overlap.
template <class C, typename T, typename S>
__device__ __forceinline__ void user_to_smem(T *s, const S *src, int n, bool trans, T diag, bool lower = false,
                                             S *mirror = nullptr) {
  if constexpr (sizeof(S) == 8) {
    // FP64 rows of even length from a 16-byte aligned block: pairs of elements per 16-byte load, so a
    // thread's 32 bytes in flight take half as many load requests
    if ((n & 1) == 0 && (reinterpret_cast<uintptr_t>(src) & 15) == 0) {
      constexpr int HP = C::NP / 2;  // pairs per padded row
      constexpr int TOT2 = C::NP * HP;
      constexpr int IT2 = (TOT2 + C::NT - 1) / C::NT;
      constexpr int CH2 = IT2 < 2 ? IT2 : 2;
#pragma unroll 1
      for (int i0 = 0; i0 < IT2; i0 += CH2) {
        double2 v[CH2];
#pragma unroll
        for (int u = 0; u < CH2; ++u) {
          const int q = threadIdx.x + (i0 + u) * C::NT;
          const int a = q / HP, b = 2 * (q % HP);  // source row a, columns b, b + 1 (b + 1 < n: n is even)
          v[u] = (q < TOT2 && a < n && b < n && (!lower || a >= b))
                     ? __ldg(reinterpret_cast<const double2 *>(src + (size_t)a * n + b))
                     : make_double2(0.0, 0.0);
        }
#pragma unroll
        for (int u = 0; u < CH2; ++u) {
          const int q = threadIdx.x + (i0 + u) * C::NT;
          if (q >= TOT2) continue;
          const int a = q / HP, b0 = 2 * (q % HP);
#pragma unroll
          for (int t = 0; t < 2; ++t) {
            const int b = b0 + t;
            const bool in = a < n && b < n, use = in && (!lower || a >= b);
            const double val = t ? v[u].y : v[u].x;
            if (mirror && use) mirror[(size_t)a * n + b] = val;
            const T x = use ? convert_in<T, double>(val) : (in ? T(0) : (a == b ? diag : T(0)));
            if (trans) s[b * C::LD + a] = x;
            else s[a * C::LD + b] = x;
          }
        }
      }
      return;
    }
  }
  constexpr int TOTAL = C::NP * C::NP;
  constexpr int ITER = (TOTAL + C::NT - 1) / C::NT;
  constexpr int CHMAX = 32 / (int)sizeof(S);  // 32 bytes of loads in flight per thread
  constexpr int CH = ITER < CHMAX ? ITER : CHMAX;
#pragma unroll 1
  for (int i0 = 0; i0 < ITER; i0 += CH) {
    S v[CH];
#pragma unroll
    for (int u = 0; u < CH; ++u) {
      // consecutive threads read consecutive source elements
      const int q = threadIdx.x + (i0 + u) * C::NT;
      const int a = q / C::NP, b = q % C::NP;  // source row a, column b
      v[u] = (q < TOTAL && a < n && b < n && (!lower || a >= b)) ? __ldg(src + (size_t)a * n + b) : S(0);
    }
#pragma unroll
    for (int u = 0; u < CH; ++u) {
      const int q = threadIdx.x + (i0 + u) * C::NT;
      if (q >= TOTAL) continue;
      const int a = q / C::NP, b = q % C::NP;
      const bool in = a < n && b < n;
      if (mirror && in && (!lower || a >= b)) mirror[(size_t)a * n + b] = v[u];
      const T x = in ? convert_in<T, S>(v[u]) : (a == b ? diag : T(0));
      if (trans) s[b * C::LD + a] = x;
      else s[a * C::LD + b] = x;
    }
  }
}

// Caller's block (n x n row-major, type S) -> one register tile, padded like
// user_to_smem. trans: element (i, k) is src(k, i). mirror (optional): every
// element read is also stored there at its source offset. Each tile row's
// loads precede its conversions.
template <class C, typename T, typename S>
__device__ __forceinline__ void tile_from_user(T (&a)[C::R][C::R], const S *src, int n, int r0, int c0, bool trans,
                                               T diag, S *mirror = nullptr) {
#pragma unroll
  for (int r = 0; r < C::R; ++r) {
    S v[C::R];
    const int i = r0 + r;
#pragma unroll
    for (int c = 0; c < C::R; ++c) {
      const int k = c0 + c;
      v[c] = (i < n && k < n) ? (trans ? __ldg(src + (size_t)k * n + i) : __ldg(src + (size_t)i * n + k)) : S(0);
    }
#pragma unroll
    for (int c = 0; c < C::R; ++c) {
      const int k = c0 + c;
      if (mirror && i < n && k < n) mirror[trans ? (size_t)k * n + i : (size_t)i * n + k] = v[c];
      a[r][c] = (i < n && k < n) ? convert_in<T, S>(v[c]) : ((i == k) ? diag : T(0));
    }
  }
}

// ------------------------------------------------------------ tile algebra
template <class C, typename T>
__device__ __forceinline__ void tile_zero(T (&a)[C::R][C::R]) {
#pragma unroll
  for (int r = 0; r < C::R; ++r)
#pragma unroll
    for (int c = 0; c < C::R; ++c) a[r][c] = T(0);
}

template <class C, typename T>
__device__ __forceinline__ void tile_from_smem(T (&a)[C::R][C::R], const T *s, int r0, int c0) {
#pragma unroll
  for (int r = 0; r < C::R; ++r) vload<T, C::R>(s + (r0 + r) * C::LD + c0, a[r]);
}

template <class C, typename T>
__device__ __forceinline__ void tile_to_smem(T *s, const T (&a)[C::R][C::R], int r0, int c0) {
#pragma unroll
  for (int r = 0; r < C::R; ++r) vstore<T, C::R>(s + (r0 + r) * C::LD + c0, a[r]);
}

// Global load that bypasses L1 (pool blocks may have been written by another
// CTA of the same persistent launch).
template <typename T, int R>
__device__ __forceinline__ void vload_cg(const T *p, T (&v)[R]) {
  if constexpr (sizeof(T) * R == 16) {
    const float4 q = __ldcg(reinterpret_cast<const float4 *>(p));
    const T *s = reinterpret_cast<const T *>(&q);
#pragma unroll
    for (int i = 0; i < R; ++i) v[i] = s[i];
  } else if constexpr (sizeof(T) * R == 32) {
    const float4 q0 = __ldcg(reinterpret_cast<const float4 *>(p));
    const float4 q1 = __ldcg(reinterpret_cast<const float4 *>(p) + 1);
    const T *s0 = reinterpret_cast<const T *>(&q0);
    const T *s1 = reinterpret_cast<const T *>(&q1);
#pragma unroll
    for (int i = 0; i < R / 2; ++i) {
      v[i] = s0[i];
      v[i + R / 2] = s1[i];
    }
  } else if constexpr (sizeof(T) * R == 8) {
    const float2 q = __ldcg(reinterpret_cast<const float2 *>(p));
    const T *s = reinterpret_cast<const T *>(&q);
#pragma unroll
    for (int i = 0; i < R; ++i) v[i] = s[i];
  } else {
#pragma unroll
    for (int i = 0; i < R; ++i) v[i] = __ldcg(p + i);
  }
}

template <class C, typename T, typename P>
__device__ __forceinline__ void tile_from_pool(T (&a)[C::R][C::R], const P *g, int r0, int c0) {
#pragma unroll
  for (int r = 0; r < C::R; ++r) {
    P v[C::R];
    vload_cg<P, C::R>(g + (size_t)(r0 + r) * C::NP + c0, v);
#pragma unroll
    for (int c = 0; c < C::R; ++c) a[r][c] = convert_in<T, P>(v[c]);
  }
}

template <class C, typename T, typename P>
__device__ __forceinline__ void tile_to_pool(P *g, const T (&a)[C::R][C::R], int r0, int c0) {
#pragma unroll
  for (int r = 0; r < C::R; ++r) {
    P v[C::R];
#pragma unroll
    for (int c = 0; c < C::R; ++c) v[c] = convert_in<P, T>(a[r][c]);
    vstore<P, C::R>(g + (size_t)(r0 + r) * C::NP + c0, v);
  }
}

// a -= X^T Y over k in [k0, k0 + KLEN): a[r][c] -= sum_k X[k][r0+r] Y[k][c0+c].
template <class C, int KLEN, typename T>
__device__ __forceinline__ void tile_sub_xty(T (&a)[C::R][C::R], const T *X, const T *Y, int r0, int c0,
                                             int k0 = 0) {
#pragma unroll 4
  for (int kk = 0; kk < KLEN; ++kk) {
    const int k = k0 + kk;
    T x[C::R], y[C::R];
    vload<T, C::R>(X + k * C::LD + r0, x);
    vload<T, C::R>(Y + k * C::LD + c0, y);
#pragma unroll
    for (int r = 0; r < C::R; ++r)
#pragma unroll
      for (int c = 0; c < C::R; ++c) a[r][c] = fma(-x[r], y[c], a[r][c]);
  }
}

// ------------------------------------------------------- dataflow signalling
// Completion flags of a persistent launch: the producer CTA publishes with a
// release store after a CTA barrier; consumers poll with acquire loads. Every
// wait is bounded: after kMaxPolls polls (about a second) the CTA records
// kFlowTimeout in *status and gives up; a nonzero status makes every later
// wait give up at once, so a failed launch drains quickly.
constexpr long long kMaxPolls = 1ll << 23;
constexpr int kFlowTimeout = 1;

__device__ __forceinline__ int ld_acquire_gpu(const int *p) {
  int v;
  asm volatile("ld.acquire.gpu.global.u32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
  return v;
}
__device__ __forceinline__ void st_release_gpu(int *p, int v) {
  asm volatile("st.release.gpu.global.u32 [%0], %1;" ::"l"(p), "r"(v) : "memory");
}

struct FlowSync {
  int *ticket;                // next item to claim
  int *done;                  // one flag per item
  int *status;                // 0 = ok; kFlowTimeout when a wait gave up
  unsigned long long *trace;  // optional: 4 words per item (claim, ready, done ns; SM id), or null
  long long max_polls = kMaxPolls;  // poll limit of every wait (lowered only by the failure-detection tests)
};

__device__ __forceinline__ unsigned long long global_ns() {
  unsigned long long t;
  asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
  return t;
}
__device__ __forceinline__ unsigned sm_id() {
  unsigned s;
  asm volatile("mov.u32 %0, %%smid;" : "=r"(s));
  return s;
}

// Trace hooks (thread 0 only; no-ops when tracing is off).
__device__ __forceinline__ void flow_trace(const FlowSync &fs, int t, int slot) {
  if (fs.trace && threadIdx.x == 0) {
    fs.trace[4 * (size_t)t + slot] = global_ns();
    if (slot == 0) fs.trace[4 * (size_t)t + 3] = sm_id();
  }
}

// Claim the next item (ticket order = dependency order). Returns the item
// index, or -1 when all `total` items are taken. All threads of the CTA call it.
__device__ __forceinline__ int flow_claim(const FlowSync &fs, int total, int *s_slot) {
  __syncthreads();  // the previous item's shared memory is no longer read
  if (threadIdx.x == 0) *s_slot = atomicAdd(fs.ticket, 1);
  __syncthreads();
  const int t = *s_slot;
  return t < total ? t : -1;
}

// Completion flags take two values: kFlagCore when a factor item has stored
// its factor blocks (U_e and the two off-diagonal blocks; its trailing
// products may still run), kFlagDone when the item is complete. A dependency
// d >= 0 waits for item d to be done; d <= -2 waits only for item -d-2's
// factor blocks (kFlagCore or later); -1 is none. Items that publish only at
// the end satisfy both kinds of wait.
constexpr int kFlagCore = 1;
constexpr int kFlagDone = 2;

// Wait until the listed dependencies are met (all: done for d >= 0, factor blocks
// for d <= -2; core_only: the factor blocks of every listed item; full_only: only
// the d >= 0 ones, done). Thread 0 polls; returns false (for every thread) when
// the wait gave up.
enum FlowWaitKind { kWaitAll = 0, kWaitCoreOnly = 1, kWaitFullOnly = 2 };
__device__ __forceinline__ bool flow_wait(const FlowSync &fs, const int32_t *deps, int ndeps, int *s_ok,
                                          int kind = kWaitAll) {
  if (threadIdx.x == 0) {
    int ok = 1;
    for (int k = 0; k < ndeps && ok; ++k) {
      const int dd = deps[k];
      if (dd == -1) continue;
      const int d = dd >= 0 ? dd : -dd - 2;
      if (kind == kWaitFullOnly && dd < 0) continue;
      const int need = (dd < 0 || kind == kWaitCoreOnly) ? kFlagCore : kFlagDone;
      long long polls = 0;
      while (ld_acquire_gpu(fs.done + d) < need) {
        // the status word is checked every 64 polls; the first polls spin without sleeping
        if ((++polls & 63) == 0 && (polls > fs.max_polls || *((volatile int *)fs.status) != 0)) {
          atomicOr(fs.status, kFlowTimeout);
          ok = 0;
          break;
        }
        if (polls > 32) __nanosleep(64);
      }
    }
    *s_ok = ok;
  }
  __syncthreads();
  return *s_ok != 0;
}

// Publish item t as done (after all of this CTA's global writes for it). The CTA barrier orders
// every thread's writes before thread 0's release store (barriers synchronize the threads of a CTA
// in the memory model's causality order, and a release is cumulative over it), so no separate
// sequentially consistent fence is needed; a consumer's acquire load of the flag followed by its
// own CTA barrier makes the writes visible to all of its threads.
__device__ __forceinline__ void flow_publish(const FlowSync &fs, int t) {
  __syncthreads();
  if (threadIdx.x == 0) st_release_gpu(fs.done + t, kFlagDone);
}

// Publish that factor item t has stored its factor blocks (kFlagCore); the same ordering as flow_publish.
__device__ __forceinline__ void flow_publish_core(const FlowSync &fs, int t) {
  __syncthreads();
  if (threadIdx.x == 0) st_release_gpu(fs.done + t, kFlagCore);
}

// Result of a failed pivot: packed (node, column) for an atomicMin.
__device__ __forceinline__ unsigned long long pack_info(int node, int col) {
  return ((unsigned long long)(unsigned)node << 20) | (unsigned)col;
}

// ----------------------------------------------------- blocked factorization
// Column-wise forward substitution with the transposed diagonal block:
// X[p0 .. p0+PB)[col] <- U_pp^{-T} X[p0 .. p0+PB)[col] for one column of a
// shared-memory block X (U_pp read from S, reciprocal diagonal from dinv).
template <class C, typename T>
__device__ __forceinline__ void col_subst_ut(T *X, int col, const T *S, const T *dinv, int p0) {
  constexpr int PB = C::PB;
  constexpr int LD = C::LD;
  T w[PB];
#pragma unroll
  for (int t = 0; t < PB; ++t) w[t] = X[(p0 + t) * LD + col];
#pragma unroll
  for (int t = 0; t < PB; ++t) {
    w[t] *= dinv[p0 + t];
#pragma unroll
    for (int u = t + 1; u < PB; ++u) w[u] = fma(-S[(p0 + t) * LD + p0 + u], w[t], w[u]);
  }
#pragma unroll
  for (int t = 0; t < PB; ++t) X[(p0 + t) * LD + col] = w[t];
}

// One warp factors the PB-row panel of S (rows p0 .. p0+PB, columns p0 .. NP)
// in registers: right-looking upper Cholesky of the diagonal block fused with
// the solve of the panel's right part, U[p, j] = U_pp^{-T} S[p, j]. Lane l
// holds column p0 + l + 32 s (all PB rows) in v[s][.]; step k broadcasts the
// pivot (lane k) and the scaled row k (lanes k+1 .. PB-1) with shuffles.
// Entries below the diagonal are left stale. A pivot that is not positive (or
// NaN) is reported and replaced by 1 so that the remaining arithmetic stays
// finite. Writes 1/U_kk to dinv.
template <class C, typename T>
__device__ __forceinline__ void warp_panel_potrf(T *S, int p0, T *dinv, unsigned long long *info, int node,
                                                 int col_base = 0) {
  constexpr int PB = C::PB, NP = C::NP, LD = C::LD;
  constexpr int CPL = (NP + 31) / 32;  // column slots per lane
  const int lane = threadIdx.x & 31;
  T v[CPL][PB];
#pragma unroll
  for (int s = 0; s < CPL; ++s) {
    const int j = p0 + lane + 32 * s;
#pragma unroll
    for (int t = 0; t < PB; ++t) v[s][t] = j < NP ? S[(p0 + t) * LD + j] : T(0);
  }
  // next pivot candidate: lane k+1 forms S[k+1][k+1] - U[k][k+1]^2 from its own entry, so the pivot chain
  // is shuffle, rsqrt, scale, fma per step (the same operation the update loop applies to that entry)
  T piv = v[0][0];
#pragma unroll
  for (int k = 0; k < PB; ++k) {
    T d = __shfl_sync(0xffffffffu, piv, k);
    if (!(d > T(0))) {  // uniform across the warp
      if (lane == 0 && info) atomicMin(info, pack_info(node, col_base + p0 + k));
      d = T(1);
      if (lane == k) v[0][k] = T(1);
    }
    const T rs = rsqrt(d);
    if (lane == 0) dinv[p0 + k] = rs;
#pragma unroll
    for (int s = 0; s < CPL; ++s) v[s][k] *= rs;  // row k of U (the pivot becomes sqrt(d))
    if (k + 1 < PB) piv = fma(-v[0][k], v[0][k], v[0][k + 1 < PB ? k + 1 : k]);
#pragma unroll
    for (int t = k + 1; t < PB; ++t) {
      const T ukt = __shfl_sync(0xffffffffu, v[0][k], t);  // U[k][p0 + t]
#pragma unroll
      for (int s = 0; s < CPL; ++s) v[s][t] = fma(-ukt, v[s][k], v[s][t]);
    }
  }
#pragma unroll
  for (int s = 0; s < CPL; ++s) {
    const int j = p0 + lane + 32 * s;
    if (j < NP)
#pragma unroll
      for (int t = 0; t < PB; ++t) S[(p0 + t) * LD + j] = v[s][t];
  }
}

// FP64 blocks of one panel (n_p = 8 or 16) whose rows fit one per lane group
// of the CTA's warps: the elimination of block_potrf_trsm with the rows spread
// over the warps instead of one warp. A warp's FP64 instruction holds its SM
// sub-partition's FP64 pipe for the same time whatever its active lanes, so the
// single panel warp's rank-1 updates and column substitutions (one instruction
// per row and step) made that warp's pipe the chain; here the lanes of a group
// of n_p lanes hold one row (lane = column), the owner of row k forms the pivot
// and scales its row, stores it, and after a CTA barrier every row below takes
// its update: one FP64 instruction per warp and step. The solve of Z0, Z1 runs
// the same way (the lanes of a 2 n_p group hold one row of both blocks). Every
// element receives the same operations in the same order as block_potrf_trsm
// (pivot d_k, U(k, j) = S(k, j) rsqrt(d_k), S(t, j) -= U(k, t) U(k, j); then
// z_t *= 1 / U_tt, z_u -= U(t, u) z_t), so the factors are the same bits.
template <class C, typename T>
struct RowsPotrf {
  static constexpr int NP = C::NP, NW = C::NT / 32, HALF = 32 / C::NP, ZG = HALF / 2;
  static constexpr bool value = sizeof(T) == 8 && C::NPAN == 1 && (NP == 8 || NP == 16) && NW * HALF >= NP;
};

template <class C, typename T, class WaitOperands>
__device__ __forceinline__ void block_potrf_trsm_rows(T *S, T *dinv, T *Z0, T *Z1, unsigned long long *info,
                                                      int node, WaitOperands &&wait_operands, int col_base) {
  using RP = RowsPotrf<C, T>;
  constexpr int NP = RP::NP, LD = C::LD, NW = RP::NW, ZG = RP::ZG;
  constexpr int ZS = (NP + NW * ZG - 1) / (NW * ZG);  // row slots per lane in the solve
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  // ---- Cholesky: lane group hf of warp w holds row hf * NW + w, lane col its column
  {
    const int hf = lane / NP, col = lane % NP, t_own = hf * NW + warp;
    T v = t_own < NP ? S[t_own * LD + col] : T(0);
#pragma unroll
    for (int k = 0; k < NP; ++k) {
      const int ow = k % NW, oh = k / NW;
      if (warp == ow) {  // warp-uniform: the owner of row k
        T d = __shfl_sync(0xffffffffu, v, oh * NP + k);
        if (!(d > T(0))) {
          if (lane == 0 && info) atomicMin(info, pack_info(node, col_base + k));
          d = T(1);
          if (hf == oh && col == k) v = T(1);
        }
        const T rs = rsqrt(d);
        if (hf == oh) {
          v *= rs;  // row k of U (the pivot becomes sqrt(d))
          S[k * LD + col] = v;
        }
        if (lane == 0) dinv[k] = rs;
      }
      __syncthreads();
      if (t_own > k && t_own < NP) v = fma(-S[k * LD + t_own], S[k * LD + col], v);
    }
  }
  wait_operands();
  if (!Z0 && !Z1) return;
  __syncthreads();
  // ---- Z <- U^{-T} Z: lane group zg of warp w holds rows s * NW * ZG + zg * NW + w of Z0 (lanes
  // 0 .. NP-1 of the group) and Z1 (the next NP lanes)
  {
    const int zg = lane / (2 * NP), zc = lane % (2 * NP), col = zc % NP;
    T *Z = zc < NP ? Z0 : Z1;
    T z[ZS];
#pragma unroll
    for (int sl = 0; sl < ZS; ++sl) {
      const int u = sl * NW * ZG + zg * NW + warp;
      z[sl] = (Z && u < NP) ? Z[u * LD + col] : T(0);
    }
#pragma unroll
    for (int t = 0; t < NP; ++t) {
      const int ow = t % NW, og = (t / NW) % ZG, os = t / (NW * ZG);
      if (warp == ow && zg == og && Z) {
        z[os] *= dinv[t];
        Z[t * LD + col] = z[os];
      }
      __syncthreads();
#pragma unroll
      for (int sl = 0; sl < ZS; ++sl) {
        const int u = sl * NW * ZG + zg * NW + warp;
        if (Z && u > t && u < NP) z[sl] = fma(-S[t * LD + u], Z[t * LD + col], z[sl]);
      }
    }
  }
}

// Blocked upper Cholesky S = U^T U fused with Z <- U^{-T} Z for up to two
// right-hand-side blocks (either may be null), pipelined by panels: while
// warp 0 factors panel p, the other warps apply panel p-1 to the rows of S
// below panel p and Z_{p-1} to the rows of Z from p on; then all threads solve
// panel p of Z (column substitution) and update the next panel's rows of S
// with panel p. Every element receives the same updates in the same order as
// the unpipelined blocked Cholesky followed by the blocked triangular solve
// (right-looking by panels), so the results are identical; the pipelining only
// overlaps the single-warp panel factorization with the trailing updates. wait_operands(): called by every thread after the first
// panel, before Z0/Z1 are first read (their asynchronous copies were issued
// before the call). col_base: column of S's first row within the node's block,
// for the pivot report (S is a diagonal tile of a larger block).
template <class C, typename T, class WaitOperands>
__device__ __forceinline__ void block_potrf_trsm(T *S, T *dinv, T *Z0, T *Z1, unsigned long long *info, int node,
                                                 WaitOperands &&wait_operands, int col_base = 0) {
  if constexpr (RowsPotrf<C, T>::value) {
    block_potrf_trsm_rows<C>(S, dinv, Z0, Z1, info, node, wait_operands, col_base);
    __syncthreads();
    return;
  }
  constexpr int PB = C::PB, NP = C::NP, R = C::R, TXN = C::TXN, NT = C::NT;
  const int tid = threadIdx.x;
  const bool solve = Z0 || Z1;
#pragma unroll 1
  for (int p = 0; p < C::NPAN; ++p) {
    const int p0 = p * PB;
    if (tid < 32) {
      warp_panel_potrf<C>(S, p0, dinv, info, node, col_base);
    } else if (p > 0) {
      const int q0 = p0 - PB;                     // panel p-1
      const int tb = (NP - p0 - PB) / R;          // tile rows of S below panel p
      const int nb = tb * (tb + 1) / 2;           // their upper tiles
      const int zr = (NP - p0) / R;               // tile rows of Z from p0 on
      const int nz = solve ? 2 * zr * TXN : 0;
      for (int u = tid - 32; u < nb + nz; u += NT - 32) {
        if (u < nb) {
          int tr = 0, rem = u;
          while (rem >= tb - tr) {
            rem -= tb - tr;
            ++tr;
          }
          const int r0 = p0 + PB + tr * R, c0 = r0 + rem * R;
          T a[R][R];
          tile_from_smem<C>(a, S, r0, c0);
          tile_sub_xty<C, PB>(a, S, S, r0, c0, q0);
          tile_to_smem<C>(S, a, r0, c0);
        } else {
          const int v = u - nb, w = v % (zr * TXN);
          T *Z = v < zr * TXN ? Z0 : Z1;
          if (Z) {
            const int r0 = p0 + (w / TXN) * R, c0 = (w % TXN) * R;
            T a[R][R];
            tile_from_smem<C>(a, Z, r0, c0);
            tile_sub_xty<C, PB>(a, S, Z, r0, c0, q0);  // Z[i][j] -= sum_k U[k][i] Z[k][j], k in panel p-1
            tile_to_smem<C>(Z, a, r0, c0);
          }
        }
      }
    }
    if (p == 0) wait_operands();
    __syncthreads();
    if (solve)
      for (int q = tid; q < 2 * NP; q += NT) {
        T *Z = q < NP ? Z0 : Z1;
        if (Z) col_subst_ut<C>(Z, q % NP, S, dinv, p0);
      }
    if (p + 1 < C::NPAN) {  // the next panel's rows of S with panel p
      constexpr int ta = PB / R;
      const int tcols = (NP - p0 - PB) / R;
      const int na = ta * tcols - ta * (ta - 1) / 2;
      for (int u = tid; u < na; u += NT) {
        int i = 0, rem = u;
        while (rem >= tcols - i) {
          rem -= tcols - i;
          ++i;
        }
        const int r0 = p0 + PB + i * R, c0 = r0 + rem * R;
        T a[R][R];
        tile_from_smem<C>(a, S, r0, c0);
        tile_sub_xty<C, PB>(a, S, S, r0, c0, p0);
        tile_to_smem<C>(S, a, r0, c0);
      }
    }
    __syncthreads();
  }
}

// Z <- U^{-T} Z with an upper factor U already in shared memory (dinv holds
// 1 / U_kk), right-looking by panels: the column substitution of panel p on
// every column of Z, then the rows below it receive the panel's contribution
// (the same steps block_potrf_trsm applies to its right-hand sides).
template <class C, typename T>
__device__ __forceinline__ void block_trsm_ut(T *Z, const T *U, const T *dinv) {
  constexpr int PB = C::PB, NP = C::NP, R = C::R, TXN = C::TXN, NT = C::NT;
  const int tid = threadIdx.x;
#pragma unroll 1
  for (int p = 0; p < C::NPAN; ++p) {
    const int p0 = p * PB;
    for (int q = tid; q < NP; q += NT) col_subst_ut<C>(Z, q, U, dinv, p0);
    __syncthreads();
    const int tb = (NP - p0 - PB) / R;  // tile rows below the panel
    for (int u = tid; u < tb * TXN; u += NT) {
      const int r0 = p0 + PB + (u / TXN) * R, c0 = (u % TXN) * R;
      T a[R][R];
      tile_from_smem<C>(a, Z, r0, c0);
      tile_sub_xty<C, PB>(a, U, Z, r0, c0, p0);
      tile_to_smem<C>(Z, a, r0, c0);
    }
    __syncthreads();
  }
}

}  // namespace btc
