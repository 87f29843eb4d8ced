// Level-wise forward and backward substitution (Alg. 7), residual, norms and
// the vector conversions around them.
//
// Work vector layout: y[node][np][m] (node = global node index, rows padded to
// np with zeros), element type T of the factor.
#pragma once
#include <cuda_runtime.h>
#include <stdint.h>

#include "btc_internal.h"

namespace btc {

constexpr int kSolveThreads = 128;

template <typename T, int NP>
struct SolveCfg {
  // padded leading dimension; rows stay 16-byte aligned for cp.async
  static constexpr int LDL = NP + 16 / (int)sizeof(T);
};

__device__ __forceinline__ void cp_async16_s(void *smem, const void *gmem) {
  const unsigned s = (unsigned)__cvta_generic_to_shared(smem);
  asm volatile("cp.async.cg.shared.global [%0], [%1], 16;\n" ::"r"(s), "l"(gmem) : "memory");
}
__device__ __forceinline__ void cp_async_wait_all_s() {
  asm volatile("cp.async.commit_group;\ncp.async.wait_all;\n" ::: "memory");
}

template <typename T>
__device__ __forceinline__ T warp_bcast(T v, int lane) {
  return __shfl_sync(0xffffffffu, v, lane);
}

// Pool block (np x np, row-major) -> shared memory with leading dimension LDL,
// by cp.async (completes at cp_async_wait_all_s() + __syncthreads()).
template <typename T, int NP>
__device__ __forceinline__ void stage_block(T *dst, const T *g) {
  constexpr int LDL = SolveCfg<T, NP>::LDL;
  constexpr int V = 16 / sizeof(T);
  constexpr int CPR = NP / V;
  constexpr int CHUNKS = NP * CPR;
#pragma unroll 4
  for (int q = threadIdx.x; q < CHUNKS; q += kSolveThreads) {
    const int row = q / CPR, col = (q % CPR) * V;
    cp_async16_s(dst + row * LDL + col, g + (size_t)row * NP + col);
  }
}

// Contiguous vector of `count` elements (count * sizeof(T) a multiple of 16) -> shared memory.
template <typename T>
__device__ __forceinline__ void stage_vec(T *dst, const T *g, int count) {
  constexpr int V = 16 / sizeof(T);
  for (int q = threadIdx.x; q < count / V; q += blockDim.x) cp_async16_s(dst + q * V, g + q * V);
}

// Y <- U^{-T} Y (forward, with the upper factor U) for the m columns of Y
// (np x m in shared memory), by warps: warp w takes columns w, w + nwarps, ...;
// lane t holds rows t and t + 32. Row j of U is read (U[j][i], i > j).
template <typename T, int NP>
__device__ __forceinline__ void warp_trsv_ut(T *Y, int m, const T *Us, const T *dinv) {
  constexpr int LDL = SolveCfg<T, NP>::LDL;
  constexpr int RPL = (NP + 31) / 32;  // rows per lane
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nw = blockDim.x >> 5;
  for (int q = warp; q < m; q += nw) {
    T v[RPL];
#pragma unroll
    for (int s = 0; s < RPL; ++s) {
      const int i = lane + 32 * s;
      v[s] = i < NP ? Y[i * m + q] : T(0);
    }
#pragma unroll 4
    for (int j = 0; j < NP; ++j) {
      const T zj = warp_bcast((RPL == 1 || j < 32) ? v[0] : v[RPL - 1], j & 31) * dinv[j];
#pragma unroll
      for (int s = 0; s < RPL; ++s) {
        const int i = lane + 32 * s;
        if (i > j && i < NP) v[s] = fma(-Us[j * LDL + i], zj, v[s]);
        if (i == j) v[s] = zj;
      }
    }
#pragma unroll
    for (int s = 0; s < RPL; ++s) {
      const int i = lane + 32 * s;
      if (i < NP) Y[i * m + q] = v[s];
    }
  }
}

// Y <- U^{-1} Y (backward substitution with the upper factor; column j of U read).
template <typename T, int NP>
__device__ __forceinline__ void warp_trsv_u(T *Y, int m, const T *Us, const T *dinv) {
  constexpr int LDL = SolveCfg<T, NP>::LDL;
  constexpr int RPL = (NP + 31) / 32;
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nw = blockDim.x >> 5;
  for (int q = warp; q < m; q += nw) {
    T v[RPL];
#pragma unroll
    for (int s = 0; s < RPL; ++s) {
      const int i = lane + 32 * s;
      v[s] = i < NP ? Y[i * m + q] : T(0);
    }
#pragma unroll 4
    for (int j = NP - 1; j >= 0; --j) {
      const T xj = warp_bcast((RPL == 1 || j < 32) ? v[0] : v[RPL - 1], j & 31) * dinv[j];
#pragma unroll
      for (int s = 0; s < RPL; ++s) {
        const int i = lane + 32 * s;
        if (i < j) v[s] = fma(-Us[i * LDL + j], xj, v[s]);
        if (i == j) v[s] = xj;
      }
    }
#pragma unroll
    for (int s = 0; s < RPL; ++s) {
      const int i = lane + 32 * s;
      if (i < NP) Y[i * m + q] = v[s];
    }
  }
}

struct SolveArgs {
  const void *items;
  int count;
  const void *dpool;
  const void *epool;
  void *y;  // work vector
  int m;
};

// Forward step of one level (pull form): one CTA per surviving node j.
//   y_j -= U(j-h, j)^T y_{j-h} + U(j+h, j)^T y_{j+h}   (contributions of level l-1)
//   y_j <- U_j^{-T} y_j                                 (if j is eliminated at level l)
template <typename T, int NP>
__global__ void __launch_bounds__(kSolveThreads) k_fwd_level(SolveArgs a) {
  constexpr int LDL = SolveCfg<T, NP>::LDL;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  const int m = a.m;
  T *Us = reinterpret_cast<T *>(smem_raw);  // U_j
  T *Ul = Us + NP * LDL;                    // U(j-h, j)
  T *Ur = Ul + NP * LDL;                    // U(j+h, j)
  T *dinv = Ur + NP * LDL;                  // NP
  T *ys = dinv + NP;                        // NP*m
  T *yl = ys + NP * m;
  T *yr = yl + NP * m;
  const FwdItem it = reinterpret_cast<const FwdItem *>(a.items)[blockIdx.x];
  T *y = reinterpret_cast<T *>(a.y);
  const T *dpool = reinterpret_cast<const T *>(a.dpool);
  const T *epool = reinterpret_cast<const T *>(a.epool);
  const int nm = NP * m;
  T *yself = y + it.y_self * nm;
  if (it.d_self >= 0) stage_block<T, NP>(Us, dpool + it.d_self);
  if (it.y_l >= 0) stage_block<T, NP>(Ul, epool + it.e_l);
  if (it.y_r >= 0) stage_block<T, NP>(Ur, epool + it.e_r);
  stage_vec<T>(ys, yself, nm);
  if (it.y_l >= 0) stage_vec<T>(yl, y + it.y_l * nm, nm);
  if (it.y_r >= 0) stage_vec<T>(yr, y + it.y_r * nm, nm);
  cp_async_wait_all_s();
  __syncthreads();
  if (it.d_self >= 0)
    for (int j = threadIdx.x; j < NP; j += blockDim.x) dinv[j] = T(1) / Us[j * LDL + j];
  if (it.y_l >= 0) {
    const bool right = it.y_r >= 0;
    for (int q = threadIdx.x; q < nm; q += blockDim.x) {
      const int c = q / m, col = q % m;
      T acc = ys[q];
#pragma unroll 8
      for (int r = 0; r < NP; ++r) acc = fma(-Ul[r * LDL + c], yl[r * m + col], acc);
      if (right)
#pragma unroll 8
        for (int r = 0; r < NP; ++r) acc = fma(-Ur[r * LDL + c], yr[r * m + col], acc);
      ys[q] = acc;
    }
  }
  __syncthreads();
  if (it.d_self >= 0) {
    warp_trsv_ut<T, NP>(ys, m, Us, dinv);
    __syncthreads();
  }
  for (int q = threadIdx.x; q < nm; q += blockDim.x) yself[q] = ys[q];
}

// Backward step of one level: one CTA per eliminated node e.
//   x_e <- U_e^{-1} (y_e - U(e, e+s) x_{e+s} - U(e, e-s) x_{e-s})
template <typename T, int NP>
__global__ void __launch_bounds__(kSolveThreads) k_bwd_level(SolveArgs a) {
  constexpr int LDL = SolveCfg<T, NP>::LDL;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  const int m = a.m;
  T *Us = reinterpret_cast<T *>(smem_raw);  // U_e
  T *Ud = Us + NP * LDL;                    // U(e, e+s)
  T *Uu = Ud + NP * LDL;                    // U(e, e-s)
  T *dinv = Uu + NP * LDL;                  // NP
  T *ys = dinv + NP;                        // NP*m
  T *xd = ys + NP * m;
  T *xu = xd + NP * m;
  const BwdItem it = reinterpret_cast<const BwdItem *>(a.items)[blockIdx.x];
  T *y = reinterpret_cast<T *>(a.y);
  const T *dpool = reinterpret_cast<const T *>(a.dpool);
  const T *epool = reinterpret_cast<const T *>(a.epool);
  const int nm = NP * m;
  T *yself = y + it.x_self * nm;
  stage_block<T, NP>(Us, dpool + it.d_self);
  if (it.x_dn >= 0) stage_block<T, NP>(Ud, epool + it.e_dn);
  if (it.x_up >= 0) stage_block<T, NP>(Uu, epool + it.e_up);
  stage_vec<T>(ys, yself, nm);
  if (it.x_dn >= 0) stage_vec<T>(xd, y + it.x_dn * nm, nm);
  if (it.x_up >= 0) stage_vec<T>(xu, y + it.x_up * nm, nm);
  cp_async_wait_all_s();
  __syncthreads();
  for (int j = threadIdx.x; j < NP; j += blockDim.x) dinv[j] = T(1) / Us[j * LDL + j];
  if (it.x_dn >= 0 || it.x_up >= 0) {
    const bool dn = it.x_dn >= 0, up = it.x_up >= 0;
    for (int q = threadIdx.x; q < nm; q += blockDim.x) {
      const int r = q / m, col = q % m;
      T acc = ys[q];
      if (dn)
#pragma unroll 8
        for (int c = 0; c < NP; ++c) acc = fma(-Ud[r * LDL + c], xd[c * m + col], acc);
      if (up)
#pragma unroll 8
        for (int c = 0; c < NP; ++c) acc = fma(-Uu[r * LDL + c], xu[c * m + col], acc);
      ys[q] = acc;
    }
  }
  __syncthreads();
  warp_trsv_u<T, NP>(ys, m, Us, dinv);
  __syncthreads();
  for (int q = threadIdx.x; q < nm; q += blockDim.x) yself[q] = ys[q];
}

template <typename T, int NP>
constexpr size_t fwd_smem_bytes(int m) {
  return sizeof(T) * (3 * (size_t)NP * SolveCfg<T, NP>::LDL + NP + 3 * (size_t)NP * m);
}
template <typename T, int NP>
constexpr size_t bwd_smem_bytes(int m) {
  return sizeof(T) * (3 * (size_t)NP * SolveCfg<T, NP>::LDL + NP + 3 * (size_t)NP * m);
}

// ---------------------------------------------------------------- vectors
// Columns [col0, col0+m) of the user array b [N*n][ldb] (type S) -> y [N][np][m]
// (type T), zero padding.
template <typename T, typename S>
__global__ void k_pack_rhs(T *y, const S *b, int N, int n, int np, int m, int ldb, int col0, int64_t node_base) {
  const int64_t total = (int64_t)N * np * m;
  for (int64_t q = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; q < total; q += (int64_t)gridDim.x * blockDim.x) {
    const int64_t i = q / ((int64_t)np * m);
    const int r = (int)((q / m) % np), c = (int)(q % m);
    y[node_base * np * m + q] = r < n ? (T)b[(i * n + r) * ldb + col0 + c] : T(0);
  }
}

// y -> columns [col0, col0+m) of the user array x [N*n][ldx]; if accumulate:
// x += y (the FP64 update of the refinement).
template <typename T, typename S>
__global__ void k_unpack(S *x, const T *y, int N, int n, int np, int m, int ldx, int col0, int64_t node_base,
                         int accumulate) {
  const int64_t total = (int64_t)N * n * m;
  for (int64_t q = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; q < total; q += (int64_t)gridDim.x * blockDim.x) {
    const int64_t i = q / ((int64_t)n * m);
    const int r = (int)((q / m) % n), c = (int)(q % m);
    const S v = (S)y[node_base * np * m + (i * np + r) * m + c];
    S *dst = x + (i * n + r) * ldx + col0 + c;
    *dst = accumulate ? *dst + v : v;
  }
}

// Non-negative doubles order like their bit patterns.
__device__ __forceinline__ void atomic_max_nonneg(double *addr, double v) {
  atomicMax(reinterpret_cast<unsigned long long *>(addr), (unsigned long long)__double_as_longlong(v));
}

// Leading dimension of a staged n x n FP64 block: rows 16-byte aligned when n is even.
__host__ __device__ constexpr int f64_ld(int n) { return (n % 2 == 0) ? n + 2 : n + 1; }

// Copy an n x n FP64 block (row-major, contiguous) into shared memory with
// leading dimension f64_ld(n): cp.async of 16-byte chunks when n is even (the
// block and its rows are then 16-byte aligned), batched scalar loads otherwise.
// Completes at cp_async_wait_all_s() + __syncthreads().
__device__ __forceinline__ void stage_f64(double *dst, const double *src, int n) {
  const int ld = f64_ld(n);
  if (n % 2 == 0) {
    const int cpr = n / 2, total = n * cpr;
    for (int q = threadIdx.x; q < total; q += blockDim.x) {
      const int row = q / cpr, col = (q % cpr) * 2;
      cp_async16_s(dst + row * ld + col, src + (size_t)row * n + col);
    }
    return;
  }
  const int total = n * n;
  for (int base = threadIdx.x; base < total; base += 8 * blockDim.x) {
    double v[8];
#pragma unroll
    for (int u = 0; u < 8; ++u) {
      const int q = base + u * blockDim.x;
      v[u] = q < total ? __ldg(src + q) : 0.0;
    }
#pragma unroll
    for (int u = 0; u < 8; ++u) {
      const int q = base + u * blockDim.x;
      if (q < total) dst[(q / n) * ld + q % n] = v[u];
    }
  }
}

// r = b - Psi x in FP64 for one block row per CTA; writes r (converted to T)
// into the padded work vector y when y != nullptr, and max|r|, max|x| into
// norms[0], norms[1]. D: lower triangles read.
template <typename T>
__global__ void k_residual(T *y, const double *D, const double *B, const double *x, const double *b, int N, int n,
                           int np, int m, int64_t node_base, double *norms) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  const int i = blockIdx.x;
  const int ld = f64_ld(n);
  double *Ds = reinterpret_cast<double *>(smem_raw);
  double *Bl = Ds + n * ld;  // B_{i-1}: row i's left block
  double *Br = Bl + n * ld;  // B_i:     transposed: row i's right block
  const size_t bs = (size_t)n * n;
  stage_f64(Ds, D + i * bs, n);
  if (i > 0) stage_f64(Bl, B + (i - 1) * bs, n);
  if (i + 1 < N) stage_f64(Br, B + i * bs, n);
  cp_async_wait_all_s();
  __syncthreads();
  double rmax = 0.0, xmax = 0.0;
  const double *xi = x + (size_t)i * n * m;
  for (int q = threadIdx.x; q < n * m; q += blockDim.x) {
    const int r = q / m, col = q % m;
    double v = b[((size_t)i * n + r) * m + col];
    for (int c = 0; c < n; ++c) v = fma(-(r >= c ? Ds[r * ld + c] : Ds[c * ld + r]), xi[c * m + col], v);
    if (i > 0) {
      const double *xp = x + (size_t)(i - 1) * n * m;
      for (int c = 0; c < n; ++c) v = fma(-Bl[r * ld + c], xp[c * m + col], v);
    }
    if (i + 1 < N) {
      const double *xn = x + (size_t)(i + 1) * n * m;
      for (int c = 0; c < n; ++c) v = fma(-Br[c * ld + r], xn[c * m + col], v);
    }
    if (y) y[(node_base + i) * np * m + r * m + col] = (T)v;
    rmax = fmax(rmax, fabs(v));
    xmax = fmax(xmax, fabs(xi[r * m + col]));
  }
  if (y) {
    for (int q = threadIdx.x; q < (np - n) * m; q += blockDim.x) y[(node_base + i) * np * m + n * m + q] = T(0);
  }
  for (int o = 16; o > 0; o >>= 1) {
    rmax = fmax(rmax, __shfl_xor_sync(0xffffffffu, rmax, o));
    xmax = fmax(xmax, __shfl_xor_sync(0xffffffffu, xmax, o));
  }
  if ((threadIdx.x & 31) == 0) {
    atomic_max_nonneg(norms + 0, rmax);
    atomic_max_nonneg(norms + 1, xmax);
  }
}

}  // namespace btc
