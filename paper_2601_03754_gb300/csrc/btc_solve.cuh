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

template <int NP>
struct SolveCfg {
  static constexpr int LDL = NP + 1;  // padded leading dimension: conflict-free row and column reads
};

template <typename T>
__device__ __forceinline__ T warp_bcast(T v, int lane) {
  return __shfl_sync(0xffffffffu, v, lane);
}

// Dense lower block L (np x np, row-major, global) -> shared memory with
// leading dimension NP+1, and 1/L_jj into dinv.
template <typename T, int NP>
__device__ __forceinline__ void stage_lower(T *Ls, T *dinv, const T *g) {
  constexpr int LDL = SolveCfg<NP>::LDL;
  for (int q = threadIdx.x; q < NP * NP; q += blockDim.x) Ls[(q / NP) * LDL + q % NP] = g[q];
  __syncthreads();
  for (int j = threadIdx.x; j < NP; j += blockDim.x) dinv[j] = T(1) / Ls[j * LDL + j];
}

// y <- L^{-1} y for the m columns of Y (np x m in shared memory), by warps:
// warp w takes columns w, w + nwarps, ...; lane t holds rows t and t + 32.
template <typename T, int NP>
__device__ __forceinline__ void warp_trsv_lower(T *Y, int m, const T *Ls, const T *dinv) {
  constexpr int LDL = SolveCfg<NP>::LDL;
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
      const T yj = warp_bcast((RPL == 1 || j < 32) ? v[0] : v[RPL - 1], j & 31) * dinv[j];
#pragma unroll
      for (int s = 0; s < RPL; ++s) {
        const int i = lane + 32 * s;
        if (i > j && i < NP) v[s] = fma(-Ls[i * LDL + j], yj, v[s]);
        if (i == j) v[s] = yj;
      }
    }
#pragma unroll
    for (int s = 0; s < RPL; ++s) {
      const int i = lane + 32 * s;
      if (i < NP) Y[i * m + q] = v[s];
    }
  }
}

// x <- L^{-T} x (backward substitution with the transpose).
template <typename T, int NP>
__device__ __forceinline__ void warp_trsv_lower_t(T *Y, int m, const T *Ls, const T *dinv) {
  constexpr int LDL = SolveCfg<NP>::LDL;
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
        if (i < j) v[s] = fma(-Ls[j * LDL + i], xj, v[s]);
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
template <typename T, int NP>
__global__ void __launch_bounds__(kSolveThreads) k_fwd_level(SolveArgs a) {
  constexpr int LDL = SolveCfg<NP>::LDL;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  const int m = a.m;
  T *Ls = reinterpret_cast<T *>(smem_raw);  // NP * LDL
  T *dinv = Ls + NP * LDL;                  // NP
  T *ys = dinv + NP;                        // NP*m
  T *yl = ys + NP * m;                      // NP*m
  T *yr = yl + NP * m;                      // NP*m
  const FwdItem it = reinterpret_cast<const FwdItem *>(a.items)[blockIdx.x];
  T *y = reinterpret_cast<T *>(a.y);
  const T *dpool = reinterpret_cast<const T *>(a.dpool);
  const T *epool = reinterpret_cast<const T *>(a.epool);
  const int nm = NP * m;
  T *yself = y + it.y_self * nm;
  for (int q = threadIdx.x; q < nm; q += blockDim.x) {
    ys[q] = yself[q];
    if (it.y_l >= 0) yl[q] = y[it.y_l * nm + q];
    if (it.y_r >= 0) yr[q] = y[it.y_r * nm + q];
  }
  if (it.d_self >= 0) stage_lower<T, NP>(Ls, dinv, dpool + it.d_self);
  __syncthreads();
  if (it.y_l >= 0) {
    const T *Ul = epool + it.e_l;
    const T *Ur = it.y_r >= 0 ? epool + it.e_r : nullptr;
    for (int q = threadIdx.x; q < nm; q += blockDim.x) {
      const int c = q / m, col = q % m;
      T acc = ys[q];
#pragma unroll 8
      for (int r = 0; r < NP; ++r) acc = fma(-Ul[r * NP + c], yl[r * m + col], acc);
      if (Ur)
#pragma unroll 8
        for (int r = 0; r < NP; ++r) acc = fma(-Ur[r * NP + c], yr[r * m + col], acc);
      ys[q] = acc;
    }
    __syncthreads();
  }
  if (it.d_self >= 0) {
    warp_trsv_lower<T, NP>(ys, m, Ls, dinv);
    __syncthreads();
  }
  for (int q = threadIdx.x; q < nm; q += blockDim.x) yself[q] = ys[q];
}

// Backward step of one level: one CTA per eliminated node e.
template <typename T, int NP>
__global__ void __launch_bounds__(kSolveThreads) k_bwd_level(SolveArgs a) {
  constexpr int LDL = SolveCfg<NP>::LDL;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  const int m = a.m;
  T *Ls = reinterpret_cast<T *>(smem_raw);  // NP * LDL
  T *Ud = Ls + NP * LDL;                    // NP * LDL
  T *Uu = Ud + NP * LDL;                    // NP * LDL
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
  for (int q = threadIdx.x; q < nm; q += blockDim.x) {
    ys[q] = yself[q];
    if (it.x_dn >= 0) xd[q] = y[it.x_dn * nm + q];
    if (it.x_up >= 0) xu[q] = y[it.x_up * nm + q];
  }
  for (int q = threadIdx.x; q < NP * NP; q += blockDim.x) {
    const int r = q / NP, c = q % NP;
    if (it.x_dn >= 0) Ud[r * LDL + c] = epool[it.e_dn + q];
    if (it.x_up >= 0) Uu[r * LDL + c] = epool[it.e_up + q];
  }
  stage_lower<T, NP>(Ls, dinv, dpool + it.d_self);
  __syncthreads();
  if (it.x_dn >= 0 || it.x_up >= 0) {
    for (int q = threadIdx.x; q < nm; q += blockDim.x) {
      const int r = q / m, col = q % m;
      T acc = ys[q];
      if (it.x_dn >= 0)
#pragma unroll 8
        for (int c = 0; c < NP; ++c) acc = fma(-Ud[r * LDL + c], xd[c * m + col], acc);
      if (it.x_up >= 0)
#pragma unroll 8
        for (int c = 0; c < NP; ++c) acc = fma(-Uu[r * LDL + c], xu[c * m + col], acc);
      ys[q] = acc;
    }
    __syncthreads();
  }
  warp_trsv_lower_t<T, NP>(ys, m, Ls, dinv);
  __syncthreads();
  for (int q = threadIdx.x; q < nm; q += blockDim.x) yself[q] = ys[q];
}

template <typename T, int NP>
constexpr size_t fwd_smem_bytes(int m) {
  return sizeof(T) * ((size_t)NP * SolveCfg<NP>::LDL + NP + 3 * (size_t)NP * m);
}
template <typename T, int NP>
constexpr size_t bwd_smem_bytes(int m) {
  return sizeof(T) * (3 * (size_t)NP * SolveCfg<NP>::LDL + NP + 3 * (size_t)NP * m);
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

// r = b - Psi x in FP64 for one block row per CTA; writes r (converted to T)
// into the padded work vector y when y != nullptr, and max|r|, max|x| into
// norms[0], norms[1]. D: lower triangles read.
template <typename T>
__global__ void k_residual(T *y, const double *D, const double *B, const double *x, const double *b, int N, int n,
                           int np, int m, int64_t node_base, double *norms) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  const int i = blockIdx.x;
  const int ld = n + 1;
  double *Ds = reinterpret_cast<double *>(smem_raw);
  double *Bl = Ds + n * ld;  // B_{i-1}: row i's left block
  double *Br = Bl + n * ld;  // B_i:     transposed: row i's right block
  const size_t bs = (size_t)n * n;
  for (int q = threadIdx.x; q < n * n; q += blockDim.x) {
    const int r = q / n, c = q % n;
    Ds[r * ld + c] = D[i * bs + q];
    if (i > 0) Bl[r * ld + c] = B[(i - 1) * bs + q];
    if (i + 1 < N) Br[r * ld + c] = B[i * bs + q];
  }
  __syncthreads();
  double rmax = 0.0, xmax = 0.0;
  for (int q = threadIdx.x; q < n * m; q += blockDim.x) {
    const int r = q / m, col = q % m;
    double v = b[((size_t)i * n + r) * m + col];
    const double *xi = x + (size_t)i * n * m;
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
