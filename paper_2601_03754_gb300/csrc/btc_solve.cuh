// Level-wise forward and backward substitution (Alg. 7), residual, norms and
// the vector conversions around them.
//
// Work vector layout: y[node][np][m] (node = global node index, rows padded to
// np with zeros), element type T of the factor.
#pragma once
#include <cuda_runtime.h>
#include <stdint.h>

#include "btc_internal.h"
#include "btc_runtime.h"
#include "btc_tile.cuh"

namespace btc {

constexpr int kSolveThreads = 128;

template <typename T, int NP>
struct SolveCfg {
  // padded leading dimension; rows stay 16-byte aligned for cp.async
  static constexpr int LDL = NP + 16 / (int)sizeof(T);
  // large blocks: only the diagonal factor is staged in shared memory; the two
  // coupling blocks are read once from global memory inside the products
  // (three staged 128 x 128 blocks would leave one CTA per SM)
  static constexpr bool STREAM = NP >= 96;
  // blocks larger than 128 (256 KB in FP32): the diagonal factor is read from
  // global memory too, row by row inside the triangular solves
  static constexpr bool DIAG_GLOBAL = NP > 128;
  static constexpr int LDU = DIAG_GLOBAL ? NP : LDL;  // leading dimension of the diagonal factor as read
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
  for (int q = threadIdx.x; q < CHUNKS; q += blockDim.x) {
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

// Warp triangular solves, in chunks of CH rows (one row per lane): a chunk's
// CH-step substitution chain keeps one value per lane in a register, then the
// rows outside the chunk receive its contribution as a plain product.
template <typename T, int NP>
struct TrsvCfg {
  static constexpr int CH = NP % 32 == 0 ? 32 : (NP % 16 == 0 ? 16 : NP);
  static constexpr int V = 16 / (int)sizeof(T);  // elements per 16-byte load
};

// Y <- U^{-T} Y (forward, with the upper factor U) for the m columns of Y
// (np x m in shared memory), by warps: warp w takes columns w, w + nwarps, ...,
// QG of them at a time (their substitution chains interleaved, the same
// operations per column). Row j of U is read (U[j][i], i > j), contiguous
// across lanes. U: shared memory, or global memory for the blocks of
// SolveCfg::DIAG_GLOBAL.
template <typename T, int NP, int QG>
__device__ __forceinline__ void warp_trsv_ut_cols(T *Y, int m, const T *Us, const T *dinv) {
  constexpr int LDL = SolveCfg<T, NP>::LDU, CH = TrsvCfg<T, NP>::CH;
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nw = blockDim.x >> 5;  // full warps only
  for (int q0 = warp; q0 < m && warp < nw; q0 += QG * nw) {
    int qc[QG];
    bool ok[QG];
#pragma unroll
    for (int c = 0; c < QG; ++c) {
      qc[c] = q0 + c * nw;
      ok[c] = qc[c] < m;
    }
#pragma unroll 1
    for (int base = 0; base < NP; base += CH) {
      T v[QG];
#pragma unroll
      for (int c = 0; c < QG; ++c) v[c] = (ok[c] && lane < CH) ? Y[(base + lane) * m + qc[c]] : T(0);
#pragma unroll
      for (int j = 0; j < CH; ++j) {
        T zj[QG];
#pragma unroll
        for (int c = 0; c < QG; ++c) zj[c] = warp_bcast(v[c], j) * dinv[base + j];
        if (lane > j && lane < CH) {
          const T uj = Us[(base + j) * LDL + base + lane];
#pragma unroll
          for (int c = 0; c < QG; ++c) v[c] = fma(-uj, zj[c], v[c]);
        }
        if (lane == j)
#pragma unroll
          for (int c = 0; c < QG; ++c) v[c] = zj[c];
      }
#pragma unroll
      for (int c = 0; c < QG; ++c)
        if (ok[c] && lane < CH) Y[(base + lane) * m + qc[c]] = v[c];
      __syncwarp();
#pragma unroll
      for (int c = 0; c < QG; ++c) {
        if (!ok[c]) continue;
        const int q = qc[c];
        for (int i = base + CH + lane; i < NP; i += 32) {  // rows below the chunk
          T acc = Y[i * m + q];
#pragma unroll 8
          for (int j = 0; j < CH; ++j) acc = fma(-Us[(base + j) * LDL + i], Y[(base + j) * m + q], acc);
          Y[i * m + q] = acc;
        }
      }
      __syncwarp();
    }
  }
}

template <typename T, int NP>
__device__ __forceinline__ void warp_trsv_ut(T *Y, int m, const T *Us, const T *dinv) {
  if (m == 1) warp_trsv_ut_cols<T, NP, 1>(Y, m, Us, dinv);
  else warp_trsv_ut_cols<T, NP, 4>(Y, m, Us, dinv);
}

// Y <- U^{-1} Y (backward substitution with the upper factor), chunks from the
// bottom, QG columns of a warp at a time. A lane's row of the chunk's diagonal
// block is loaded into registers with 16-byte loads (conflict-free at the
// padded leading dimension), so the substitution chain reads no shared memory.
template <typename T, int NP, int QG>
__device__ __forceinline__ void warp_trsv_u_cols(T *Y, int m, const T *Us, const T *dinv) {
  constexpr int LDL = SolveCfg<T, NP>::LDU, CH = TrsvCfg<T, NP>::CH, V = TrsvCfg<T, NP>::V;
  static_assert(CH % V == 0, "chunk rows must hold whole 16-byte loads");
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nw = blockDim.x >> 5;  // full warps only
  for (int q0 = warp; q0 < m && warp < nw; q0 += QG * nw) {
    int qc[QG];
    bool ok[QG];
#pragma unroll
    for (int c = 0; c < QG; ++c) {
      qc[c] = q0 + c * nw;
      ok[c] = qc[c] < m;
    }
#pragma unroll 1
    for (int base = NP - CH; base >= 0; base -= CH) {
      T u[CH];
      const int row = base + (lane < CH ? lane : 0);
#pragma unroll
      for (int j = 0; j < CH; j += V) {
        T w[V];
        vload<T, V>(Us + row * LDL + base + j, w);
#pragma unroll
        for (int t = 0; t < V; ++t) u[j + t] = w[t];
      }
      T v[QG];
#pragma unroll
      for (int c = 0; c < QG; ++c) v[c] = (ok[c] && lane < CH) ? Y[(base + lane) * m + qc[c]] : T(0);
#pragma unroll
      for (int j = CH - 1; j >= 0; --j) {
        T xj[QG];
#pragma unroll
        for (int c = 0; c < QG; ++c) xj[c] = warp_bcast(v[c], j) * dinv[base + j];
        if (lane < j)
#pragma unroll
          for (int c = 0; c < QG; ++c) v[c] = fma(-u[j], xj[c], v[c]);
        if (lane == j)
#pragma unroll
          for (int c = 0; c < QG; ++c) v[c] = xj[c];
      }
#pragma unroll
      for (int c = 0; c < QG; ++c)
        if (ok[c] && lane < CH) Y[(base + lane) * m + qc[c]] = v[c];
      __syncwarp();
#pragma unroll
      for (int c = 0; c < QG; ++c) {
        if (!ok[c]) continue;
        const int q = qc[c];
        for (int i = lane; i < base; i += 32) {  // rows above the chunk
          T acc = Y[i * m + q];
#pragma unroll
          for (int j = 0; j < CH; j += V) {
            T w[V];
            vload<T, V>(Us + i * LDL + base + j, w);
#pragma unroll
            for (int t = 0; t < V; ++t) acc = fma(-w[t], Y[(base + j + t) * m + q], acc);
          }
          Y[i * m + q] = acc;
        }
      }
      __syncwarp();
    }
  }
}

template <typename T, int NP>
__device__ __forceinline__ void warp_trsv_u(T *Y, int m, const T *Us, const T *dinv) {
  if (m == 1) warp_trsv_u_cols<T, NP, 1>(Y, m, Us, dinv);
  else warp_trsv_u_cols<T, NP, 4>(Y, m, Us, dinv);
}

struct SolveArgs {
  const void *items;
  int count;
  const void *dpool;
  const void *epool;
  void *y;  // work vector
  int m;
};

// Shared-memory layout of one solve item: the node's own factor block and
// (unless SolveCfg::STREAM) the two coupling blocks, the reciprocal diagonal,
// and three np x m vectors.
template <typename T, int NP>
struct SolveSmem {
  T *U0, *U1, *U2, *dinv, *y0, *y1, *y2, *part;
  __device__ __forceinline__ explicit SolveSmem(unsigned char *raw, int m) {
    constexpr int LDL = SolveCfg<T, NP>::LDL;
    constexpr int NB = SolveCfg<T, NP>::DIAG_GLOBAL ? 0 : SolveCfg<T, NP>::STREAM ? 1 : 3;
    U0 = reinterpret_cast<T *>(raw);
    U1 = NB == 3 ? U0 + NP * LDL : nullptr;
    U2 = NB == 3 ? U1 + NP * LDL : nullptr;
    dinv = U0 + NB * NP * LDL;
    y0 = dinv + NP;
    y1 = y0 + NP * m;
    y2 = y1 + NP * m;
    part = y2 + NP * m;  // partial sums of the second half of split products (NP * m)
  }
};

// The products of a solve item split each output's sum between two threads when there are at
// least two threads per output among the first kSolveThreads (one right-hand side and n_p <= 64):
// the second half's partial sum passes through SolveSmem::part and is added after the first half's
// (a fixed order). The condition does not depend on the block size, so the interlaced launch (more
// threads) and the solve launches do the same arithmetic.
__device__ __forceinline__ bool split_outputs(int nm) { return 2 * nm <= kSolveThreads; }

// Issue the copies of an item's factor blocks (they do not depend on other
// items of the solve, so a persistent CTA starts them before it waits for
// the item's inputs). d0: dpool offset or -1; e1/e2: epool offsets, used when
// the matching vector index v1/v2 is >= 0.
template <typename T, int NP>
__device__ __forceinline__ void stage_item_blocks(const SolveSmem<T, NP> &sm, const SolveArgs &a, int64_t d0,
                                                  int64_t v1, int64_t e1, int64_t v2, int64_t e2) {
  const T *dpool = reinterpret_cast<const T *>(a.dpool);
  const T *epool = reinterpret_cast<const T *>(a.epool);
  if (!SolveCfg<T, NP>::DIAG_GLOBAL && d0 >= 0) stage_block<T, NP>(sm.U0, dpool + d0);
  if constexpr (!SolveCfg<T, NP>::STREAM) {
    if (v1 >= 0) stage_block<T, NP>(sm.U1, epool + e1);
    if (v2 >= 0) stage_block<T, NP>(sm.U2, epool + e2);
  }
}

// Forward step for one surviving node j (pull form, Alg. 7 forward sweep):
//   y_j -= U(j-h, j)^T y_{j-h} + U(j+h, j)^T y_{j+h}   (contributions of level l-1)
//   y_j <- U_j^{-T} y_j                                 (if j is eliminated at this level)
// STAGED: the factor blocks were already issued by stage_item_blocks.
template <typename T, int NP, bool STAGED = false>
__device__ __forceinline__ void fwd_node(int64_t y_self, int64_t y_l, int64_t e_l, int64_t y_r, int64_t e_r,
                                         int64_t d_self, const SolveArgs &a, unsigned char *smem_raw) {
  constexpr int LDL = SolveCfg<T, NP>::LDL, LDU = SolveCfg<T, NP>::LDU;
  const int m = a.m;
  const SolveSmem<T, NP> sm(smem_raw, m);
  const T *Us = SolveCfg<T, NP>::DIAG_GLOBAL ? reinterpret_cast<const T *>(a.dpool) + (d_self >= 0 ? d_self : 0)
                                             : sm.U0;
  T *Ul = sm.U1, *Ur = sm.U2, *dinv = sm.dinv, *ys = sm.y0, *yl = sm.y1, *yr = sm.y2;
  T *y = reinterpret_cast<T *>(a.y);
  const int nm = NP * m;
  T *yself = y + y_self * nm;
  if (!STAGED) stage_item_blocks<T, NP>(sm, a, d_self, y_l, e_l, y_r, e_r);
  stage_vec<T>(ys, yself, nm);
  if (y_l >= 0) stage_vec<T>(yl, y + y_l * nm, nm);
  if (y_r >= 0) stage_vec<T>(yr, y + y_r * nm, nm);
  cp_async_wait_all_s();
  __syncthreads();
  if (d_self >= 0)
    for (int j = threadIdx.x; j < NP; j += blockDim.x) dinv[j] = T(1) / Us[j * LDU + j];
  if (y_l >= 0) {
    const bool right = y_r >= 0;
    if constexpr (SolveCfg<T, NP>::STREAM) {  // coupling blocks from global memory, coalesced over c
      const T *gl = reinterpret_cast<const T *>(a.epool) + e_l;
      const T *gr = right ? reinterpret_cast<const T *>(a.epool) + e_r : gl;
      for (int q = threadIdx.x; q < nm; q += blockDim.x) {
        const int c = q / m, col = q % m;
        T acc = ys[q];
#pragma unroll 32
        for (int r = 0; r < NP; ++r) acc = fma(-__ldcg(gl + r * NP + c), yl[r * m + col], acc);
        if (right)
#pragma unroll 32
          for (int r = 0; r < NP; ++r) acc = fma(-__ldcg(gr + r * NP + c), yr[r * m + col], acc);
        ys[q] = acc;
      }
    } else if (split_outputs(nm)) {  // rows 0 .. NP/2-1 and NP/2 .. NP-1 of both blocks on two threads
      const int t = threadIdx.x, q = t % nm, h = t / nm;
      T acc = T(0);
      if (h < 2) {
        const int c = q / m, col = q % m, r0 = h * (NP / 2);
        acc = h == 0 ? ys[q] : T(0);
#pragma unroll 8
        for (int r = r0; r < r0 + NP / 2; ++r) acc = fma(-Ul[r * LDL + c], yl[r * m + col], acc);
        if (right)
#pragma unroll 8
          for (int r = r0; r < r0 + NP / 2; ++r) acc = fma(-Ur[r * LDL + c], yr[r * m + col], acc);
        if (h == 1) sm.part[q] = acc;
      }
      __syncthreads();
      if (h == 0) ys[q] = acc + sm.part[q];
    } else {  // several outputs per thread, OG of them interleaved (each output's sum in the same order)
      constexpr int OG = 4;
      for (int q0 = threadIdx.x; q0 < nm; q0 += OG * blockDim.x) {
        int cq[OG], colq[OG];
        T acc[OG];
#pragma unroll
        for (int k = 0; k < OG; ++k) {
          const int q = min(q0 + k * (int)blockDim.x, nm - 1);
          cq[k] = q / m;
          colq[k] = q % m;
          acc[k] = ys[q];
        }
#pragma unroll 4
        for (int r = 0; r < NP; ++r)
#pragma unroll
          for (int k = 0; k < OG; ++k) acc[k] = fma(-Ul[r * LDL + cq[k]], yl[r * m + colq[k]], acc[k]);
        if (right)
#pragma unroll 4
          for (int r = 0; r < NP; ++r)
#pragma unroll
            for (int k = 0; k < OG; ++k) acc[k] = fma(-Ur[r * LDL + cq[k]], yr[r * m + colq[k]], acc[k]);
#pragma unroll
        for (int k = 0; k < OG; ++k)
          if (q0 + k * (int)blockDim.x < nm) ys[q0 + k * blockDim.x] = acc[k];
      }
    }
  }
  __syncthreads();
  if (d_self >= 0) {
    warp_trsv_ut<T, NP>(ys, m, Us, dinv);
    __syncthreads();
  }
  for (int q = threadIdx.x; q < nm; q += blockDim.x) yself[q] = ys[q];
}

template <typename T, int NP>
__global__ void __launch_bounds__(kSolveThreads) k_fwd_level(SolveArgs a) {
  grid_dep_enter();
  extern __shared__ __align__(16) unsigned char smem_raw[];
  const FwdItem it = reinterpret_cast<const FwdItem *>(a.items)[blockIdx.x];
  fwd_node<T, NP>(it.y_self, it.y_l, it.e_l, it.y_r, it.e_r, it.d_self, a, smem_raw);
}

// Backward step for one eliminated node e (Alg. 7 backward sweep):
//   x_e <- U_e^{-1} (y_e - U(e, e+s) x_{e+s} - U(e, e-s) x_{e-s})
template <typename T, int NP, bool STAGED = false>
__device__ __forceinline__ void bwd_node(int64_t x_self, int64_t x_dn, int64_t e_dn, int64_t x_up, int64_t e_up,
                                         int64_t d_self, const SolveArgs &a, unsigned char *smem_raw) {
  constexpr int LDL = SolveCfg<T, NP>::LDL, LDU = SolveCfg<T, NP>::LDU;
  const int m = a.m;
  const SolveSmem<T, NP> sm(smem_raw, m);
  const T *Us = SolveCfg<T, NP>::DIAG_GLOBAL ? reinterpret_cast<const T *>(a.dpool) + d_self : sm.U0;
  T *Ud = sm.U1, *Uu = sm.U2, *dinv = sm.dinv, *ys = sm.y0, *xd = sm.y1, *xu = sm.y2;
  T *y = reinterpret_cast<T *>(a.y);
  const int nm = NP * m;
  T *yself = y + x_self * nm;
  if (!STAGED) stage_item_blocks<T, NP>(sm, a, d_self, x_dn, e_dn, x_up, e_up);
  stage_vec<T>(ys, yself, nm);
  if (x_dn >= 0) stage_vec<T>(xd, y + x_dn * nm, nm);
  if (x_up >= 0) stage_vec<T>(xu, y + x_up * nm, nm);
  cp_async_wait_all_s();
  __syncthreads();
  for (int j = threadIdx.x; j < NP; j += blockDim.x) dinv[j] = T(1) / Us[j * LDU + j];
  if (x_dn >= 0 || x_up >= 0) {
    const bool dn = x_dn >= 0, up = x_up >= 0;
    if constexpr (SolveCfg<T, NP>::STREAM) {
      // coupling blocks from global memory: one warp per output (row r, column col), lanes
      // split the row (coalesced loads), a shuffle reduction sums the parts
      const T *gd = reinterpret_cast<const T *>(a.epool) + (dn ? e_dn : 0);
      const T *gu = reinterpret_cast<const T *>(a.epool) + (up ? e_up : 0);
      const int lane = threadIdx.x & 31, nw = blockDim.x >> 5;
      for (int q = threadIdx.x >> 5; q < nm && (threadIdx.x >> 5) < nw; q += nw) {
        const int r = q / m, col = q % m;
        T part = T(0);
#pragma unroll
        for (int c = lane; c < NP; c += 32) {
          if (dn) part = fma(__ldcg(gd + r * NP + c), xd[c * m + col], part);
          if (up) part = fma(__ldcg(gu + r * NP + c), xu[c * m + col], part);
        }
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) part += __shfl_xor_sync(0xffffffffu, part, o);
        if (lane == 0) ys[q] -= part;
      }
    } else if (split_outputs(nm)) {  // columns 0 .. NP/2-1 and NP/2 .. NP-1 of both blocks on two threads
      const int t = threadIdx.x, q = t % nm, h = t / nm;
      T acc = T(0);
      if (h < 2) {
        const int r = q / m, col = q % m, c0 = h * (NP / 2);
        acc = h == 0 ? ys[q] : T(0);
        if (dn)
#pragma unroll 8
          for (int c = c0; c < c0 + NP / 2; ++c) acc = fma(-Ud[r * LDL + c], xd[c * m + col], acc);
        if (up)
#pragma unroll 8
          for (int c = c0; c < c0 + NP / 2; ++c) acc = fma(-Uu[r * LDL + c], xu[c * m + col], acc);
        if (h == 1) sm.part[q] = acc;
      }
      __syncthreads();
      if (h == 0) ys[q] = acc + sm.part[q];
    } else {  // several outputs per thread, OG of them interleaved (each output's sum in the same order)
      constexpr int OG = 4;
      for (int q0 = threadIdx.x; q0 < nm; q0 += OG * blockDim.x) {
        int rq[OG], colq[OG];
        T acc[OG];
#pragma unroll
        for (int k = 0; k < OG; ++k) {
          const int q = min(q0 + k * (int)blockDim.x, nm - 1);
          rq[k] = q / m;
          colq[k] = q % m;
          acc[k] = ys[q];
        }
        if (dn)
#pragma unroll 4
          for (int c = 0; c < NP; ++c)
#pragma unroll
            for (int k = 0; k < OG; ++k) acc[k] = fma(-Ud[rq[k] * LDL + c], xd[c * m + colq[k]], acc[k]);
        if (up)
#pragma unroll 4
          for (int c = 0; c < NP; ++c)
#pragma unroll
            for (int k = 0; k < OG; ++k) acc[k] = fma(-Uu[rq[k] * LDL + c], xu[c * m + colq[k]], acc[k]);
#pragma unroll
        for (int k = 0; k < OG; ++k)
          if (q0 + k * (int)blockDim.x < nm) ys[q0 + k * blockDim.x] = acc[k];
      }
    }
  }
  __syncthreads();
  warp_trsv_u<T, NP>(ys, m, Us, dinv);
  __syncthreads();
  for (int q = threadIdx.x; q < nm; q += blockDim.x) yself[q] = ys[q];
}

template <typename T, int NP>
__global__ void __launch_bounds__(kSolveThreads) k_bwd_level(SolveArgs a) {
  grid_dep_enter();
  extern __shared__ __align__(16) unsigned char smem_raw[];
  const BwdItem it = reinterpret_cast<const BwdItem *>(a.items)[blockIdx.x];
  bwd_node<T, NP>(it.x_self, it.x_dn, it.e_dn, it.x_up, it.e_up, it.d_self, a, smem_raw);
}

// Persistent dataflow form of the whole solve (forward items of all levels,
// then backward items top-down) in one launch; each item waits only for the
// items that produce its inputs.
template <typename T, int NP>
__global__ void __launch_bounds__(kSolveThreads) k_solve_flow(SolveArgs a, FlowSync fs) {
  grid_dep_enter();
  extern __shared__ __align__(16) unsigned char smem_raw[];
  __shared__ int s_slot, s_ok;
  const SolveFlowItem *items = reinterpret_cast<const SolveFlowItem *>(a.items);
  for (;;) {
    const int t = flow_claim(fs, a.count, &s_slot);
    if (t < 0) break;
    const SolveFlowItem it = items[t];
    flow_trace(fs, t, 0);
    // the factor blocks load while the item waits for its inputs
    stage_item_blocks<T, NP>(SolveSmem<T, NP>(smem_raw, a.m), a, it.d_self, it.y_a, it.e_a, it.y_b, it.e_b);
    if (flow_wait(fs, it.dep, 3, &s_ok)) {
      flow_trace(fs, t, 1);
      if (it.kind == 0) fwd_node<T, NP, true>(it.y_self, it.y_a, it.e_a, it.y_b, it.e_b, it.d_self, a, smem_raw);
      else bwd_node<T, NP, true>(it.y_self, it.y_a, it.e_a, it.y_b, it.e_b, it.d_self, a, smem_raw);
    } else {
      cp_async_wait_all_s();  // no copy may still target shared memory when the CTA moves on
    }
    __syncthreads();
    flow_trace(fs, t, 2);
    flow_publish(fs, t);
  }
}

// ---------------------------------------------------------------- small systems
// A whole solve (or the tail of an interlaced one) in one CTA for small plans (FP32 factor,
// n_p <= 16, one right-hand side): the items are grouped in waves (an item's dependencies all lie in earlier waves)
// and a CTA barrier separates the waves, instead of one completion flag per item between CTAs. A
// group of n_p lanes takes one item (32 / n_p items per warp); lane c of the group owns output c
// and reads its column (forward) or row (backward) of the blocks straight into registers. An item
// does exactly the arithmetic of fwd_node / bwd_node for this case (the two-halves products, the
// one-chunk triangular solve with z_j = y_j * (1 / U_jj) formed on lane j), so both forms give the
// same bits. The item descriptors and the work vector live in shared memory for the whole launch.
template <typename T, int NP>
struct SmallCfg {
  static_assert(NP == 8 || NP == 16 || NP == 32, "lane groups of n_p lanes (n_p = 32: one item per warp)");
  static_assert(2 * NP <= kSolveThreads, "one chunk, two threads per output in fwd_node");
  static constexpr int G = 32 / NP;  // items per warp
  // register budget: a lane holds a row or column of the diagonal block and one of each coupling block
  static constexpr int MAXT = (int)sizeof(T) * NP <= 32 ? 1024 : (int)sizeof(T) * NP <= 128 ? 512 : 256;
};

template <typename T, int V>
__device__ __forceinline__ void small_vload(const T *p, T *dst) {
  T w[V];
  vload<T, V>(p, w);
#pragma unroll
  for (int t = 0; t < V; ++t) dst[t] = w[t];
}

// Forward step (kind 0) for the lanes with act set; every lane of the warp runs the substitution's
// shuffles. y: the work vector in shared memory.
template <typename T, int NP>
__device__ __forceinline__ void group_fwd_item(const SolveFlowItem &it, bool act, const SolveArgs &a, T *y) {
  const int c = threadIdx.x & (NP - 1);
  const T *dpool = reinterpret_cast<const T *>(a.dpool);
  const T *epool = reinterpret_cast<const T *>(a.epool);
  T *ys = y + it.y_self * NP;
  const bool diag = act && it.d_self >= 0;
  T u[NP], dl = T(0);  // column c of U_j (u[k] = U_j(k, c)) and 1 / U_j(c, c)
  if (diag) {
    const T *U = dpool + it.d_self;
#pragma unroll
    for (int k = 0; k < NP; ++k) u[k] = U[k * NP + c];
    dl = T(1) / U[c * NP + c];
  }
  T v = act ? ys[c] : T(0);
  if (act && it.y_a >= 0) {
    const bool right = it.y_b >= 0;
    const T *ya = y + it.y_a * NP, *Ua = epool + it.e_a;
    const T *yb = right ? y + it.y_b * NP : ya, *Ub = right ? epool + it.e_b : Ua;
    T acc0 = v, acc1 = T(0);
#pragma unroll
    for (int r = 0; r < NP / 2; ++r) acc0 = fma(-Ua[r * NP + c], ya[r], acc0);
    if (right)
#pragma unroll
      for (int r = 0; r < NP / 2; ++r) acc0 = fma(-Ub[r * NP + c], yb[r], acc0);
#pragma unroll
    for (int r = NP / 2; r < NP; ++r) acc1 = fma(-Ua[r * NP + c], ya[r], acc1);
    if (right)
#pragma unroll
      for (int r = NP / 2; r < NP; ++r) acc1 = fma(-Ub[r * NP + c], yb[r], acc1);
    v = acc0 + acc1;
  }
  if (__any_sync(0xffffffffu, diag)) {  // y_j <- U_j^{-T} y_j
#pragma unroll
    for (int j = 0; j < NP; ++j) {
      const T zj = __shfl_sync(0xffffffffu, v * dl, j, NP);
      if (diag && c > j) v = fma(-u[j], zj, v);
      if (diag && c == j) v = zj;
    }
  }
  if (act) ys[c] = v;
}

// Backward step (kind 1) for the lanes with act set.
template <typename T, int NP>
__device__ __forceinline__ void group_bwd_item(const SolveFlowItem &it, bool act, const SolveArgs &a, T *y) {
  constexpr int V = 16 / (int)sizeof(T) < NP ? 16 / (int)sizeof(T) : NP;
  constexpr int HV = NP / 2 >= V ? V : NP / 2;
  const int c = threadIdx.x & (NP - 1);
  const T *dpool = reinterpret_cast<const T *>(a.dpool);
  const T *epool = reinterpret_cast<const T *>(a.epool);
  T *ys = y + it.y_self * NP;
  const T *U = dpool + it.d_self;
  T u[NP], dl = T(0), v = T(0);  // row c of U_e, 1 / U_e(c, c)
  if (act) {
#pragma unroll
    for (int k = 0; k < NP; k += V) small_vload<T, V>(U + c * NP + k, u + k);
    dl = T(1) / U[c * NP + c];
    v = ys[c];
  }
  const bool dn = act && it.y_a >= 0, up = act && it.y_b >= 0;
  if (dn || up) {
    const T *xd = dn ? y + it.y_a * NP : ys, *Ud = dn ? epool + it.e_a : U;
    const T *xu = up ? y + it.y_b * NP : ys, *Uu = up ? epool + it.e_b : U;
    T acc[2] = {v, T(0)};
#pragma unroll
    for (int h = 0; h < 2; ++h) {  // columns h * NP/2 .. of both blocks into acc[h]
      T wd[NP / 2], wu[NP / 2];
#pragma unroll
      for (int k = 0; k < NP / 2; k += HV) {
        small_vload<T, HV>(Ud + c * NP + h * (NP / 2) + k, wd + k);
        small_vload<T, HV>(Uu + c * NP + h * (NP / 2) + k, wu + k);
      }
      if (dn)
#pragma unroll
        for (int k = 0; k < NP / 2; ++k) acc[h] = fma(-wd[k], xd[h * (NP / 2) + k], acc[h]);
      if (up)
#pragma unroll
        for (int k = 0; k < NP / 2; ++k) acc[h] = fma(-wu[k], xu[h * (NP / 2) + k], acc[h]);
    }
    v = acc[0] + acc[1];
  }
#pragma unroll
  for (int j = NP - 1; j >= 0; --j) {  // x_e <- U_e^{-1} (...)
    const T xj = __shfl_sync(0xffffffffu, v * dl, j, NP);
    if (act && c < j) v = fma(-u[j], xj, v);
    if (act && c == j) v = xj;
  }
  if (act) ys[c] = v;
}

// order: the items of a.items grouped by wave; wave_off: nwaves + 1 offsets into order; ycount: the
// work-vector nodes the items touch. The item descriptors (in wave order), those nodes of the
// work vector and the wave offsets are staged in shared memory for the whole launch, so a wave
// reads only the factor blocks from global memory; the vector is written back at the end.
template <typename T, int NP>
__global__ void __launch_bounds__(SmallCfg<T, NP>::MAXT) k_solve_small(SolveArgs a, const int32_t *order,
                                                                     const int32_t *wave_off, int nwaves,
                                                                     int ycount) {
  grid_dep_enter();
  constexpr int G = SmallCfg<T, NP>::G;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  SolveFlowItem *sit = reinterpret_cast<SolveFlowItem *>(smem_raw);
  T *sy = reinterpret_cast<T *>(sit + a.count);
  int *soff = reinterpret_cast<int *>(sy + ycount * NP);
  const SolveFlowItem *items = reinterpret_cast<const SolveFlowItem *>(a.items);
  T *y = reinterpret_cast<T *>(a.y);
  for (int q = threadIdx.x; q < a.count; q += blockDim.x) sit[q] = items[order[q]];
  for (int q = threadIdx.x; q < ycount * NP; q += blockDim.x) sy[q] = y[q];
  for (int q = threadIdx.x; q <= nwaves; q += blockDim.x) soff[q] = wave_off[q];
  __syncthreads();
  const int warp = threadIdx.x >> 5, nw = blockDim.x >> 5, grp = (threadIdx.x & 31) / NP;
  for (int w = 0; w < nwaves; ++w) {
    const int t1 = soff[w + 1];
    for (int t0 = soff[w] + warp * G; t0 < t1; t0 += nw * G) {  // warp-uniform loop
      const int t = t0 + grp;
      const SolveFlowItem it = sit[t < t1 ? t : t0];
      const bool fwd = t < t1 && it.kind == 0, bwd = t < t1 && it.kind != 0;
      if (__any_sync(0xffffffffu, fwd)) group_fwd_item<T, NP>(it, fwd, a, sy);
      if (__any_sync(0xffffffffu, bwd)) group_bwd_item<T, NP>(it, bwd, a, sy);
    }
    __syncthreads();
  }
  for (int q = threadIdx.x; q < ycount * NP; q += blockDim.x) y[q] = sy[q];
}

// Shared memory of k_solve_small.
inline size_t small_solve_smem(int count, int ycount, int nwaves, int np, size_t elem) {
  return (size_t)count * sizeof(SolveFlowItem) + (size_t)ycount * np * elem + sizeof(int) * ((size_t)nwaves + 1);
}

// Typed launch of k_solve_small (one CTA of `threads` threads, a multiple of 32).
template <typename T, int NP>
int launch_solve_small(const void *items, int count, const void *dpool, const void *epool, void *y,
                       const int32_t *order, const int32_t *wave_off, int nwaves, int ycount, int threads,
                       cudaStream_t s) {
  if (count <= 0) return BTC_OK;
  SolveArgs a;
  a.items = items;
  a.count = count;
  a.dpool = dpool;
  a.epool = epool;
  a.y = y;
  a.m = 1;
  threads = threads < SmallCfg<T, NP>::MAXT ? threads : SmallCfg<T, NP>::MAXT;
  k_solve_small<T, NP><<<1, threads, small_solve_smem(count, ycount, nwaves, NP, sizeof(T)), s>>>(
      a, order, wave_off, nwaves, ycount);
  const cudaError_t e = cudaGetLastError();
  return e == cudaSuccess ? BTC_OK : fail(BTC_ERR_CUDA, "small solve launch: %s", cudaGetErrorString(e));
}

template <typename T, int NP>
constexpr size_t fwd_smem_bytes(int m) {
  constexpr size_t nb = SolveCfg<T, NP>::DIAG_GLOBAL ? 0 : SolveCfg<T, NP>::STREAM ? 1 : 3;
  return sizeof(T) * (nb * NP * SolveCfg<T, NP>::LDL + NP + 4 * (size_t)NP * m);
}
template <typename T, int NP>
constexpr size_t bwd_smem_bytes(int m) {
  return fwd_smem_bytes<T, NP>(m);
}

// ---------------------------------------------------------------- vectors
// Columns [col0, col0+m) of the user array b [N*n][ldb] (type S) -> y [N][np][m]
// (type T), zero padding.
template <typename T, typename S>
__global__ void k_pack_rhs(T *y, const S *b, int N, int n, int np, int m, int ldb, int col0, int64_t node_base) {
  grid_dep_enter();
  const int64_t total = (int64_t)N * np * m;
  for (int64_t q = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; q < total; q += (int64_t)gridDim.x * blockDim.x) {
    const int64_t i = q / ((int64_t)np * m);
    const int r = (int)((q / m) % np), c = (int)(q % m);
    y[node_base * np * m + q] = r < n ? convert_in<T, S>(b[(i * n + r) * ldb + col0 + c]) : T(0);
  }
}

// y -> columns [col0, col0+m) of the user array x [N*n][ldx]; if accumulate:
// x += y (the FP64 update of the refinement).
template <typename T, typename S>
__global__ void k_unpack(S *x, const T *y, int N, int n, int np, int m, int ldx, int col0, int64_t node_base,
                         int accumulate) {
  grid_dep_enter();
  const int64_t total = (int64_t)N * n * m;
  for (int64_t q = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; q < total; q += (int64_t)gridDim.x * blockDim.x) {
    const int64_t i = q / ((int64_t)n * m);
    const int r = (int)((q / m) % n), c = (int)(q % m);
    const S v = (S)y[node_base * np * m + (i * np + r) * m + c];
    S *dst = x + (i * n + r) * ldx + col0 + c;
    *dst = accumulate ? *dst + v : v;
  }
}

// max(a, b) that propagates NaN (fmax drops it): a NaN entry of r or x must
// reach the host, where it stops the refinement instead of vanishing from the
// norms.
__device__ __forceinline__ double nan_max(double a, double b) { return (b > a || b != b) ? b : a; }
__device__ __forceinline__ float nan_maxf(float a, float b) { return (b > a || b != b) ? b : a; }

// Non-negative doubles order like their bit patterns; a NaN with the sign bit
// clear (fabs of any NaN) orders above +inf, so it wins the maximum.
__device__ __forceinline__ void atomic_max_nonneg(double *addr, double v) {
  atomicMax(reinterpret_cast<unsigned long long *>(addr), (unsigned long long)__double_as_longlong(v));
}

// |a| rounded toward zero to FP32 from the high word of the double with 32-bit
// integer operations only (FP64 conversions, and a sign-bit clear on the
// 64-bit value, run on the slow FP64 pipe of this GPU): keep the exponent and
// the top 20 mantissa bits. Magnitudes below the FP32 normal range give 0 and
// above it FLT_MAX, both lower bounds of |a|.
__device__ __forceinline__ float abs_lower_f32(double a) {
  const int hi = __double2hiint(a) & 0x7fffffff;
  const int e = (hi >> 20) - 1023 + 127;
  if (e <= 0) return 0.0f;
  if (e >= 255) return 3.402823466e38f;
  return __int_as_float((e << 23) | ((hi & 0xfffff) << 3));
}

// r = b - Psi x in FP64 for one block row per CTA; writes r (converted to T)
// into the padded work vector y when y != nullptr, and max|r|, max|x| into
// norms[0], norms[1]. D: lower triangles read. Each output's 3n-term dot
// product is split into kResParts interleaved column sets, each with one
// FP64 chain per block (D_i, B_{i-1}, B_i^T terms, interleaved so three
// multiply-adds are in flight per thread), added in a fixed order
// (deterministic). Matrix entries are read straight from global memory (each
// block's rows stay in L1 across the partial sums); x_{i-1}, x_i, x_{i+1} are
// staged in shared memory. with_anorm != 0: the same pass also forms a lower
// bound of ||Psi||_inf into norms[2] (each |a_ij| truncated to FP32, row sums
// with round-toward-zero additions, so the stopping test
// ||r|| <= tol ||Psi|| ||x|| is never met early). Dynamic shared memory:
// residual_smem_bytes(n, m). Grid: residual_grid(N, m) CTAs, each one block row and one group of
// residual_cols(m) right-hand sides (mg).
constexpr int kResParts = 4;
constexpr int kResThreads = 256;

template <typename T>
__global__ void __launch_bounds__(kResThreads) k_residual(T *y, const double *D, const double *B, const double *x,
                                                          const double *b, int N, int n, int np, int m,
                                                          int64_t node_base, double *norms, int with_anorm, int mg) {
  grid_dep_enter();
  extern __shared__ __align__(16) unsigned char smem_raw[];
  // CTA: block row i, columns cb .. cb + mc - 1 of the m right-hand sides (mg per CTA)
  const int ng = (m + mg - 1) / mg;
  const int i = blockIdx.x / ng, cb = (blockIdx.x % ng) * mg;
  const int mc = min(mg, m - cb);
  const int nm = n * mc;
  double *xs = reinterpret_cast<double *>(smem_raw);  // [3][n*mc]: x_{i-1}, x_i, x_{i+1}
  double *ps = xs + 3 * nm;                            // [kResParts][n*mc]
  float *as = reinterpret_cast<float *>(ps + kResParts * nm);  // [kResParts][n] row-sum parts
  const size_t bs = (size_t)n * n;
  for (int q = threadIdx.x; q < 3 * nm; q += blockDim.x) {
    const int which = q / nm, off = q % nm, row = i - 1 + which;
    xs[q] = (row >= 0 && row < N) ? x[((size_t)row * n + off / mc) * m + cb + off % mc] : 0.0;
  }
  __syncthreads();
  const double *Di = D + i * bs;
  const double *Bl = i > 0 ? B + (i - 1) * bs : D;  // a valid address when the block is absent
  const double *Br = i + 1 < N ? B + i * bs : D;
  const bool has_l = i > 0, has_u = i + 1 < N;
  const double *x0 = xs, *x1 = xs + nm, *x2 = xs + 2 * nm;
  for (int idx = threadIdx.x; idx < kResParts * nm; idx += blockDim.x) {
    // part fastest: the kResParts threads of an output are neighbours and part p sums the columns
    // c = p, p + kResParts, ..., so a row-major read of the warp touches consecutive columns
    const int part = idx % kResParts, q = idx / kResParts;
    const int r = q / mc, cc = q % mc, col = cb + cc;
    const bool lb = with_anorm && col == 0;
    double vd = 0.0, vl = 0.0, vu = 0.0;
    float s = 0.0f;
#pragma unroll 4
    for (int c = part; c < n; c += kResParts) {
      const double ad = __ldg(r >= c ? Di + r * n + c : Di + c * n + r);
      const double al = has_l ? __ldg(Bl + r * n + c) : 0.0;
      const double au = has_u ? __ldg(Br + c * n + r) : 0.0;
      vd = fma(ad, x1[c * mc + cc], vd);
      vl = fma(al, x0[c * mc + cc], vl);
      vu = fma(au, x2[c * mc + cc], vu);
      if (lb) s = __fadd_rz(__fadd_rz(__fadd_rz(s, abs_lower_f32(ad)), abs_lower_f32(al)), abs_lower_f32(au));
    }
    ps[part * nm + q] = (vd + vl) + vu;
    if (lb) as[part * n + r] = s;
  }
  __syncthreads();
  double rmax = 0.0, xmax = 0.0;
  float amax = 0.0f;
  for (int q = threadIdx.x; q < nm; q += blockDim.x) {
    double ax = 0.0;
#pragma unroll
    for (int k = 0; k < kResParts; ++k) ax += ps[k * nm + q];
    const int r = q / mc, col = cb + q % mc;
    const double v = b[((size_t)i * n + r) * m + col] - ax;
    if (y) y[(node_base + i) * np * m + r * m + col] = convert_in<T, double>(v);
    rmax = nan_max(rmax, fabs(v));
    xmax = nan_max(xmax, fabs(xs[nm + q]));
    if (with_anorm && col == 0) {
      float rs = 0.0f;
#pragma unroll
      for (int k = 0; k < kResParts; ++k) rs = __fadd_rz(rs, as[k * n + r]);
      amax = nan_maxf(amax, rs);
    }
  }
  if (y) {
    for (int q = threadIdx.x; q < (np - n) * mc; q += blockDim.x)
      y[(node_base + i) * np * m + (n + q / mc) * m + cb + q % mc] = T(0);
  }
  for (int o = 16; o > 0; o >>= 1) {
    rmax = nan_max(rmax, __shfl_xor_sync(0xffffffffu, rmax, o));
    xmax = nan_max(xmax, __shfl_xor_sync(0xffffffffu, xmax, o));
    amax = nan_maxf(amax, __shfl_xor_sync(0xffffffffu, amax, o));
  }
  if ((threadIdx.x & 31) == 0) {
    atomic_max_nonneg(norms + 0, rmax);
    atomic_max_nonneg(norms + 1, xmax);
    if (with_anorm) atomic_max_nonneg(norms + 2, (double)amax);
  }
}

// Columns per CTA of k_residual for m right-hand sides: up to 4 in one CTA, else groups of 8 (about two
// waves of resident CTAs at N=1024, n=64, m=16 instead of 2.25 waves of three per SM).
inline int residual_cols(int m) { return m <= 4 ? m : 8; }
inline int residual_grid(int N, int m) { return N * ((m + residual_cols(m) - 1) / residual_cols(m)); }

// Dynamic shared memory of k_residual for m right-hand sides (its column group).
inline size_t residual_smem_bytes(int n, int m) {
  const int mc = residual_cols(m) < m ? residual_cols(m) : m;
  return sizeof(double) * (size_t)(3 + kResParts) * n * mc + sizeof(float) * (size_t)kResParts * n;
}

// Typed launch of k_residual over N block rows and m right-hand sides (argument types checked at
// compile time; the dynamic shared memory attribute must allow residual_smem_bytes(n, m)).
template <typename T>
static int launch_residual(void *y, const double *D, const double *B, const double *x, const double *b, int N, int n,
                    int np, int m, int64_t node_base, double *norms, int with_anorm, cudaStream_t s) {
  if (N <= 0) return BTC_OK;
  T *yt = static_cast<T *>(y);
  int mg = residual_cols(m);
  // the argument list of k_residual, in order and with its parameter types
  void *args[] = {&yt, &D, &B, &x, &b, &N, &n, &np, &m, &node_base, &norms, &with_anorm, &mg};
  static_assert(sizeof(args) / sizeof(args[0]) == 13, "one entry per parameter of k_residual");
  BTC_CUDA(launch_ex((const void *)&k_residual<T>, dim3(residual_grid(N, m)), dim3(kResThreads), args,
                     residual_smem_bytes(n, m), s));
  return BTC_OK;
}


}  // namespace btc
