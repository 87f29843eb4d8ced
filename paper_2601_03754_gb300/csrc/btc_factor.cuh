// Level-elimination kernel: one CTA per eliminated node of one dissection
// level (Alg. 5, one iteration of its parallel loop). The whole elimination of
// the node is fused in one CTA, with the node's blocks held in registers and
// shared memory:
//   Dhat_e  -= P_a^T P_a                         deferred syrk (level > 1)
//   Dhat_e   = chol(Dhat_e)                       potrf
//   U(e,e-s) = Dhat_e^{-1} S(e,e-s)               trsm (up)
//   U(e,e+s) = Dhat_e^{-1} S(e,e+s)               trsm (down)
//   Dhat_{e+s} -= P_b^T P_b + U(e,e+s)^T U(e,e+s) deferred + immediate syrk
//   S'(e-s,e+s) or S'(e+s,e-s) = -U^T U           fill gemm for level l+1
// Level 1 reads the caller's D and B directly (with conversion and padding),
// so no separate packing pass is needed.
#pragma once
#include "btc_internal.h"
#include "btc_tile.cuh"

namespace btc {

struct InstDesc {
  const void *D;  // user D [N][n][n] (source type)
  const void *B;  // user B [N-1][n][n]
  int N, n;
};

struct FactorArgs {
  const FactorItem *items;
  int count;
  void *dpool;
  void *epool;
  const InstDesc *inst;      // per-instance descriptors (batched); NULL: use the by-value one
  unsigned long long *info;  // one word per instance
};

template <typename T, int NP, int R>
constexpr size_t factor_smem_bytes() {
  using C = TileCfg<T, NP, R>;
  return sizeof(T) * (3 * C::BLK + 3 * C::NP);
}

// T: arithmetic type; P: element type of the pools; S: element type of the
// caller's D and B (read at level 1 only). The FP64 top-separator Cholesky of
// the mixed-precision path is the instantiation T = double, P = float.
template <typename T, typename P, typename S, int NP, int R, bool FIRST>
__global__ void __launch_bounds__(TileCfg<T, NP, R>::NT) k_factor_level(FactorArgs args, InstDesc single) {
  using C = TileCfg<T, NP, R>;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  T *sA = reinterpret_cast<T *>(smem_raw);  // staging: P_a, then U(e,e-s)
  T *sB = sA + C::BLK;                      // L^T of Dhat_e, then P_b
  T *sC = sB + C::BLK;                      // U(e,e+s)
  T *cbuf = sC + C::BLK;                    // 2 * NP publish buffers
  T *dinv = cbuf + 2 * NP;                  // NP

  const FactorItem it = args.items[blockIdx.x];
  P *dpool = reinterpret_cast<P *>(args.dpool);
  P *epool = reinterpret_cast<P *>(args.epool);
  const int tid = threadIdx.x;
  const int ty = tid / C::TXN, tx = tid % C::TXN;
  const int r0 = ty * R, c0 = tx * R;
  const bool lower = ty >= tx;
  unsigned long long *info = args.info + it.inst;
  const InstDesc ins = args.inst ? args.inst[it.inst] : single;
  const int e = it.node;
  const S *uD = reinterpret_cast<const S *>(ins.D);
  const S *uB = reinterpret_cast<const S *>(ins.B);
  const size_t ubs = (size_t)ins.n * ins.n;

  T a[R][R];
  // ---- Dhat_e (with the deferred update of level l-1)
  if constexpr (FIRST) {
    tile_from_user<C>(a, uD + e * ubs, ins.n, r0, c0, false, T(1));
  } else {
    tile_from_pool<C>(a, dpool + it.d_self, r0, c0);
    if (it.p_a >= 0) {
      block_to_smem<C>(sA, epool + it.p_a);
      __syncthreads();
      if (lower) tile_sub_xty<C>(a, sA, sA, r0, c0);
    }
  }
  // ---- potrf
  tile_potrf<C>(a, r0, c0, lower, cbuf, sB, dinv, info, e);
  tile_to_pool<C>(dpool + it.d_self, a, r0, c0);
  __syncthreads();  // L^T and dinv visible; sA free

  // ---- trsm up: U(e, e-s) = Dhat_e^{-1} S(e, e-s)
  const bool has_up = it.r_up >= 0, has_dn = it.r_down >= 0;
  if (has_up) {
    T z[R][R];
    if constexpr (FIRST) tile_from_user<C>(z, uB + (e - 1) * ubs, ins.n, r0, c0, false, T(0));
    else tile_from_pool<C>(z, epool + it.r_up, r0, c0);
    tile_trsm_llnn<C>(z, r0, c0, sB, dinv, cbuf);
    tile_to_pool<C>(epool + it.r_up, z, r0, c0);
    tile_to_smem<C>(sA, z, r0, c0);
  }
  // ---- trsm down: U(e, e+s) = Dhat_e^{-1} S(e, e+s); level 1: S(e, e+1) = B_e^T
  if (has_dn) {
    T z[R][R];
    if constexpr (FIRST) tile_from_user<C>(z, uB + e * ubs, ins.n, r0, c0, true, T(0));
    else tile_from_pool<C>(z, epool + it.r_down, r0, c0);
    tile_trsm_llnn<C>(z, r0, c0, sB, dinv, cbuf);
    tile_to_pool<C>(epool + it.r_down, z, r0, c0);
    tile_to_smem<C>(sC, z, r0, c0);
  }
  __syncthreads();  // sA/sC hold U blocks; sB (L^T) free

  // ---- Dhat_{e+s} -= P_b^T P_b + U_dn^T U_dn
  if (it.d_next >= 0) {
    T d[R][R];
    if constexpr (FIRST) {
      tile_from_user<C>(d, uD + (e + 1) * ubs, ins.n, r0, c0, false, T(1));
    } else {
      tile_from_pool<C>(d, dpool + it.d_next, r0, c0);
      if (it.p_b >= 0) {
        block_to_smem<C>(sB, epool + it.p_b);
        __syncthreads();
        if (lower) tile_sub_xty<C>(d, sB, sB, r0, c0);
      }
    }
    if (lower) {
      tile_sub_xty<C>(d, sC, sC, r0, c0);
      tile_to_pool<C>(dpool + it.d_next, d, r0, c0);
    }
  }
  // ---- fill for level l+1
  if (it.fill >= 0) {
    T f[R][R];
#pragma unroll
    for (int r = 0; r < R; ++r)
#pragma unroll
      for (int c = 0; c < R; ++c) f[r][c] = T(0);
    if (it.flags & FI_FILL_UPFIRST) tile_sub_xty<C>(f, sA, sC, r0, c0);  // S'(e-s, e+s) = -U_up^T U_dn
    else tile_sub_xty<C>(f, sC, sA, r0, c0);                             // S'(e+s, e-s) = -U_dn^T U_up
    tile_to_pool<C>(epool + it.fill, f, r0, c0);
  }
}

}  // namespace btc
