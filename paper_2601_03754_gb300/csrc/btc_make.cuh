// Builds the KernelSet of one (arithmetic, pool, source, np) instantiation.
#pragma once
#include "btc_factor.cuh"
#include "btc_fused.cuh"
#include "btc_kernels.h"
#include "btc_solve.cuh"

namespace btc {

// Register tile edge per padded block size: (np/R)^2 threads per CTA. FP64 at n_p = 16 takes R = 1
// (256 threads): a warp's FP64 instruction occupies its SM sub-partition's FP64 pipe for the same
// time whatever its active lanes, so the node's products need warps on all four sub-partitions.
template <typename T, int NP>
struct TileEdge {
  static constexpr int R =
      NP == 8 ? 1 : NP == 16 ? (sizeof(T) == 8 ? 1 : 2) : NP == 32 ? 2 : NP == 128 ? 8 : 4;  // 96 -> 576 threads
};

template <typename T, int NP>
size_t fwd_smem_fn(int m) { return fwd_smem_bytes<T, NP>(m); }
template <typename T, int NP>
size_t bwd_smem_fn(int m) { return bwd_smem_bytes<T, NP>(m); }
template <typename T, int NP, int R>
size_t fused_smem_fn(int m) { return fused_smem_bytes<T, NP, R>(m); }
inline size_t zero_smem_fn(int) { return 0; }

// Residency variants of the persistent factor kernels: caps 1, 2, 3, 4 CTAs per
// SM (1, 2, 4, 8, 16 for 64-thread CTAs: many small nodes resident on one SM),
// those that shared memory and threads allow.
template <typename T, typename S, int NP, int R, int MINB>
void add_flow_variant(KernelSet &k) {
  if constexpr (MINB == 1 || MINB <= FlowFit<T, NP, R>::value) {
    FlowVariant &v = k.flow_v[k.n_flow_v++];
    v.minb = MINB;
    v.fac = (const void *)&k_factor_flow<T, T, S, NP, R, MINB>;
    v.fac_fwd = (const void *)&k_factor_fwd_flow<T, T, S, NP, R, MINB>;
    v.fac_rl = (const void *)&k_factor_flow_rl<T, T, S, NP, R, MINB>;
  }
}

template <typename T, typename S, int NP, bool MIXED>
KernelSet make_set() {
  constexpr int R = TileEdge<T, NP>::R;
  KernelSet k;
  k.valid = true;
  k.np = NP;
  k.elem = sizeof(T);
  k.src_elem = sizeof(S);
  k.fac_first = (const void *)&k_factor_level<T, T, S, NP, R, true>;
  k.fac_rest = (const void *)&k_factor_level<T, T, S, NP, R, false>;
  k.fac_threads = TileCfg<T, NP, R>::NT;
  k.fac_smem = factor_smem_bytes<T, NP, R>();
  if constexpr (MIXED) {
    k.root_first = (const void *)&k_root_chol<T, S, NP, R, true, false>;
    k.root_rest = (const void *)&k_root_chol<T, S, NP, R, false, false>;
    k.root_rl = (const void *)&k_root_chol<T, S, NP, R, false, true>;
    k.root64_first = (const void *)&k_root_chol_f64<T, S, NP, R, true, false>;
    k.root64_rest = (const void *)&k_root_chol_f64<T, S, NP, R, false, false>;
    k.root64_rl = (const void *)&k_root_chol_f64<T, S, NP, R, false, true>;
    k.root_threads = TileCfg<float, NP, R>::NT;
    k.root_smem = root_smem_bytes<NP, R>();
  }
  constexpr bool small = TileCfg<T, NP, R>::NT <= 64;
  add_flow_variant<T, S, NP, R, 1>(k);
  add_flow_variant<T, S, NP, R, 2>(k);
  add_flow_variant<T, S, NP, R, small ? 4 : 3>(k);
  add_flow_variant<T, S, NP, R, small ? 8 : 4>(k);
  if constexpr (small) add_flow_variant<T, S, NP, R, 16>(k);
  // default without tuning: two resident CTAs where they fit (more registers per
  // thread than the maximum residency; measured best at N = 1024, n = 64)
  k.flow_default = k.n_flow_v > 1 ? 1 : 0;
  k.fac_flow = k.flow_v[k.flow_default].fac;
  k.fac_fwd_flow = k.flow_v[k.flow_default].fac_fwd;
  k.fac_flow_rl = k.flow_v[k.flow_default].fac_rl;
  k.fused_smem = &fused_smem_fn<T, NP, R>;
  k.pack_pools = &launch_pack<T, S, NP>;
  k.pack_batch = &launch_pack_batch<T, S, NP>;
  k.fac_rl = (const void *)&k_factor_level<T, T, S, NP, R, false, true>;
  k.solve_flow = (const void *)&k_solve_flow<T, NP>;
  // FP32 and n_p <= 16 only: an FP64 solve confined to one SM is bound by that SM's FP64 rate, and at
  // n_p = 32 the longer chains of a lane-per-output item lose to the dataflow kernel's CTA per item
  if constexpr (NP <= 16 && sizeof(T) == 4) k.solve_small = &launch_solve_small<T, NP>;
  k.fwd = (const void *)&k_fwd_level<T, NP>;
  k.bwd = (const void *)&k_bwd_level<T, NP>;
  k.fwd_smem = &fwd_smem_fn<T, NP>;
  k.max_cols = 16;
  while (k.max_cols > 1 && fwd_smem_bytes<T, NP>(k.max_cols) > 232448 - 64) --k.max_cols;
  k.bwd_smem = &bwd_smem_fn<T, NP>;
  k.pack = (const void *)&k_pack_rhs<T, S>;
  k.unpack = (const void *)&k_unpack<T, S>;
  k.resid = (const void *)&k_residual<T>;
  k.residual = &launch_residual<T>;
  return k;
}

}  // namespace btc
