// Interlaced factorization and forward substitution: one persistent launch
// runs the factor items of Alg. 5 and the forward items of Alg. 7, the forward
// item of node j at level l as soon as the factor items that write the blocks
// it reads (U_j at level l, U(j-h, j) and U(j+h, j) at level l-1) and the
// forward items that finish its inputs are done. The paper overlaps the
// forward substitution with the factorization in the same way (Sec. 5, the
// interlaced kernel traces).
#pragma once
#include "btc_factor.cuh"
#include "btc_solve.cuh"

namespace btc {

template <typename T, int NP, int R>
size_t fused_smem_bytes(int m) {
  const size_t f = factor_smem_bytes<T, NP, R>(), s = fwd_smem_bytes<T, NP>(m);
  return f > s ? f : s;
}

// code[t] >= 0: factor item code[t] of fa.items (level 1 when < nfirst);
// code[t] < 0: forward item -code[t]-1 of sa.items. kInterDeps dependencies
// per entry.
template <typename T, typename P, typename S, int NP, int R, int MINB>
__global__ void __launch_bounds__(TileCfg<T, NP, R>::NT, MINB)
    k_factor_fwd_flow(FactorArgs fa, InstDesc single, SolveArgs sa, const int32_t *code, const int32_t *deps,
                      int nfirst, int count, FlowSync fs) {
  grid_dep_enter();
  extern __shared__ __align__(16) unsigned char smem_raw[];
  __shared__ int s_slot, s_ok;
  const SolveFlowItem *fwd = reinterpret_cast<const SolveFlowItem *>(sa.items);
  for (;;) {
    const int t = flow_claim(fs, count, &s_slot);
    if (t < 0) break;
    const int c = code[t];
    flow_trace(fs, t, 0);
    // a factor entry first waits for its dependencies' factor blocks (factor_node waits for the rest)
    if (flow_wait(fs, deps + (size_t)kInterDeps * t, kInterDeps, &s_ok, c >= 0 ? kWaitCoreOnly : kWaitAll)) {
      flow_trace(fs, t, 1);
      if (c >= 0) {
        const FactorItem it = fa.items[c];
        const FlowCtl fc{&fs, deps + (size_t)kInterDeps * t, kInterDeps, t, &s_ok};
        if (c < nfirst) factor_node<T, P, S, NP, R, true>(it, fa, single, smem_raw, &fc);
        else factor_node<T, P, S, NP, R, false>(it, fa, single, smem_raw, &fc);
      } else {
        const SolveFlowItem it = fwd[-1 - c];
        fwd_node<T, NP>(it.y_self, it.y_a, it.e_a, it.y_b, it.e_b, it.d_self, sa, smem_raw);
      }
    }
    __syncthreads();
    flow_trace(fs, t, 2);
    flow_publish(fs, t);
  }
}

}  // namespace btc
