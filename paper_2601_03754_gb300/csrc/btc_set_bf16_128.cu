// Kernel set: FP64 inputs, FP32 factor with the level-elimination products on
// tcgen05 (BF16 operands, FP32 accumulation), FP32 correction solves, FP64 (or
// double-FP32) top-separator Cholesky; padded block size 128.
#include "btc_make.cuh"
#include "btc_tc.cuh"

namespace btc {
// Mixed BF16 set for block size 128: the mixed FP32 set with the level
// elimination (per-level, persistent and interlaced forms) replaced by its
// tcgen05 form with BF16 operands; the right-looking variant keeps the FP32
// FMA kernels.
KernelSet make_set_bf16_128() {
  KernelSet k = make_set<float, double, kTcNP, true>();
  k.fac_first = (const void *)&k_factor_level_tc<double, true, 2>;
  k.fac_rest = (const void *)&k_factor_level_tc<double, false, 2>;
  k.n_flow_v = 1;
  k.flow_default = 0;
  FlowVariant &v = k.flow_v[0];
  v.minb = 1;
  v.fac = (const void *)&k_factor_flow_tc<double, 2>;
  v.fac_fwd = (const void *)&k_factor_fwd_flow_tc<double, 2>;
  k.fac_flow = v.fac;
  k.fac_fwd_flow = v.fac_fwd;
  k.fac_flow_rl = v.fac_rl;
  k.tensor_cores = true;
  return k;
}

}  // namespace btc
