// Kernel table: the compiled instantiations for one (dtype, np) pair, filled
// by the per-dtype translation units and launched by the runtime.
#pragma once
#include <cuda_runtime.h>
#include <stddef.h>
#include <stdint.h>

namespace btc {

struct KernelSet {
  bool valid = false;
  int np = 0;
  size_t elem = 0;        // bytes per pool element
  size_t src_elem = 0;    // bytes per element of the caller's D, B, rhs
  // factor levels: level 1 reads the caller's arrays, later levels the pools
  const void *fac_first = nullptr, *fac_rest = nullptr;
  int fac_threads = 0;
  size_t fac_smem = 0;
  // FP64 top-separator Cholesky for the mixed path (T = double, pools FP32)
  const void *root_first = nullptr, *root_rest = nullptr;
  int root_threads = 0;
  size_t root_smem = 0;
  // persistent dataflow forms (all levels in one launch)
  const void *fac_flow = nullptr, *solve_flow = nullptr;
  // interlaced factorization + forward substitution (same CTA shape as fac_flow)
  const void *fac_fwd_flow = nullptr;
  size_t (*fused_smem)(int m) = nullptr;
  // right-looking variant (Alg. 6): packing pass, per-level and persistent kernels, FP64 root
  const void *pack_matrix = nullptr, *fac_rl = nullptr, *fac_flow_rl = nullptr, *root_rl = nullptr;
  // solve
  const void *fwd = nullptr, *bwd = nullptr;
  size_t (*fwd_smem)(int m) = nullptr;
  int max_cols = 16;  // right-hand sides per solve launch that fit in shared memory
  size_t (*bwd_smem)(int m) = nullptr;
  const void *pack = nullptr, *unpack = nullptr, *resid = nullptr;
};

// dtype codes as in btc.h
const KernelSet &kernels_for(int dtype, int np);
void register_f64(KernelSet *table, int *count);
void register_f32(KernelSet *table, int *count);
void register_mixed(KernelSet *table, int *count);

}  // namespace btc
