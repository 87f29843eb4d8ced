// Kernel table: the compiled instantiations for one (dtype, np) pair, filled
// by the per-dtype translation units and launched by the runtime.
#pragma once
#include <cuda_runtime.h>
#include <stddef.h>
#include <stdint.h>

namespace btc {

// One compiled form of the persistent factorization kernels: the register
// budget is set for `minb` resident CTAs per SM (launch bounds), so the
// variants trade registers per thread against CTAs per SM. The autotuner of a
// plan picks the variant and the grid (btc_plan_set_autotune).
struct FlowVariant {
  int minb = 0;  // 0: absent
  const void *fac = nullptr, *fac_fwd = nullptr, *fac_rl = nullptr;
};
constexpr int kFlowVariants = 5;

struct KernelSet {
  bool valid = false;
  int np = 0;
  size_t elem = 0;        // bytes per pool element
  size_t src_elem = 0;    // bytes per element of the caller's D, B, rhs
  // factor levels: level 1 reads the caller's arrays, later levels the pools
  const void *fac_first = nullptr, *fac_rest = nullptr;
  int fac_threads = 0;
  size_t fac_smem = 0;
  // top-separator Cholesky of the mixed path (FP32 pools): double-FP32 and FP64 forms
  const void *root_first = nullptr, *root_rest = nullptr;
  const void *root64_first = nullptr, *root64_rest = nullptr, *root64_rl = nullptr;  // FP64 form (default)
  int root_threads = 0;
  size_t root_smem = 0;
  // persistent dataflow forms (all levels in one launch)
  const void *fac_flow = nullptr, *solve_flow = nullptr;
  // interlaced factorization + forward substitution (same CTA shape as fac_flow)
  const void *fac_fwd_flow = nullptr;
  size_t (*fused_smem)(int m) = nullptr;
  // all compiled residency variants of the three persistent factor kernels;
  // fac_flow, fac_fwd_flow and fac_flow_rl above are those of flow_v[flow_default]
  FlowVariant flow_v[kFlowVariants];
  int n_flow_v = 0, flow_default = 0;
  bool tensor_cores = false;  // level elimination products on tcgen05 (TF32 or BF16 operands)
  // blocked nodes of tile tasks (padded n = 256): a packing pass (pack_pools) and one persistent
  // launch of tile tasks replace the node kernels; the top separator is one more node of that launch
  bool tiled = false;
  const void *tile_flow = nullptr;
  size_t tile_smem = 0;
  // right-looking variant (Alg. 6): packing pass, per-level and persistent kernels, double-FP32 root (its FP64 form is root64_rl)
  const void *fac_rl = nullptr, *fac_flow_rl = nullptr, *root_rl = nullptr;
  // the packing pass, launched through a typed wrapper (N CTAs): D, B the caller's arrays in the
  // set's source type; orient null (the ND level-1 orientation) or one flag per coupling
  int (*pack_pools)(void *dpool, void *epool, const void *D, const void *B, int N, int n, const int8_t *orient,
              cudaStream_t s) = nullptr;
  // the batched packing pass over a group's nodes (PackNode list, per-instance descriptors)
  int (*pack_batch)(void *dpool, void *epool, const void *nodes, const void *inst, int count, cudaStream_t s) = nullptr;
  // solve
  const void *fwd = nullptr, *bwd = nullptr;
  // the whole solve of a small plan in one CTA, items by dependency waves (FP32 factor, np <= 16,
  // one right-hand side; null otherwise)
  int (*solve_small)(const void *items, int count, const void *dpool, const void *epool, void *y,
                     const int32_t *order, const int32_t *wave_off, int nwaves, int ycount, int threads,
                     cudaStream_t s) = nullptr;
  size_t (*fwd_smem)(int m) = nullptr;
  int max_cols = 16;  // right-hand sides per solve launch that fit in shared memory
  size_t (*bwd_smem)(int m) = nullptr;
  const void *pack = nullptr, *unpack = nullptr, *resid = nullptr;
  // the FP64 residual (k_residual<T>), launched through a typed wrapper: y the work vector (pool type)
  int (*residual)(void *y, const double *D, const double *B, const double *x, const double *b, int N, int n, int np,
                  int m, int64_t node_base, double *norms, int with_anorm, cudaStream_t s) = nullptr;
};

// dtype codes as in btc.h
const KernelSet &kernels_for(int dtype, int np);

// Every compiled (dtype, padded block size) pair; each has its own translation
// unit btc_set_<dtype>_<np>.cu so that the build compiles them in parallel.
// FP64 stops at 96 (three 128 x 128 FP64 blocks exceed one SM's shared memory);
// the TF32 and BF16 tensor-core dtypes have their own sets at 128 and 256 (the
// blocked node of tile tasks) and share the mixed FP32 sets below 128.
#define BTC_FOR_EACH_SET(X)                                                                              \
  X(f64, 8) X(f64, 16) X(f64, 32) X(f64, 48) X(f64, 64) X(f64, 96)                                        \
  X(f32, 8) X(f32, 16) X(f32, 32) X(f32, 48) X(f32, 64) X(f32, 96) X(f32, 128)                            \
  X(mixed, 8) X(mixed, 16) X(mixed, 32) X(mixed, 48) X(mixed, 64) X(mixed, 96) X(mixed, 128)                \
  X(tf32, 128) X(bf16, 128) X(tf32, 256) X(bf16, 256)
#define BTC_DECLARE_SET(dt, np) KernelSet make_set_##dt##_##np();
BTC_FOR_EACH_SET(BTC_DECLARE_SET)
#undef BTC_DECLARE_SET

}  // namespace btc
