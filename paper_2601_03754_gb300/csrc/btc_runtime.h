// Helpers shared by the single-instance (btc_api.cu) and batched
// (btc_batch.cu) runtimes. Not part of the public ABI.
#pragma once
#include <cuda_runtime.h>

#include <algorithm>
#include <cstdint>

#include "../../include/btc.h"
#include "btc_kernels.h"

namespace btc {

// Record a formatted message for btc_last_error() and return `code`.
int fail(int code, const char *fmt, ...);
int set_smem(const void *fn, size_t bytes);
bool dtype_ok(int dtype);
bool dtype_mixed(int dtype);  // FP64 inputs, FP32 factor, FP64 (or double-FP32) root, FP64 refinement

constexpr int kMaxCols = 16;     // right-hand sides per solve launch
constexpr int kFlowHeader = 4;   // ints before the done flags of a flow state array
// widest dependency wave of a solve that the one-CTA small solve takes (two rounds of its 32 warps)
constexpr int kSmallSolveWidth = 64;

#define BTC_CUDA(call)                                                                                       \
  do {                                                                                                       \
    cudaError_t e_ = (call);                                                                                 \
    if (e_ != cudaSuccess)                                                                                   \
      return ::btc::fail(e_ == cudaErrorMemoryAllocation ? BTC_ERR_OOM : BTC_ERR_CUDA, "%s: %s (%s:%d)", #call, \
                         cudaGetErrorString(e_), __FILE__, __LINE__);                                        \
  } while (0)

#ifdef __CUDACC__
// Programmatic dependent launch. Every kernel starts with this wait, which returns once the previous
// kernel of the stream has completed and its writes are visible (at once for a launch without that
// dependency). No kernel triggers its dependents early: the trigger is the implicit one when all of its
// CTAs have exited, so the next kernel's launch overlaps only this kernel's completion. (Triggering at
// kernel entry let the next kernel's CTAs sit resident beside the running dependency chains and made
// the refined N=1024, n=64 step 5 % slower.)
__device__ __forceinline__ void grid_dep_enter() { asm volatile("griddepcontrol.wait;" ::: "memory"); }
#endif

// Launch with programmatic stream serialization (the kernel must start with grid_dep_enter).
inline cudaError_t launch_ex(const void *fn, dim3 grid, dim3 block, void **args, size_t smem, cudaStream_t s) {
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = grid;
  cfg.blockDim = block;
  cfg.dynamicSmemBytes = smem;
  cfg.stream = s;
  cudaLaunchAttribute attr[1];
  attr[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
  attr[0].val.programmaticStreamSerializationAllowed = 1;
  cfg.attrs = attr;
  cfg.numAttrs = 1;
  return cudaLaunchKernelExC(&cfg, fn, args);
}

template <typename... A>
inline int launch_n(const void *fn, int grid, int block, size_t smem, cudaStream_t s, A... a) {
  if (grid <= 0) return BTC_OK;
  void *args[] = {(void *)&a...};
  BTC_CUDA(launch_ex(fn, dim3(grid), dim3(block), args, smem, s));
  return BTC_OK;
}

// CTAs-per-SM counts a tuner tries: 1, 2, 4, ... and the largest that fits (occ); after occ: occ + 1 (stop).
inline int next_ctas(int c, int occ) { return c >= occ ? occ + 1 : (2 * c <= occ ? 2 * c : occ); }

inline int grid_for(int64_t total) {
  int64_t g = (total + 255) / 256;
  return (int)std::max<int64_t>(1, std::min<int64_t>(g, 152 * 8));
}

}  // namespace btc
