// Kernel set: FP64 inputs, FP32 factor and correction solves, FP64 (or double-FP32) top-separator Cholesky, padded block size 16.
#include "btc_make.cuh"

namespace btc {
KernelSet make_set_mixed_16() { return make_set<float, double, 16, true>(); }
}  // namespace btc
