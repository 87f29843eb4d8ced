// Kernel set: FP64 inputs, FP32 factor and correction solves, FP64 (or double-FP32) top-separator Cholesky, padded block size 128.
#include "btc_make.cuh"

namespace btc {
KernelSet make_set_mixed_128() { return make_set<float, double, 128, true>(); }
}  // namespace btc
