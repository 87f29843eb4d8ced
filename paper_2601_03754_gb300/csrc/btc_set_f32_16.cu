// Kernel set: FP32 inputs, factor and solves, padded block size 16.
#include "btc_make.cuh"

namespace btc {
KernelSet make_set_f32_16() { return make_set<float, float, 16, false>(); }
}  // namespace btc
