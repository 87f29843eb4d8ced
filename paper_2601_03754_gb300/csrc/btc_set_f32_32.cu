// Kernel set: FP32 inputs, factor and solves, padded block size 32.
#include "btc_make.cuh"

namespace btc {
KernelSet make_set_f32_32() { return make_set<float, float, 32, false>(); }
}  // namespace btc
