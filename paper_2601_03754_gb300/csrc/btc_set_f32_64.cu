// Kernel set: FP32 inputs, factor and solves, padded block size 64.
#include "btc_make.cuh"

namespace btc {
KernelSet make_set_f32_64() { return make_set<float, float, 64, false>(); }
}  // namespace btc
