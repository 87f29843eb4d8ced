// Kernel set: FP32 inputs, factor and solves, padded block size 8.
#include "btc_make.cuh"

namespace btc {
KernelSet make_set_f32_8() { return make_set<float, float, 8, false>(); }
}  // namespace btc
