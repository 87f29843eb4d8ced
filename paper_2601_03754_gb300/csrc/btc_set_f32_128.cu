// Kernel set: FP32 inputs, factor and solves, padded block size 128.
#include "btc_make.cuh"

namespace btc {
KernelSet make_set_f32_128() { return make_set<float, float, 128, false>(); }
}  // namespace btc
