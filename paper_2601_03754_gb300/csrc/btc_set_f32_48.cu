// Kernel set: FP32 inputs, factor and solves, padded block size 48.
#include "btc_make.cuh"

namespace btc {
KernelSet make_set_f32_48() { return make_set<float, float, 48, false>(); }
}  // namespace btc
