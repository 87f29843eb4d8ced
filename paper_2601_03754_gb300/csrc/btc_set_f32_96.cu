// Kernel set: FP32 inputs, factor and solves, padded block size 96.
#include "btc_make.cuh"

namespace btc {
KernelSet make_set_f32_96() { return make_set<float, float, 96, false>(); }
}  // namespace btc
