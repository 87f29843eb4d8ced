// Kernel set: FP64 inputs, FP32 factor with the level-elimination products on
// tcgen05 (TF32), FP32 correction solves, FP64 top-separator Cholesky; padded
// block size 128.
#include "btc_make.cuh"

namespace btc {
KernelSet make_set_tf32_128() { return make_set_tc128(); }
}  // namespace btc
