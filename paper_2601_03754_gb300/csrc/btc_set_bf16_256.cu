// Kernel set: FP64 inputs, blocked 256 x 256 nodes of tile tasks with the
// products on tcgen05 (BF16 operands, FP32 accumulation), FP32 correction
// solves; padded block size 256.
#include "btc_tiles.cuh"

namespace btc {
KernelSet make_set_bf16_256() { return make_set_tiled<2>(); }
}  // namespace btc
