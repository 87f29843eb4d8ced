// Kernel set: FP64 factor and solves, padded block size 64.
#include "btc_make.cuh"

namespace btc {
KernelSet make_set_f64_64() { return make_set<double, double, 64, false>(); }
}  // namespace btc
