// Kernel set: FP64 factor and solves, padded block size 16.
#include "btc_make.cuh"

namespace btc {
KernelSet make_set_f64_16() { return make_set<double, double, 16, false>(); }
}  // namespace btc
