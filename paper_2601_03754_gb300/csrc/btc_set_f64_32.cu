// Kernel set: FP64 factor and solves, padded block size 32.
#include "btc_make.cuh"

namespace btc {
KernelSet make_set_f64_32() { return make_set<double, double, 32, false>(); }
}  // namespace btc
