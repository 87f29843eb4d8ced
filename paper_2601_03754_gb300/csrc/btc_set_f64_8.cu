// Kernel set: FP64 factor and solves, padded block size 8.
#include "btc_make.cuh"

namespace btc {
KernelSet make_set_f64_8() { return make_set<double, double, 8, false>(); }
}  // namespace btc
