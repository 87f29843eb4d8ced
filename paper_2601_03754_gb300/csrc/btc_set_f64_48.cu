// Kernel set: FP64 factor and solves, padded block size 48.
#include "btc_make.cuh"

namespace btc {
KernelSet make_set_f64_48() { return make_set<double, double, 48, false>(); }
}  // namespace btc
