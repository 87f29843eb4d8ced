// Kernel set: FP64 factor and solves, padded block size 96.
#include "btc_make.cuh"

namespace btc {
KernelSet make_set_f64_96() { return make_set<double, double, 96, false>(); }
}  // namespace btc
