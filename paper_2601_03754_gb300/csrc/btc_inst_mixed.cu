// Mixed-precision instantiations: FP64 inputs, FP32 factor and correction
// solves, FP64 top-separator Cholesky.
#include "btc_make.cuh"

namespace btc {
void register_mixed(KernelSet *t, int *count) {
  int c = 0;
  t[c++] = make_set<float, double, 8, true>();
  t[c++] = make_set<float, double, 16, true>();
  t[c++] = make_set<float, double, 32, true>();
  t[c++] = make_set<float, double, 48, true>();
  t[c++] = make_set<float, double, 64, true>();
  t[c++] = make_set<float, double, 96, true>();
  t[c++] = make_set<float, double, 128, true>();
  *count = c;
}
}  // namespace btc
