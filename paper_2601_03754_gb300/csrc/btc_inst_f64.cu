// FP64 instantiations (the plain FP64 path).
#include "btc_make.cuh"

namespace btc {
void register_f64(KernelSet *t, int *count) {
  int c = 0;
  t[c++] = make_set<double, double, 8, false>();
  t[c++] = make_set<double, double, 16, false>();
  t[c++] = make_set<double, double, 32, false>();
  t[c++] = make_set<double, double, 48, false>();
  t[c++] = make_set<double, double, 64, false>();
  t[c++] = make_set<double, double, 96, false>();
  *count = c;
}
}  // namespace btc
