// FP32 instantiations: plain FP32 inputs.
#include "btc_make.cuh"

namespace btc {
void register_f32(KernelSet *t, int *count) {
  int c = 0;
  t[c++] = make_set<float, float, 8, false>();
  t[c++] = make_set<float, float, 16, false>();
  t[c++] = make_set<float, float, 32, false>();
  t[c++] = make_set<float, float, 48, false>();
  t[c++] = make_set<float, float, 64, false>();
  t[c++] = make_set<float, float, 96, false>();
  t[c++] = make_set<float, float, 128, false>();
  *count = c;
}
}  // namespace btc
