// FP64 vector kernels of the GMRES-based refinement (btc_solve_gmres_ir): the
// dot products, updates and scalings of the Arnoldi process on vectors of
// length L = N n. Every reduction has a fixed order, so results are
// reproducible run to run.
#pragma once
#include <cstdint>

namespace btc {

constexpr int kKryThreads = 512;

// out[j] = V_j . w for j < gridDim.x (V_j = V + j * ldv): one CTA per vector,
// strided partial sums, then a shared-memory tree.
__global__ void __launch_bounds__(kKryThreads) k_mdot(const double *V, int64_t ldv, const double *w, int64_t L,
                                                      double *out) {
  grid_dep_enter();
  __shared__ double red[kKryThreads];
  const double *v = V + (int64_t)blockIdx.x * ldv;
  double s = 0.0;
  for (int64_t i = threadIdx.x; i < L; i += kKryThreads) s = fma(v[i], w[i], s);
  red[threadIdx.x] = s;
  __syncthreads();
  for (int o = kKryThreads / 2; o > 0; o >>= 1) {
    if (threadIdx.x < o) red[threadIdx.x] += red[threadIdx.x + o];
    __syncthreads();
  }
  if (threadIdx.x == 0) out[blockIdx.x] = red[0];
}

// w += sign * sum_{j < k} h[j] V_j (h on the device).
__global__ void k_mupdate(double *w, const double *V, int64_t ldv, const double *h, int k, int64_t L, double sign) {
  grid_dep_enter();
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < L; i += (int64_t)gridDim.x * blockDim.x) {
    double a = w[i];
    for (int j = 0; j < k; ++j) a = fma(sign * h[j], V[(int64_t)j * ldv + i], a);
    w[i] = a;
  }
}

// v = s * w, with s = scale, or s = 1 / sqrt(*nrm2) when nrm2 is given (a squared norm on the device).
__global__ void k_vscale(double *v, const double *w, double scale, const double *nrm2, int64_t L) {
  grid_dep_enter();
  const double s = nrm2 ? (*nrm2 > 0.0 ? 1.0 / sqrt(*nrm2) : 0.0) : scale;
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < L; i += (int64_t)gridDim.x * blockDim.x)
    v[i] = s * w[i];
}

}  // namespace btc
