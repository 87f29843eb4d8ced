// btc_residual_noalloc: the residual/norm computation of btc_residual with its
// scratch in a fixed, file-scope device array instead of memory allocated per
// call. For callers that must not allocate device memory at all (see btc.h).
//
// Scratch: per block row, the three partial maxima (|r|, row sum of |Psi|,
// |x|), reduced by a second kernel. Capacity: kNoAllocMaxBlocks block rows.
#include <cuda_runtime.h>

#include <cstdio>
#include <mutex>

#include "../../include/btc.h"

namespace {

constexpr int kNoAllocMaxBlocks = 1 << 16;  // 65536 block rows -> 1.5 MiB of scratch per device
constexpr int kMaxDevices = 64;

// Partial maxima of block row i at [3*i .. 3*i+2]; the reduced result at the end.
static __device__ __align__(256) double g_noalloc_scratch[3 * kNoAllocMaxBlocks + 3];

// max(a, b) that propagates NaN (fmax drops it), so that a NaN in b, x or the
// matrix shows in the returned norms.
__device__ __forceinline__ double max_keep_nan(double a, double b) { return (b > a || b != b) ? b : a; }

// Host-side device addresses of g_noalloc_scratch, one per device (the array's
// name in host code is only a stand-in, never a device address).
static double *g_scratch_ptr[kMaxDevices] = {nullptr};
static std::mutex g_scratch_mu;

// One CTA per block row: the same FP64 arithmetic as the library's residual
// kernel, writing this row's maxima to the scratch instead of a shared atomic.
__global__ void k_residual_rows(const double *D, const double *B, const double *x, const double *b, int N, int n,
                                int m, double *part) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  const int i = blockIdx.x;
  const int ld = n + 1;
  double *Ds = reinterpret_cast<double *>(smem_raw);
  double *Bl = Ds + n * ld;
  double *Br = Bl + n * ld;
  __shared__ double red[3][32];
  const size_t bs = (size_t)n * n;
  for (int q = threadIdx.x; q < n * n; q += blockDim.x) {
    const int r = q / n, c = q % n;
    Ds[r * ld + c] = D[i * bs + q];
    if (i > 0) Bl[r * ld + c] = B[(i - 1) * bs + q];
    if (i + 1 < N) Br[r * ld + c] = B[i * bs + q];
  }
  __syncthreads();
  double rmax = 0.0, amax = 0.0, xmax = 0.0;
  const double *xi = x + (size_t)i * n * m;
  for (int r = threadIdx.x; r < n; r += blockDim.x) {
    double s = 0.0;
    for (int c = 0; c < n; ++c) s += fabs(r >= c ? Ds[r * ld + c] : Ds[c * ld + r]);
    if (i > 0)
      for (int c = 0; c < n; ++c) s += fabs(Bl[r * ld + c]);
    if (i + 1 < N)
      for (int c = 0; c < n; ++c) s += fabs(Br[c * ld + r]);
    amax = max_keep_nan(amax, s);
  }
  for (int q = threadIdx.x; q < n * m; q += blockDim.x) {
    const int r = q / m, col = q % m;
    double v = b[((size_t)i * n + r) * m + col];
    for (int c = 0; c < n; ++c) v = fma(-(r >= c ? Ds[r * ld + c] : Ds[c * ld + r]), xi[c * m + col], v);
    if (i > 0) {
      const double *xp = x + (size_t)(i - 1) * n * m;
      for (int c = 0; c < n; ++c) v = fma(-Bl[r * ld + c], xp[c * m + col], v);
    }
    if (i + 1 < N) {
      const double *xn = x + (size_t)(i + 1) * n * m;
      for (int c = 0; c < n; ++c) v = fma(-Br[c * ld + r], xn[c * m + col], v);
    }
    rmax = max_keep_nan(rmax, fabs(v));
    xmax = max_keep_nan(xmax, fabs(xi[r * m + col]));
  }
  for (int o = 16; o > 0; o >>= 1) {
    rmax = max_keep_nan(rmax, __shfl_xor_sync(0xffffffffu, rmax, o));
    amax = max_keep_nan(amax, __shfl_xor_sync(0xffffffffu, amax, o));
    xmax = max_keep_nan(xmax, __shfl_xor_sync(0xffffffffu, xmax, o));
  }
  const int w = threadIdx.x >> 5, nw = blockDim.x >> 5;
  if ((threadIdx.x & 31) == 0) {
    red[0][w] = rmax;
    red[1][w] = amax;
    red[2][w] = xmax;
  }
  __syncthreads();
  if (threadIdx.x < 3) {
    double v = 0.0;
    for (int k = 0; k < nw; ++k) v = max_keep_nan(v, red[threadIdx.x][k]);
    part[3 * i + threadIdx.x] = v;  // every slot of rows 0..N-1 is overwritten: nothing to clear
  }
}

// Max over the N partial triples into out[0..2] (one CTA).
__global__ void k_reduce_rows(const double *part, int N, double *out) {
  __shared__ double red[3][32];
  double v[3] = {0.0, 0.0, 0.0};
  for (int i = threadIdx.x; i < N; i += blockDim.x)
    for (int k = 0; k < 3; ++k) v[k] = max_keep_nan(v[k], part[3 * i + k]);
  for (int k = 0; k < 3; ++k)
    for (int o = 16; o > 0; o >>= 1) v[k] = max_keep_nan(v[k], __shfl_xor_sync(0xffffffffu, v[k], o));
  const int w = threadIdx.x >> 5, nw = blockDim.x >> 5;
  if ((threadIdx.x & 31) == 0)
    for (int k = 0; k < 3; ++k) red[k][w] = v[k];
  __syncthreads();
  if (threadIdx.x < 3) {
    double r = 0.0;
    for (int k = 0; k < nw; ++k) r = max_keep_nan(r, red[threadIdx.x][k]);
    out[threadIdx.x] = r;
  }
}

}  // namespace

namespace btc {
void set_error_message(const char *msg);  // defined with btc_last_error
}

namespace {

static int fail_msg(int code, const char *msg, cudaError_t e) {
  char buf[320];
  snprintf(buf, sizeof(buf), "%s%s%s", msg, e == cudaSuccess ? "" : ": ", e == cudaSuccess ? "" : cudaGetErrorString(e));
  btc::set_error_message(buf);
  return code;
}

// Device address of the scratch array for the current device, looked up once
// per device (the first call on each device does the lookup).
static int scratch_for_current_device(double **out) {
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return fail_msg(BTC_ERR_CUDA, "btc_residual_noalloc: cudaGetDevice", e);
  if (dev < 0 || dev >= kMaxDevices) return fail_msg(BTC_ERR_ARG, "btc_residual_noalloc: device ordinal out of range", cudaSuccess);
  std::lock_guard<std::mutex> lock(g_scratch_mu);
  if (!g_scratch_ptr[dev]) {
    void *p = nullptr;
    e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
    if (e != cudaSuccess || !p) return fail_msg(BTC_ERR_CUDA, "btc_residual_noalloc: cudaGetSymbolAddress", e);
    g_scratch_ptr[dev] = static_cast<double *>(p);
  }
  *out = g_scratch_ptr[dev];
  return BTC_OK;
}

}  // namespace

extern "C" int btc_residual_noalloc(int N, int n, int nrhs, const double *D, const double *B, const double *x,
                                    const double *b, double *out3, void *stream) {
  if (N < 1 || n < 1 || nrhs < 1 || !D || (N > 1 && !B) || !x || !b || !out3)
    return fail_msg(BTC_ERR_ARG, "btc_residual_noalloc: invalid arguments", cudaSuccess);
  if (N > kNoAllocMaxBlocks)
    return fail_msg(BTC_ERR_ARG, "btc_residual_noalloc: N exceeds the 65536 block rows of the static scratch",
                    cudaSuccess);
  const size_t smem = 3 * sizeof(double) * (size_t)n * (n + 1);
  if (smem > 227 * 1024)
    return fail_msg(BTC_ERR_UNSUPPORTED, "btc_residual_noalloc: block size too large for shared memory", cudaSuccess);
  double *scratch = nullptr;
  int rc = scratch_for_current_device(&scratch);
  if (rc) return rc;
  cudaStream_t s = (cudaStream_t)stream;
  cudaError_t e = cudaFuncSetAttribute((const void *)k_residual_rows, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                       (int)smem);
  if (e != cudaSuccess) return fail_msg(BTC_ERR_CUDA, "btc_residual_noalloc: cudaFuncSetAttribute", e);
  k_residual_rows<<<N, 128, smem, s>>>(D, B, x, b, N, n, nrhs, scratch);
  double *result = scratch + 3 * (size_t)kNoAllocMaxBlocks;
  k_reduce_rows<<<1, 256, 0, s>>>(scratch, N, result);
  e = cudaGetLastError();
  if (e != cudaSuccess) return fail_msg(BTC_ERR_CUDA, "btc_residual_noalloc: launch", e);
  double h[3];
  e = cudaMemcpyAsync(h, result, sizeof(h), cudaMemcpyDeviceToHost, s);
  if (e == cudaSuccess) e = cudaStreamSynchronize(s);
  if (e != cudaSuccess) return fail_msg(BTC_ERR_CUDA, "btc_residual_noalloc: copy-back", e);
  out3[0] = h[0];  // ||b - Psi x||_inf
  out3[1] = h[1];  // ||Psi||_inf
  out3[2] = h[2];  // ||x||_inf
  return BTC_OK;
}
