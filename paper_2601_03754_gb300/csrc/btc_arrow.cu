// Bordered ("arrow") systems: the block-tridiagonal Psi of a plan bordered by
// m dense coupling rows C (m x N n) and a dense m x m block A,
//   Psi_a = [[Psi, C^T], [C, A]].
// The permuted Cholesky view of Sec. 4.3 extends to it by eliminating the
// border last, after the whole nested-dissection tree: with P Psi P^T = L L^T,
// the border's Schur complement is S = A - C Psi^{-1} C^T = A - W^T W
// (W = L^{-1} P C^T) and its Cholesky factor closes the factorization.
//
// Factor: Psi by the plan (any dtype), Z = Psi^{-1} C^T by the plan's
// FP64-refined solves (m right-hand sides), S = A - C Z in FP64 (partial
// products over slices of the N n inner dimension, reduced in a fixed order),
// S = L_S L_S^T in FP64 (one CTA). Solve: z = Psi^{-1} b_T (refined),
// x_A = S^{-1} (b_A - C z), x_T = z - Z x_A, then FP64 residuals of the whole
// bordered system and correction passes until ||r|| <= tol ||Psi_a|| ||x||.
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <cstring>
#include <vector>

#include "../../include/btc.h"
#include "btc_runtime.h"
#include "btc_solve.cuh"

namespace btc {

constexpr int kArrowMax = 64;        // largest border width m
constexpr int kArrowChunk = 8;       // right-hand sides per refined solve of Z = Psi^{-1} C^T
constexpr int kArrowParts = 152;     // slices of the inner dimension of S = A - C Z
constexpr int kArrowK = 32;          // inner rows staged per step of a slice

// ct[i][k] = C[c0 + k][i]: columns c0 .. c0+cw-1 of C^T, row-major with cw columns.
__global__ void k_arrow_ct(double *ct, const double *C, int64_t L, int c0, int cw) {
  grid_dep_enter();
  for (int64_t q = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; q < L * cw; q += (int64_t)gridDim.x * blockDim.x) {
    const int64_t i = q / cw;
    const int k = (int)(q % cw);
    ct[q] = C[(int64_t)(c0 + k) * L + i];
  }
}

// Z[i][c0 + k] = zc[i][k]
__global__ void k_arrow_scatter(double *Z, const double *zc, int64_t L, int m, int c0, int cw) {
  grid_dep_enter();
  for (int64_t q = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; q < L * cw; q += (int64_t)gridDim.x * blockDim.x) {
    const int64_t i = q / cw;
    const int k = (int)(q % cw);
    Z[i * m + c0 + k] = zc[q];
  }
}

// part[p] = C[:, I_p] Z[I_p, :] over slice p of the inner dimension (m x m, FP64, fixed order).
__global__ void __launch_bounds__(256) k_arrow_schur_part(double *part, const double *C, const double *Z, int64_t L,
                                                          int m) {
  grid_dep_enter();
  __shared__ double Cs[kArrowMax * kArrowK];
  __shared__ double Zs[kArrowK * kArrowMax];
  const int64_t per = (L + gridDim.x - 1) / gridDim.x;
  const int64_t i0 = blockIdx.x * per, i1 = (i0 + per < L) ? i0 + per : L;
  double acc[(kArrowMax * kArrowMax + 255) / 256];
#pragma unroll
  for (int t = 0; t < (kArrowMax * kArrowMax + 255) / 256; ++t) acc[t] = 0.0;
  for (int64_t k0 = i0; k0 < i1; k0 += kArrowK) {
    const int kk = (int)(i1 - k0 < kArrowK ? i1 - k0 : kArrowK);
    __syncthreads();
    for (int q = threadIdx.x; q < m * kArrowK; q += blockDim.x) {
      const int r = q / kArrowK, k = q % kArrowK;
      Cs[r * kArrowK + k] = k < kk ? C[(int64_t)r * L + k0 + k] : 0.0;
    }
    for (int q = threadIdx.x; q < kArrowK * m; q += blockDim.x) {
      const int k = q / m, c = q % m;
      Zs[k * kArrowMax + c] = k < kk ? Z[(k0 + k) * m + c] : 0.0;
    }
    __syncthreads();
#pragma unroll
    for (int t = 0; t < (kArrowMax * kArrowMax + 255) / 256; ++t) {
      const int q = threadIdx.x + 256 * t;
      if (q >= m * m) break;
      const int r = q / m, c = q % m;
      double a = acc[t];
      for (int k = 0; k < kk; ++k) a = fma(Cs[r * kArrowK + k], Zs[k * kArrowMax + c], a);
      acc[t] = a;
    }
  }
#pragma unroll
  for (int t = 0; t < (kArrowMax * kArrowMax + 255) / 256; ++t) {
    const int q = threadIdx.x + 256 * t;
    if (q < m * m) part[(int64_t)blockIdx.x * m * m + q] = acc[t];
  }
}

// S = A - sum_p part[p] (A: lower triangle read, mirrored; the partials added in slice order).
__global__ void k_arrow_schur_reduce(double *S, const double *A, const double *part, int parts, int m) {
  grid_dep_enter();
  for (int q = blockIdx.x * blockDim.x + threadIdx.x; q < m * m; q += gridDim.x * blockDim.x) {
    const int r = q / m, c = q % m;
    double s = 0.0;
    for (int p = 0; p < parts; ++p) s += part[(int64_t)p * m * m + q];
    S[q] = (r >= c ? A[r * m + c] : A[c * m + r]) - s;
  }
}

// In-place lower Cholesky of S (m x m, FP64) by one CTA, right-looking, in shared memory. A pivot
// that is not positive (or NaN) is reported as (node = N, column) and replaced by 1.
__global__ void k_arrow_chol(double *S, int m, int N, unsigned long long *info) {
  grid_dep_enter();
  __shared__ double a[kArrowMax * (kArrowMax + 1)];
  constexpr int LD = kArrowMax + 1;
  for (int q = threadIdx.x; q < m * m; q += blockDim.x) a[(q / m) * LD + q % m] = S[q];
  __syncthreads();
  for (int k = 0; k < m; ++k) {
    if (threadIdx.x == 0) {
      double d = a[k * LD + k];
      if (!(d > 0.0)) {
        atomicMin(info, ((unsigned long long)(unsigned)N << 20) | (unsigned)k);
        d = 1.0;
      }
      a[k * LD + k] = sqrt(d);
    }
    __syncthreads();
    for (int i = k + 1 + threadIdx.x; i < m; i += blockDim.x) a[i * LD + k] /= a[k * LD + k];
    __syncthreads();
    for (int q = threadIdx.x; q < (m - k - 1) * (m - k - 1); q += blockDim.x) {
      const int i = k + 1 + q / (m - k - 1), j = k + 1 + q % (m - k - 1);
      if (j <= i) a[i * LD + j] = fma(-a[i * LD + k], a[j * LD + k], a[i * LD + j]);
    }
    __syncthreads();
  }
  for (int q = threadIdx.x; q < m * m; q += blockDim.x) {
    const int i = q / m, j = q % m;
    S[q] = j <= i ? a[i * LD + j] : 0.0;
  }
}

// y[r] = bA[r] - sum_i C[r][i] z[i], one CTA per border row (fixed-order tree reduction).
__global__ void __launch_bounds__(256) k_arrow_cz(double *y, const double *bA, const double *C, const double *z,
                                                  int64_t L) {
  grid_dep_enter();
  __shared__ double red[256];
  const int r = blockIdx.x;
  double s = 0.0;
  for (int64_t i = threadIdx.x; i < L; i += 256) s = fma(C[(int64_t)r * L + i], z[i], s);
  red[threadIdx.x] = s;
  __syncthreads();
  for (int o = 128; o > 0; o >>= 1) {
    if (threadIdx.x < o) red[threadIdx.x] += red[threadIdx.x + o];
    __syncthreads();
  }
  if (threadIdx.x == 0) y[r] = bA[r] - red[0];
}

// x = L_S^{-T} L_S^{-1} y (forward then backward substitution, one warp).
__global__ void k_arrow_trsv(double *x, const double *Ls, const double *y, int m) {
  grid_dep_enter();
  __shared__ double w[kArrowMax];
  const int lane = threadIdx.x;
  for (int j = 0; j < m; ++j) {
    double s = 0.0;
    for (int k = lane; k < j; k += 32) s = fma(Ls[j * m + k], w[k], s);
    for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
    if (lane == 0) w[j] = (y[j] - s) / Ls[j * m + j];
    __syncwarp();
  }
  for (int j = m - 1; j >= 0; --j) {
    double s = 0.0;
    for (int k = j + 1 + lane; k < m; k += 32) s = fma(Ls[k * m + j], w[k], s);
    for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
    if (lane == 0) w[j] = (w[j] - s) / Ls[j * m + j];
    __syncwarp();
  }
  for (int j = lane; j < m; j += 32) x[j] = w[j];
}

// xT[i] = z[i] - sum_c Z[i][c] xA[c]  (accumulate: xT[i] += that)
__global__ void k_arrow_zx(double *xT, const double *z, const double *Z, const double *xA, int64_t L, int m,
                           int accumulate) {
  grid_dep_enter();
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < L; i += (int64_t)gridDim.x * blockDim.x) {
    double v = z[i];
    for (int c = 0; c < m; ++c) v = fma(-Z[i * m + c], xA[c], v);
    xT[i] = accumulate ? xT[i] + v : v;
  }
}

// bp[i] = bT[i] - sum_r C[r][i] xA[r]  (the border's contribution moved to the right-hand side)
__global__ void k_arrow_ctx(double *bp, const double *bT, const double *C, const double *xA, int64_t L, int m) {
  grid_dep_enter();
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < L; i += (int64_t)gridDim.x * blockDim.x) {
    double v = bT[i];
    for (int r = 0; r < m; ++r) v = fma(-C[(int64_t)r * L + i], xA[r], v);
    bp[i] = v;
  }
}

// Border rows of the residual: rA[r] = bA[r] - C[r] xT - A[r] xA (one CTA per row, fixed-order
// reduction); max |rA| into norms[0] and max |xA| into norms[1] (NaN propagates).
__global__ void __launch_bounds__(256) k_arrow_border_resid(double *rA, double *norms, const double *bA,
                                                            const double *C, const double *xT, const double *A,
                                                            const double *xA, int64_t L, int m) {
  grid_dep_enter();
  __shared__ double red[256];
  const int r = blockIdx.x;
  double s = 0.0;
  for (int64_t i = threadIdx.x; i < L; i += 256) s = fma(C[(int64_t)r * L + i], xT[i], s);
  for (int c = threadIdx.x; c < m; c += 256) s = fma(r >= c ? A[r * m + c] : A[c * m + r], xA[c], s);
  red[threadIdx.x] = s;
  __syncthreads();
  for (int o = 128; o > 0; o >>= 1) {
    if (threadIdx.x < o) red[threadIdx.x] += red[threadIdx.x + o];
    __syncthreads();
  }
  if (threadIdx.x == 0) {
    const double v = bA[r] - red[0];
    if (rA) rA[r] = v;
    atomic_max_nonneg(norms + 0, nan_max(0.0, fabs(v)));
    atomic_max_nonneg(norms + 1, nan_max(0.0, fabs(xA[r])));
  }
}

// x[i] += d[i] for the m border entries.
__global__ void k_arrow_add(double *x, const double *d, int m) {
  grid_dep_enter();
  for (int i = threadIdx.x; i < m; i += blockDim.x) x[i] += d[i];
}

// ||Psi_a||_inf over the border rows: sum_i |C[r][i]| + sum_c |A[r][c]| (one CTA per row), into norms[2].
__global__ void __launch_bounds__(256) k_arrow_anorm_border(double *norms, const double *C, const double *A,
                                                            int64_t L, int m) {
  grid_dep_enter();
  __shared__ double red[256];
  const int r = blockIdx.x;
  double s = 0.0;
  for (int64_t i = threadIdx.x; i < L; i += 256) s += fabs(C[(int64_t)r * L + i]);
  for (int c = threadIdx.x; c < m; c += 256) s += fabs(r >= c ? A[r * m + c] : A[c * m + r]);
  red[threadIdx.x] = s;
  __syncthreads();
  for (int o = 128; o > 0; o >>= 1) {
    if (threadIdx.x < o) red[threadIdx.x] += red[threadIdx.x + o];
    __syncthreads();
  }
  if (threadIdx.x == 0) atomic_max_nonneg(norms + 2, nan_max(0.0, red[0]));
}

// ||Psi_a||_inf over the block-tridiagonal rows: each row's absolute sum of D, B and the border
// column C^T (one CTA per block row), into norms[2].
__global__ void k_arrow_anorm_rows(const double *D, const double *B, const double *C, int N, int n, int m,
                                   double *norms) {
  grid_dep_enter();
  const int i = blockIdx.x;
  const size_t bs = (size_t)n * n;
  const int64_t L = (int64_t)N * n;
  double best = 0.0;
  for (int r = threadIdx.x; r < n; r += blockDim.x) {
    double s = 0.0;
    for (int c = 0; c < n; ++c) s += fabs(r >= c ? D[i * bs + r * n + c] : D[i * bs + c * n + r]);
    if (i > 0)
      for (int c = 0; c < n; ++c) s += fabs(B[(i - 1) * bs + r * n + c]);
    if (i + 1 < N)
      for (int c = 0; c < n; ++c) s += fabs(B[i * bs + c * n + r]);
    for (int q = 0; q < m; ++q) s += fabs(C[(int64_t)q * L + (int64_t)i * n + r]);
    best = nan_max(best, s);
  }
  for (int o = 16; o > 0; o >>= 1) best = nan_max(best, __shfl_xor_sync(0xffffffffu, best, o));
  if ((threadIdx.x & 31) == 0) atomic_max_nonneg(norms + 2, best);
}

}  // namespace btc

using namespace btc;

struct btc_arrow_s {
  btc_plan_t plan = nullptr;
  int N = 0, n = 0, m = 0;
  int64_t L = 0;
  cudaStream_t stream = nullptr;
  double *ct = nullptr, *zc = nullptr;  // [L][kArrowChunk] each
  double *Z = nullptr;                  // [L][m]
  double *part = nullptr;               // [kArrowParts][m][m]
  double *S = nullptr;                  // [m][m]: S, then its lower Cholesky factor
  double *z = nullptr, *bp = nullptr, *r = nullptr, *d = nullptr;  // [L + m] work vectors
  double *yA = nullptr;                 // [m]
  double *norms = nullptr;              // [3] device
  unsigned long long *info = nullptr;   // border pivot report
  double *h = nullptr;                  // pinned host copy: norms[3], info
  const double *D = nullptr, *B = nullptr, *C = nullptr, *A = nullptr;
  double anorm = 0.0;
  bool factored = false;
};

namespace btc {

// x = Psi_a^{-1} rhs with the factors (inner solves refined to tol); rhs, x: [L + m] device.
static int arrow_apply(btc_arrow_s *a, const double *rhs, double *x, double tol, int maxit, int accumulate) {
  int rc, it = 0;
  double rel = 0.0;
  rc = btc_solve_refined(a->plan, rhs, a->z, 1, tol, maxit, &it, &rel);
  if (rc && rc != BTC_ERR_NOT_CONVERGED) return rc;
  const int gv = grid_for(a->L);
  double *xA = x + a->L;
  if ((rc = launch_n((const void *)&k_arrow_cz, a->m, 256, 0, a->stream, a->yA, rhs + a->L, a->C,
                     (const double *)a->z, a->L)))
    return rc;
  // x_A (or a correction of it) into the last m entries of d, then x_T
  double *dA = a->d + a->L;
  if ((rc = launch_n((const void *)&k_arrow_trsv, 1, 32, 0, a->stream, dA, (const double *)a->S, (const double *)a->yA,
                     a->m)) ||
      (rc = launch_n((const void *)&k_arrow_zx, gv, 256, 0, a->stream, x, (const double *)a->z, (const double *)a->Z,
                     (const double *)dA, a->L, a->m, accumulate)))
    return rc;
  if (accumulate) {
    if ((rc = launch_n((const void *)&k_arrow_add, 1, 64, 0, a->stream, xA, (const double *)dA, a->m))) return rc;
  } else {
    BTC_CUDA(cudaMemcpyAsync(xA, dA, a->m * sizeof(double), cudaMemcpyDeviceToDevice, a->stream));
  }
  return BTC_OK;
}

// r = b - Psi_a x (FP64) into a->r when r_out, norms into a->norms; returns the relative residual.
static int arrow_residual(btc_arrow_s *a, const double *b, const double *x, double *rel, bool r_out) {
  int rc;
  BTC_CUDA(cudaMemsetAsync(a->norms, 0, 2 * sizeof(double), a->stream));
  const int gv = grid_for(a->L);
  if ((rc = launch_n((const void *)&k_arrow_ctx, gv, 256, 0, a->stream, a->bp, b, a->C, x + a->L, a->L, a->m)))
    return rc;
  double *yT = r_out ? a->r : nullptr;
  // no matrix-norm bound: the norm is exact and known from the factorization
  if ((rc = launch_residual<double>(yT, a->D, a->B, x, (const double *)a->bp, a->N, a->n, a->n, 1, 0, a->norms, 0,
                                    a->stream)) ||
      (rc = launch_n((const void *)&k_arrow_border_resid, a->m, 256, 0, a->stream, r_out ? a->r + a->L : nullptr,
                     a->norms, b + a->L, a->C, x, a->A, x + a->L, a->L, a->m)))
    return rc;
  BTC_CUDA(cudaMemcpyAsync(a->h, a->norms, 2 * sizeof(double), cudaMemcpyDeviceToHost, a->stream));
  BTC_CUDA(cudaStreamSynchronize(a->stream));
  const double rn = a->h[0], xn = a->h[1];
  *rel = (a->anorm * xn > 0) ? rn / (a->anorm * xn) : rn;
  return BTC_OK;
}

}  // namespace btc

extern "C" {

int btc_arrow_plan(btc_arrow_t *out, int N, int n, int m, int dtype, void *stream) {
  if (!out || N < 1 || n < 1 || m < 1) return fail(BTC_ERR_ARG, "btc_arrow_plan: invalid arguments");
  *out = nullptr;
  if (m > kArrowMax) return fail(BTC_ERR_UNSUPPORTED, "btc_arrow_plan: border width %d above %d", m, kArrowMax);
  if (dtype == BTC_F32) return fail(BTC_ERR_ARG, "btc_arrow_plan: needs an FP64 or mixed dtype");
  const size_t rsm = residual_smem_bytes(n, 1);
  if (rsm > 220 * 1024) return fail(BTC_ERR_UNSUPPORTED, "btc_arrow_plan: block size too large");
  btc_arrow_s *a = new btc_arrow_s();
  a->N = N;
  a->n = n;
  a->m = m;
  a->L = (int64_t)N * n;
  a->stream = (cudaStream_t)stream;
  auto cleanup = [&](int code) {
    btc_arrow_free(a);
    return code;
  };
  int rc = btc_plan(&a->plan, N, n, dtype, stream);
  if (rc) return cleanup(rc);
  const size_t L = (size_t)a->L;
  cudaError_t e;
  if ((e = cudaMalloc(&a->ct, sizeof(double) * L * kArrowChunk)) != cudaSuccess ||
      (e = cudaMalloc(&a->zc, sizeof(double) * L * kArrowChunk)) != cudaSuccess ||
      (e = cudaMalloc(&a->Z, sizeof(double) * L * m)) != cudaSuccess ||
      (e = cudaMalloc(&a->part, sizeof(double) * kArrowParts * m * m)) != cudaSuccess ||
      (e = cudaMalloc(&a->S, sizeof(double) * m * m)) != cudaSuccess ||
      (e = cudaMalloc(&a->z, sizeof(double) * (L + m))) != cudaSuccess ||
      (e = cudaMalloc(&a->bp, sizeof(double) * (L + m))) != cudaSuccess ||
      (e = cudaMalloc(&a->r, sizeof(double) * (L + m))) != cudaSuccess ||
      (e = cudaMalloc(&a->d, sizeof(double) * (L + m))) != cudaSuccess ||
      (e = cudaMalloc(&a->yA, sizeof(double) * m)) != cudaSuccess ||
      (e = cudaMalloc(&a->norms, sizeof(double) * 3)) != cudaSuccess ||
      (e = cudaMalloc(&a->info, sizeof(unsigned long long))) != cudaSuccess ||
      (e = cudaMallocHost(&a->h, sizeof(double) * 4)) != cudaSuccess)
    return cleanup(fail(e == cudaErrorMemoryAllocation ? BTC_ERR_OOM : BTC_ERR_CUDA, "btc_arrow_plan: %s",
                        cudaGetErrorString(e)));
  if ((rc = set_smem((const void *)&k_residual<double>, rsm))) return cleanup(rc);
  *out = a;
  return BTC_OK;
}

int btc_arrow_factor(btc_arrow_t a, const double *D, const double *B, const double *C, const double *A, double tol,
                     int maxit) {
  if (!a || !D || (a->N > 1 && !B) || !C || !A || maxit < 0) return fail(BTC_ERR_ARG, "btc_arrow_factor: arguments");
  a->factored = false;
  int rc = btc_factor(a->plan, D, B);
  int blk = -1, col = -1;
  if (rc || (rc = btc_info(a->plan, &blk, &col))) return rc;
  a->D = D;
  a->B = B;
  a->C = C;
  a->A = A;
  const int gv = grid_for(a->L * kArrowChunk);
  // Z = Psi^{-1} C^T, kArrowChunk columns per refined solve
  for (int c0 = 0; c0 < a->m; c0 += kArrowChunk) {
    const int cw = std::min(kArrowChunk, a->m - c0);
    int it = 0;
    double rel = 0.0;
    if ((rc = launch_n((const void *)&k_arrow_ct, gv, 256, 0, a->stream, a->ct, C, a->L, c0, cw))) return rc;
    rc = btc_solve_refined(a->plan, a->ct, a->zc, cw, tol, maxit, &it, &rel);
    if (rc) return rc;
    if ((rc = launch_n((const void *)&k_arrow_scatter, gv, 256, 0, a->stream, a->Z, (const double *)a->zc, a->L, a->m,
                       c0, cw)))
      return rc;
  }
  // S = A - C Z, then S = L_S L_S^T
  BTC_CUDA(cudaMemsetAsync(a->info, 0xFF, sizeof(unsigned long long), a->stream));
  if ((rc = launch_n((const void *)&k_arrow_schur_part, kArrowParts, 256, 0, a->stream, a->part, C,
                     (const double *)a->Z, a->L, a->m)) ||
      (rc = launch_n((const void *)&k_arrow_schur_reduce, (a->m * a->m + 255) / 256, 256, 0, a->stream, a->S, A,
                     (const double *)a->part, kArrowParts, a->m)) ||
      (rc = launch_n((const void *)&k_arrow_chol, 1, 256, 0, a->stream, a->S, a->m, a->N, a->info)))
    return rc;
  // ||Psi_a||_inf (exact): block-tridiagonal rows with their border columns, then the border rows
  BTC_CUDA(cudaMemsetAsync(a->norms, 0, 3 * sizeof(double), a->stream));
  if ((rc = launch_n((const void *)&k_arrow_anorm_rows, a->N, 64, 0, a->stream, D, B, C, a->N, a->n, a->m,
                     a->norms)) ||
      (rc = launch_n((const void *)&k_arrow_anorm_border, a->m, 256, 0, a->stream, a->norms, C, A, a->L, a->m)))
    return rc;
  BTC_CUDA(cudaMemcpyAsync(a->h, a->norms, 3 * sizeof(double), cudaMemcpyDeviceToHost, a->stream));
  BTC_CUDA(cudaMemcpyAsync(a->h + 3, a->info, sizeof(unsigned long long), cudaMemcpyDeviceToHost, a->stream));
  BTC_CUDA(cudaStreamSynchronize(a->stream));
  a->anorm = a->h[2];
  unsigned long long info;
  memcpy(&info, a->h + 3, sizeof(info));
  if (info != ~0ull)
    return fail(BTC_ERR_NOT_SPD, "border Schur complement not positive definite at column %d", (int)(info & 0xFFFFF));
  a->factored = true;
  return BTC_OK;
}

int btc_arrow_solve(btc_arrow_t a, const double *b, double *x, double tol, int maxit, int *iters, double *relres) {
  if (!a || !b || !x || maxit < 0) return fail(BTC_ERR_ARG, "btc_arrow_solve: invalid arguments");
  if (!a->factored) return fail(BTC_ERR_NOT_FACTORED, "btc_arrow_solve: no factorization");
  int rc = arrow_apply(a, b, x, tol, maxit, 0);
  if (rc) return rc;
  int it = 0;
  double rel = 0.0;
  for (;;) {
    if ((rc = arrow_residual(a, b, x, &rel, true))) return rc;
    if (!(rel == rel) || rel <= tol || it >= maxit) break;
    if ((rc = arrow_apply(a, a->r, x, tol, maxit, 1))) return rc;  // x += Psi_a^{-1} r
    ++it;
  }
  if (iters) *iters = it;
  if (relres) *relres = rel;
  if (!(rel <= tol)) return fail(BTC_ERR_NOT_CONVERGED, "arrow solve stopped at relative residual %.3e", rel);
  return BTC_OK;
}

int btc_arrow_free(btc_arrow_t a) {
  if (!a) return BTC_OK;
  if (a->stream || a->Z) cudaStreamSynchronize(a->stream);
  if (a->plan) btc_free(a->plan);
  for (void *q : {(void *)a->ct, (void *)a->zc, (void *)a->Z, (void *)a->part, (void *)a->S, (void *)a->z,
                  (void *)a->bp, (void *)a->r, (void *)a->d, (void *)a->yA, (void *)a->norms, (void *)a->info})
    if (q) cudaFree(q);
  if (a->h) cudaFreeHost(a->h);
  delete a;
  return BTC_OK;
}

}  // extern "C"
