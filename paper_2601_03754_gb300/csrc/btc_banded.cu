// Block-banded systems: Psi with Nb block rows of size b and lower block
// bandwidth w (Psi(i+k, i) = A_k[i] for k = 0..w, zero beyond), the wider band
// that the paper's conclusion names as an extension of the block-tridiagonal
// case.
//
// Grouping w consecutive block rows into one super-row makes Psi block
// tridiagonal with N = ceil(Nb / w) blocks of size n = w b:
//   D'_I(p, q) = Psi(Iw + p, Iw + q)         (p, q = 0..w-1: every |p - q| < w)
//   B'_I(p, q) = Psi((I+1)w + p, Iw + q)     (block distance w + p - q: nonzero for p <= q)
// It is the same matrix, so the multi-stage permutation of Sec. 4.3 applies
// to the super-rows unchanged: its separators are w consecutive block rows,
// which is what any vertex separator of a band of width w must contain. A
// ragged last super-row is padded with identity blocks (zero coupling,
// zero right-hand side), which leaves the solution unchanged.
//
// The grouping is one conversion pass on the device into plan-owned FP64
// arrays; factorization, solves and FP64 refinement are the inner plan's.
#include <cuda_runtime.h>

#include <algorithm>
#include <cstring>

#include "../../include/btc.h"
#include "btc_runtime.h"

namespace btc {

// D' [N][n][n] and B' [N-1][n][n] from the band A [w+1][Nb][b][b] (FP64). Of A_0 only the lower
// triangles are read; every other referenced block is read whole.
__global__ void k_band_group(double *Dg, double *Bg, const double *A, int Nb, int b, int w, int N) {
  grid_dep_enter();
  const int n = w * b;
  const int64_t nn = (int64_t)n * n, bb = (int64_t)b * b, slab = (int64_t)Nb * bb;
  const int64_t totalD = (int64_t)N * nn, total = totalD + (int64_t)(N - 1) * nn;
  for (int64_t q = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; q < total; q += (int64_t)gridDim.x * blockDim.x) {
    const bool diag = q < totalD;
    const int64_t t = diag ? q : q - totalD;
    const int I = (int)(t / nn);
    const int r = (int)((t / n) % n), c = (int)(t % n);
    const int p = r / b, pq = c / b, rr = r % b, cc = c % b;
    double v = 0.0;
    if (diag) {
      const int gi = I * w + p, gj = I * w + pq;
      if (gi >= Nb || gj >= Nb) {
        v = r == c ? 1.0 : 0.0;  // padding: identity
      } else if (p > pq) {
        v = A[(int64_t)(p - pq) * slab + gj * bb + rr * b + cc];  // Psi(gi, gj) = A_{gi-gj}[gj]
      } else if (p < pq) {
        v = A[(int64_t)(pq - p) * slab + gi * bb + cc * b + rr];  // Psi(gj, gi)^T
      } else {
        v = rr >= cc ? A[gj * bb + rr * b + cc] : A[gj * bb + cc * b + rr];  // A_0, lower triangle mirrored
      }
      Dg[q] = v;
    } else {
      const int gi = (I + 1) * w + p, gj = I * w + pq, d = w + p - pq;
      if (gi < Nb && d <= w) v = A[(int64_t)d * slab + gj * bb + rr * b + cc];
      Bg[t] = v;
    }
  }
}

}  // namespace btc

using namespace btc;

struct btc_banded_s {
  btc_plan_t plan = nullptr;
  int Nb = 0, b = 0, w = 0, N = 0, n = 0;
  cudaStream_t stream = nullptr;
  double *Dg = nullptr, *Bg = nullptr;   // grouped blocks
  double *rb = nullptr, *rx = nullptr;   // padded right-hand sides / solutions (ragged last super-row)
  int rcols = 0;                         // their capacity in columns
  bool factored = false;
};

namespace btc {

// Padded right-hand sides and solutions for a ragged grouping.
static int banded_vectors(btc_banded_s *a, int nrhs) {
  if (nrhs <= a->rcols) return BTC_OK;
  if (a->rb) cudaFree(a->rb);
  if (a->rx) cudaFree(a->rx);
  a->rb = a->rx = nullptr;
  a->rcols = 0;
  const size_t bytes = sizeof(double) * (size_t)a->N * a->n * nrhs;
  BTC_CUDA(cudaMalloc(&a->rb, bytes));
  BTC_CUDA(cudaMalloc(&a->rx, bytes));
  a->rcols = nrhs;
  return BTC_OK;
}

static bool banded_ragged(const btc_banded_s *a) { return (int64_t)a->Nb * a->b != (int64_t)a->N * a->n; }

// Run `solve` on the grouped system, through padded vectors when the grouping is ragged.
template <class F>
static int banded_run(btc_banded_s *a, const double *rhs, double *x, int nrhs, F solve) {
  if (!banded_ragged(a)) return solve(rhs, x);
  int rc = banded_vectors(a, nrhs);
  if (rc) return rc;
  const size_t have = sizeof(double) * (size_t)a->Nb * a->b * nrhs;
  const size_t all = sizeof(double) * (size_t)a->N * a->n * nrhs;
  BTC_CUDA(cudaMemsetAsync(a->rb, 0, all, a->stream));
  BTC_CUDA(cudaMemcpyAsync(a->rb, rhs, have, cudaMemcpyDeviceToDevice, a->stream));
  rc = solve(a->rb, a->rx);
  if (rc && rc != BTC_ERR_NOT_CONVERGED) return rc;
  BTC_CUDA(cudaMemcpyAsync(x, a->rx, have, cudaMemcpyDeviceToDevice, a->stream));
  BTC_CUDA(cudaStreamSynchronize(a->stream));
  return rc;
}

static int banded_group(btc_banded_s *a, const double *A) {
  const int64_t total = (int64_t)(2 * a->N - 1) * a->n * a->n;
  return launch_n((const void *)&k_band_group, grid_for(total), 256, 0, a->stream, a->Dg, a->Bg, A, a->Nb, a->b, a->w,
                  a->N);
}

}  // namespace btc

extern "C" {

int btc_banded_plan(btc_banded_t *out, int Nb, int b, int w, int dtype, void *stream) {
  if (!out || Nb < 1 || b < 1 || w < 1) return fail(BTC_ERR_ARG, "btc_banded_plan: invalid arguments");
  *out = nullptr;
  if (dtype == BTC_F32) return fail(BTC_ERR_ARG, "btc_banded_plan: needs an FP64 or mixed dtype (FP64 inputs)");
  btc_banded_s *a = new btc_banded_s();
  a->Nb = Nb;
  a->b = b;
  a->w = w;
  a->N = (Nb + w - 1) / w;
  a->n = w * b;
  a->stream = (cudaStream_t)stream;
  auto cleanup = [&](int code) {
    btc_banded_free(a);
    return code;
  };
  int rc = btc_plan(&a->plan, a->N, a->n, dtype, stream);
  if (rc) return cleanup(rc);
  const size_t nn = (size_t)a->n * a->n;
  cudaError_t e;
  if ((e = cudaMalloc(&a->Dg, sizeof(double) * nn * a->N)) != cudaSuccess ||
      (e = cudaMalloc(&a->Bg, sizeof(double) * nn * std::max(a->N - 1, 1))) != cudaSuccess)
    return cleanup(fail(e == cudaErrorMemoryAllocation ? BTC_ERR_OOM : BTC_ERR_CUDA, "btc_banded_plan: %s",
                        cudaGetErrorString(e)));
  *out = a;
  return BTC_OK;
}

btc_plan_t btc_banded_inner(btc_banded_t a) { return a ? a->plan : nullptr; }

int btc_banded_factor(btc_banded_t a, const double *A) {
  if (!a || !A) return fail(BTC_ERR_ARG, "btc_banded_factor: NULL argument");
  a->factored = false;
  int rc = banded_group(a, A);
  if (rc || (rc = btc_factor(a->plan, a->Dg, a->Bg))) return rc;
  int blk = -1, col = -1;
  if ((rc = btc_info(a->plan, &blk, &col)))
    return rc == BTC_ERR_NOT_SPD
               ? fail(rc, "pivot of block row %d, column %d not positive", blk * a->w + col / a->b, col % a->b)
               : rc;
  a->factored = true;
  return BTC_OK;
}

int btc_banded_solve_refined(btc_banded_t a, const double *rhs, double *x, int nrhs, double tol, int maxit,
                             int *iters, double *relres) {
  if (!a || !rhs || !x || nrhs < 1 || maxit < 0) return fail(BTC_ERR_ARG, "btc_banded_solve_refined: arguments");
  if (!a->factored) return fail(BTC_ERR_NOT_FACTORED, "btc_banded_solve_refined: no factorization");
  return banded_run(a, rhs, x, nrhs, [&](const double *r, double *y) {
    return btc_solve_refined(a->plan, r, y, nrhs, tol, maxit, iters, relres);
  });
}

int btc_banded_factor_solve_refined(btc_banded_t a, const double *A, const double *rhs, double *x, int nrhs,
                                    double tol, int maxit, int *iters, double *relres) {
  if (!a || !A || !rhs || !x || nrhs < 1 || maxit < 0)
    return fail(BTC_ERR_ARG, "btc_banded_factor_solve_refined: arguments");
  a->factored = false;
  int rc = banded_group(a, A);
  if (rc) return rc;
  rc = banded_run(a, rhs, x, nrhs, [&](const double *r, double *y) {
    return btc_factor_solve_refined(a->plan, a->Dg, a->Bg, r, y, nrhs, tol, maxit, iters, relres);
  });
  if (rc == BTC_ERR_NOT_SPD) {
    int blk = -1, col = -1;
    btc_info(a->plan, &blk, &col);
    return fail(rc, "pivot of block row %d, column %d not positive", blk * a->w + col / a->b, col % a->b);
  }
  if (rc == BTC_OK || rc == BTC_ERR_NOT_CONVERGED) a->factored = true;
  return rc;
}

int btc_banded_grouped(btc_banded_t a, double *D, double *B, int *N, int *n) {
  if (!a) return fail(BTC_ERR_ARG, "btc_banded_grouped: NULL handle");
  const size_t nn = (size_t)a->n * a->n;
  BTC_CUDA(cudaStreamSynchronize(a->stream));
  if (D) BTC_CUDA(cudaMemcpy(D, a->Dg, sizeof(double) * nn * a->N, cudaMemcpyDefault));
  if (B && a->N > 1) BTC_CUDA(cudaMemcpy(B, a->Bg, sizeof(double) * nn * (a->N - 1), cudaMemcpyDefault));
  if (N) *N = a->N;
  if (n) *n = a->n;
  return BTC_OK;
}

int btc_banded_free(btc_banded_t a) {
  if (!a) return BTC_OK;
  if (a->stream || a->Dg) cudaStreamSynchronize(a->stream);
  if (a->plan) btc_free(a->plan);
  for (void *q : {(void *)a->Dg, (void *)a->Bg, (void *)a->rb, (void *)a->rx})
    if (q) cudaFree(q);
  delete a;
  return BTC_OK;
}

}  // extern "C"
