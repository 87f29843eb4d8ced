// Register-tiled block operations on one padded np x np block per CTA.
//
// Thread layout: the CTA's NT = (NP/R)^2 threads form a (NP/R) x (NP/R) grid;
// thread (ty, tx) owns the R x R tile of rows [ty*R, ty*R+R) and columns
// [tx*R, tx*R+R) of every np x np operand and keeps it in registers.
// Shared-memory copies of blocks use a padded leading dimension LD so that the
// row reads of the X^T Y products and the transposed writes are bank-conflict
// free (rows stay 16-byte aligned).
#pragma once
#include <cuda_runtime.h>
#include <stdint.h>

namespace btc {

template <typename T, int NP_, int R_>
struct TileCfg {
  static constexpr int NP = NP_;
  static constexpr int R = R_;
  static constexpr int TXN = NP / R;
  static constexpr int NT = TXN * TXN;
  static constexpr int PAD = sizeof(T) == 4 ? 4 : 2;
  static constexpr int LD = NP + PAD;
  static constexpr int BLK = NP * LD;  // elements of one shared-memory block
  static_assert(NP % R == 0, "tile must divide the block");
};

// ---------------------------------------------------------------- vector io
template <typename T, int R>
__device__ __forceinline__ void vload(const T *p, T (&v)[R]) {
  if constexpr (sizeof(T) * R == 16) {
    const float4 q = *reinterpret_cast<const float4 *>(p);
    const T *s = reinterpret_cast<const T *>(&q);
#pragma unroll
    for (int i = 0; i < R; ++i) v[i] = s[i];
  } else if constexpr (sizeof(T) * R == 32) {
    const float4 q0 = reinterpret_cast<const float4 *>(p)[0];
    const float4 q1 = reinterpret_cast<const float4 *>(p)[1];
    const T *s0 = reinterpret_cast<const T *>(&q0);
    const T *s1 = reinterpret_cast<const T *>(&q1);
#pragma unroll
    for (int i = 0; i < R / 2; ++i) {
      v[i] = s0[i];
      v[i + R / 2] = s1[i];
    }
  } else if constexpr (sizeof(T) * R == 8) {
    const float2 q = *reinterpret_cast<const float2 *>(p);
    const T *s = reinterpret_cast<const T *>(&q);
#pragma unroll
    for (int i = 0; i < R; ++i) v[i] = s[i];
  } else {
#pragma unroll
    for (int i = 0; i < R; ++i) v[i] = p[i];
  }
}

template <typename T, int R>
__device__ __forceinline__ void vstore(T *p, const T (&v)[R]) {
  if constexpr (sizeof(T) * R == 16) {
    float4 q;
    T *s = reinterpret_cast<T *>(&q);
#pragma unroll
    for (int i = 0; i < R; ++i) s[i] = v[i];
    *reinterpret_cast<float4 *>(p) = q;
  } else if constexpr (sizeof(T) * R == 32) {
    float4 q0, q1;
    T *s0 = reinterpret_cast<T *>(&q0);
    T *s1 = reinterpret_cast<T *>(&q1);
#pragma unroll
    for (int i = 0; i < R / 2; ++i) {
      s0[i] = v[i];
      s1[i] = v[i + R / 2];
    }
    reinterpret_cast<float4 *>(p)[0] = q0;
    reinterpret_cast<float4 *>(p)[1] = q1;
  } else if constexpr (sizeof(T) * R == 8) {
    float2 q;
    T *s = reinterpret_cast<T *>(&q);
#pragma unroll
    for (int i = 0; i < R; ++i) s[i] = v[i];
    *reinterpret_cast<float2 *>(p) = q;
  } else {
#pragma unroll
    for (int i = 0; i < R; ++i) p[i] = v[i];
  }
}

// ------------------------------------------------------------ tile transfer
// Global pool block (np x np, row-major, contiguous; element type P) -> registers (type T).
template <class C, typename T, typename P>
__device__ __forceinline__ void tile_from_pool(T (&a)[C::R][C::R], const P *g, int r0, int c0) {
#pragma unroll
  for (int r = 0; r < C::R; ++r) {
    P v[C::R];
    vload<P, C::R>(g + (size_t)(r0 + r) * C::NP + c0, v);
#pragma unroll
    for (int c = 0; c < C::R; ++c) a[r][c] = (T)v[c];
  }
}

template <class C, typename T, typename P>
__device__ __forceinline__ void tile_to_pool(P *g, const T (&a)[C::R][C::R], int r0, int c0) {
#pragma unroll
  for (int r = 0; r < C::R; ++r) {
    P v[C::R];
#pragma unroll
    for (int c = 0; c < C::R; ++c) v[c] = (P)a[r][c];
    vstore<P, C::R>(g + (size_t)(r0 + r) * C::NP + c0, v);
  }
}

template <class C, typename T>
__device__ __forceinline__ void tile_to_smem(T *s, const T (&a)[C::R][C::R], int r0, int c0) {
#pragma unroll
  for (int r = 0; r < C::R; ++r) vstore<T, C::R>(s + (r0 + r) * C::LD + c0, a[r]);
}

// User block (n x n row-major, source type S) -> registers, padded to np with
// `diag` on the padded diagonal and 0 elsewhere. trans: read element (k, i).
template <class C, typename T, typename S>
__device__ __forceinline__ void tile_from_user(T (&a)[C::R][C::R], const S *src, int n, int r0, int c0, bool trans,
                                               T diag) {
#pragma unroll
  for (int r = 0; r < C::R; ++r)
#pragma unroll
    for (int c = 0; c < C::R; ++c) {
      const int i = r0 + r, k = c0 + c;
      T v;
      if (i < n && k < n)
        v = (T)(trans ? __ldg(src + (size_t)k * n + i) : __ldg(src + (size_t)i * n + k));
      else
        v = (i == k) ? diag : T(0);
      a[r][c] = v;
    }
}

// Cooperative copy of a pool block (type P) into padded shared memory (type T).
template <class C, typename T, typename P>
__device__ __forceinline__ void block_to_smem(T *s, const P *g) {
  constexpr int V = 16 / sizeof(P);  // source elements per 16-byte chunk
  constexpr int CPR = C::NP / V;     // chunks per row
  for (int q = threadIdx.x; q < C::NP * CPR; q += C::NT) {
    const int row = q / CPR, col = (q % CPR) * V;
    const float4 raw = __ldg(reinterpret_cast<const float4 *>(g + (size_t)row * C::NP + col));
    const P *src = reinterpret_cast<const P *>(&raw);
    if constexpr (sizeof(T) == sizeof(P)) {
      *reinterpret_cast<float4 *>(s + row * C::LD + col) = raw;
    } else {
#pragma unroll
      for (int i = 0; i < V; ++i) s[row * C::LD + col + i] = (T)src[i];
    }
  }
}

// ------------------------------------------------------------ block algebra
// a -= X^T Y over k = 0..np-1 (X, Y in shared memory): a[r][c] -= sum_k X[k][r0+r] Y[k][c0+c].
template <class C, typename T>
__device__ __forceinline__ void tile_sub_xty(T (&a)[C::R][C::R], const T *X, const T *Y, int r0, int c0) {
#pragma unroll 4
  for (int k = 0; k < C::NP; ++k) {
    T x[C::R], y[C::R];
    vload<T, C::R>(X + k * C::LD + r0, x);
    vload<T, C::R>(Y + k * C::LD + c0, y);
#pragma unroll
    for (int r = 0; r < C::R; ++r)
#pragma unroll
      for (int c = 0; c < C::R; ++c) a[r][c] = fma(-x[r], y[c], a[r][c]);
  }
}

// Result of a failed pivot: packed (node, column) for an atomicMin.
__device__ __forceinline__ unsigned long long pack_info(int node, int col) {
  return ((unsigned long long)(unsigned)node << 20) | (unsigned)col;
}

// In-register Cholesky of the symmetric block held by the lower tiles (ty >= tx):
// right-looking, one column per step, one barrier per step. Step j publishes
// column j (double-buffered in colbuf[2][np]) and every owner of an element
// (i, k) with i >= k > j applies a_ik -= a_ij a_kj / a_jj; the columns are
// scaled by 1/sqrt(pivot) at the end, giving L = chol(S) in `a` (zeros above
// the diagonal). Also writes L^T into LT (shared, padded) and 1/L_jj into dinv.
// A pivot that is not positive is reported through *info and replaced by 1
// so that the remaining arithmetic stays finite.
template <class C, typename T>
__device__ __forceinline__ void tile_potrf(T (&a)[C::R][C::R], int r0, int c0, bool lower, T *colbuf, T *LT,
                                           T *dinv, unsigned long long *info, int node) {
  constexpr int R = C::R;
  T piv_own[R];
#pragma unroll
  for (int c = 0; c < R; ++c) piv_own[c] = T(1);
  for (int j = 0; j < C::NP; ++j) {
    T *cb = colbuf + (j & 1) * C::NP;
    if (lower && j >= c0 && j < c0 + R) {
#pragma unroll
      for (int r = 0; r < R; ++r)
#pragma unroll
        for (int c = 0; c < R; ++c)
          if (c0 + c == j) cb[r0 + r] = a[r][c];
    }
    __syncthreads();
    T piv = cb[j];
    if (!(piv > T(0))) {
      if (threadIdx.x == 0 && info) atomicMin(info, pack_info(node, j));
      piv = T(1);
    }
#pragma unroll
    for (int c = 0; c < R; ++c)
      if (c0 + c == j) piv_own[c] = piv;
    if (lower) {
      const T inv = T(1) / piv;
      T ci[R], ck[R];
#pragma unroll
      for (int r = 0; r < R; ++r) ci[r] = cb[r0 + r] * inv;
#pragma unroll
      for (int c = 0; c < R; ++c) ck[c] = cb[c0 + c];
#pragma unroll
      for (int r = 0; r < R; ++r)
#pragma unroll
        for (int c = 0; c < R; ++c)
          if (c0 + c > j && r0 + r >= c0 + c) a[r][c] = fma(-ci[r], ck[c], a[r][c]);
    }
  }
  // scale columns: L_ik = a_ik / sqrt(d_k), L_kk = sqrt(d_k)
  T sq[R], isq[R];
#pragma unroll
  for (int c = 0; c < R; ++c) {
    sq[c] = sqrt(piv_own[c]);
    isq[c] = T(1) / sq[c];
  }
#pragma unroll
  for (int r = 0; r < R; ++r)
#pragma unroll
    for (int c = 0; c < R; ++c) {
      const int i = r0 + r, k = c0 + c;
      T v = (i > k && lower) ? a[r][c] * isq[c] : (i == k ? sq[c] : T(0));
      a[r][c] = v;
      if (lower) LT[k * C::LD + i] = v;
    }
  if (lower && r0 == c0) {
#pragma unroll
    for (int c = 0; c < R; ++c) dinv[c0 + c] = isq[c];
  }
}

// Z <- L^{-1} Z for the np x np block Z held in registers (all tiles), with L
// given by its transpose LT and the reciprocal diagonal dinv in shared memory:
// forward substitution by rows, one barrier per row (rowbuf[2][np] double buffer).
template <class C, typename T>
__device__ __forceinline__ void tile_trsm_llnn(T (&z)[C::R][C::R], int r0, int c0, const T *LT, const T *dinv,
                                               T *rowbuf) {
  constexpr int R = C::R;
  for (int j = 0; j < C::NP; ++j) {
    T *rb = rowbuf + (j & 1) * C::NP;
    if (j >= r0 && j < r0 + R) {
      const T dj = dinv[j];
#pragma unroll
      for (int r = 0; r < R; ++r)
        if (r0 + r == j) {
#pragma unroll
          for (int c = 0; c < R; ++c) z[r][c] *= dj;
          vstore<T, R>(rb + c0, z[r]);
        }
    }
    __syncthreads();
    if (r0 + R - 1 > j) {
      T zr[R], l[R];
      vload<T, R>(rb + c0, zr);
      vload<T, R>(LT + j * C::LD + r0, l);
#pragma unroll
      for (int r = 0; r < R; ++r)
        if (r0 + r > j) {
#pragma unroll
          for (int c = 0; c < R; ++c) z[r][c] = fma(-l[r], zr[c], z[r][c]);
        }
    }
  }
}

}  // namespace btc
