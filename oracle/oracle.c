/*
 * Reference oracle for block-tridiagonal Cholesky factor + solve (FP64, CPU).
 *
 * TEST INFRASTRUCTURE ONLY. Nothing in the product path may call this code:
 * only the test suite, the smoke check and the CPU-baseline leg of the
 * benchmark load it. It shares no source, header or helper with the CUDA
 * library; the two meet only through the seeded input generator.
 *
 * Everything here is a plain, slow, obviously-correct restatement of a textbook
 * definition, in double precision, row-major, with no blocking, fusion or
 * reordering beyond what the definition states:
 *
 *   orc_chol            unblocked Cholesky-Crout of one dense SPD matrix
 *                       (the `chol` of Sec. 3 / Table 1 "potrf").
 *   orc_seq_factor      Alg. 1 (Sec. 3): natural-order block factorization
 *                       D^_1 = chol(D_1); E^_{i-1} = E_{i-1} D^_{i-1}^{-T};
 *                       D^_i = chol(D_i - E^_{i-1} E^_{i-1}^T).
 *   orc_seq_solve       forward/back substitution with that block-bidiagonal
 *                       factor (standard; the paper does not print it).
 *   orc_assemble        the dense (Nn)x(Nn) matrix Psi of Sec. 3.
 *   orc_dense_chol      orc_chol applied to the assembled matrix.
 *   orc_gepp_solve      Gaussian elimination with partial pivoting (brute
 *                       force solution for tiny inputs).
 *   orc_nd_order        the multi-stage (nested-dissection) elimination order
 *                       P_inf of Sec. 4.3: s = 1,2,4,...; nodes s,3s,5s,...
 *   orc_bs_chol         right-looking ("submatrix") block Cholesky of
 *                       P Psi P^T for ANY elimination order (Fig. 1, left,
 *                       applied to n x n blocks), creating fill blocks when a
 *                       structurally-zero block receives an update.
 *   orc_bs_reconstruct  ||P Psi P^T - L L^T||_F / ||Psi||_F, block-sparse.
 *   orc_resid           ||b - Psi x||_inf, ||Psi||_inf, ||x||_inf.
 *   orc_arrow_assemble  the dense bordered ("arrow") matrix [[Psi, C^T], [C, A]]
 *                       of the arrow structures that Sec. 4.3 names as a
 *                       natural extension of the permuted Cholesky view (and
 *                       the conclusion as future work); C is m x (N n), A is
 *                       m x m (lower triangle read).
 *   orc_arrow_resid     ||b - Psi_a x||_inf, ||Psi_a||_inf, ||x||_inf for it.
 *   orc_band_assemble   the dense block-banded matrix with lower block
 *                       bandwidth w, Psi(i+k, i) = A_k[i] (k = 0..w), the
 *                       wider band the conclusion names as future work.
 *   orc_band_resid      ||b - Psi x||_inf, ||Psi||_inf, ||x||_inf for it,
 *                       block by block without assembling.
 *
 * Conventions: blocks are n x n, row-major. D holds N diagonal blocks (only
 * the lower triangle of each is read; the upper triangle is taken to be its
 * mirror). B holds N-1 sub-diagonal blocks, B_i = Psi(i+1, i) (the paper's
 * E_i). Node indices in public arguments are 0-based.
 */
#include <math.h>
#include <stdlib.h>
#include <string.h>

/* Element (r, c) of the symmetric block D_i read from its lower triangle. */
static double sym_lower(const double *Di, int n, int r, int c) {
  return r >= c ? Di[r * n + c] : Di[c * n + r];
}

/*
 * Cholesky-Crout: for column j, L_jj = sqrt(a_jj - sum_{k<j} L_jk^2) and
 * L_ij = (a_ij - sum_{k<j} L_ik L_jk) / L_jj for i > j.
 * Reads only the lower triangle of A (lda); writes the full L (upper = 0).
 * Returns 0, or j+1 for the first column whose pivot is not positive.
 */
int orc_chol(int n, const double *A, int lda, double *L, int ldl) {
  for (int i = 0; i < n; ++i)
    for (int j = 0; j < n; ++j) L[i * ldl + j] = 0.0;
  for (int j = 0; j < n; ++j) {
    double d = A[j * lda + j];
    for (int k = 0; k < j; ++k) d -= L[j * ldl + k] * L[j * ldl + k];
    if (!(d > 0.0)) return j + 1;
    double ljj = sqrt(d);
    L[j * ldl + j] = ljj;
    for (int i = j + 1; i < n; ++i) {
      double v = A[i * lda + j];
      for (int k = 0; k < j; ++k) v -= L[i * ldl + k] * L[j * ldl + k];
      L[i * ldl + j] = v / ljj;
    }
  }
  return 0;
}

/* X <- X L^{-T} for an m x n X and an n x n lower-triangular L: each row x of
 * X solves  y L^T = x,  i.e. y_j = (x_j - sum_{k<j} y_k L_jk) / L_jj. */
static void trsm_right_lower_t(int m, int n, const double *L, double *X) {
  for (int r = 0; r < m; ++r) {
    double *x = X + (size_t)r * n;
    for (int j = 0; j < n; ++j) {
      double v = x[j];
      for (int k = 0; k < j; ++k) v -= x[k] * L[j * n + k];
      x[j] = v / L[j * n + j];
    }
  }
}

/* C <- C - A B^T for n x n blocks. */
static void gemm_nt_sub(int n, const double *A, const double *B, double *C) {
  for (int i = 0; i < n; ++i)
    for (int j = 0; j < n; ++j) {
      double v = 0.0;
      for (int k = 0; k < n; ++k) v += A[i * n + k] * B[j * n + k];
      C[i * n + j] -= v;
    }
}

/*
 * Alg. 1 (Sec. 3, "Sequential factorization of Psi").
 * Dhat: N lower-triangular blocks; Ehat: N-1 blocks, Ehat_i = L(i+1, i).
 * Returns 0, or (block index)*65536 + (column) + 1 for the first failing pivot.
 */
int orc_seq_factor(int N, int n, const double *D, const double *B, double *Dhat, double *Ehat) {
  size_t bs = (size_t)n * n;
  double *S = (double *)malloc(bs * sizeof(double));
  int info = orc_chol(n, D, n, Dhat, n);
  if (info) { free(S); return info; }
  for (int i = 1; i < N; ++i) {
    /* Ehat_{i-1} = E_{i-1} Dhat_{i-1}^{-T}   (trsm) */
    memcpy(Ehat + (i - 1) * bs, B + (i - 1) * bs, bs * sizeof(double));
    trsm_right_lower_t(n, n, Dhat + (i - 1) * bs, Ehat + (i - 1) * bs);
    /* S = D_i - Ehat_{i-1} Ehat_{i-1}^T        (syrk) */
    for (int r = 0; r < n; ++r)
      for (int c = 0; c < n; ++c) S[r * n + c] = sym_lower(D + i * bs, n, r, c);
    gemm_nt_sub(n, Ehat + (i - 1) * bs, Ehat + (i - 1) * bs, S);
    /* Dhat_i = chol(S)                          (potrf) */
    info = orc_chol(n, S, n, Dhat + i * bs, n);
    if (info) { free(S); return i * 65536 + info; }
  }
  free(S);
  return 0;
}

/*
 * Solve Psi X = Bv with the Alg. 1 factor, for m right-hand sides.
 * x is (N n) x m row-major: on entry the right-hand sides, on exit the solution.
 * Forward:  y_1 = Dhat_1^{-1} b_1,  y_i = Dhat_i^{-1} (b_i - Ehat_{i-1} y_{i-1}).
 * Backward: x_N = Dhat_N^{-T} y_N,  x_i = Dhat_i^{-T} (y_i - Ehat_i^T x_{i+1}).
 */
void orc_seq_solve(int N, int n, int m, const double *Dhat, const double *Ehat, double *x) {
  size_t bs = (size_t)n * n;
  for (int i = 0; i < N; ++i) {
    double *xi = x + (size_t)i * n * m;
    if (i > 0) {
      const double *E = Ehat + (i - 1) * bs;
      const double *xp = x + (size_t)(i - 1) * n * m;
      for (int r = 0; r < n; ++r)
        for (int c = 0; c < m; ++c) {
          double v = 0.0;
          for (int k = 0; k < n; ++k) v += E[r * n + k] * xp[k * m + c];
          xi[r * m + c] -= v;
        }
    }
    const double *L = Dhat + i * bs;
    for (int c = 0; c < m; ++c)
      for (int r = 0; r < n; ++r) {
        double v = xi[r * m + c];
        for (int k = 0; k < r; ++k) v -= L[r * n + k] * xi[k * m + c];
        xi[r * m + c] = v / L[r * n + r];
      }
  }
  for (int i = N - 1; i >= 0; --i) {
    double *xi = x + (size_t)i * n * m;
    if (i < N - 1) {
      const double *E = Ehat + i * bs;
      const double *xn = x + (size_t)(i + 1) * n * m;
      for (int r = 0; r < n; ++r)
        for (int c = 0; c < m; ++c) {
          double v = 0.0;
          for (int k = 0; k < n; ++k) v += E[k * n + r] * xn[k * m + c];
          xi[r * m + c] -= v;
        }
    }
    const double *L = Dhat + i * bs;
    for (int c = 0; c < m; ++c)
      for (int r = n - 1; r >= 0; --r) {
        double v = xi[r * m + c];
        for (int k = r + 1; k < n; ++k) v -= L[k * n + r] * xi[k * m + c];
        xi[r * m + c] = v / L[r * n + r];
      }
  }
}

/* Dense symmetric Psi (M = N n), from D's lower triangles and B. */
void orc_assemble(int N, int n, const double *D, const double *B, double *A) {
  int M = N * n;
  size_t bs = (size_t)n * n;
  memset(A, 0, (size_t)M * M * sizeof(double));
  for (int i = 0; i < N; ++i)
    for (int r = 0; r < n; ++r)
      for (int c = 0; c < n; ++c) A[(size_t)(i * n + r) * M + i * n + c] = sym_lower(D + i * bs, n, r, c);
  for (int i = 0; i + 1 < N; ++i)
    for (int r = 0; r < n; ++r)
      for (int c = 0; c < n; ++c) {
        double v = B[i * bs + r * n + c];
        A[(size_t)((i + 1) * n + r) * M + i * n + c] = v;
        A[(size_t)(i * n + c) * M + (i + 1) * n + r] = v;
      }
}

int orc_dense_chol(int M, const double *A, double *L) { return orc_chol(M, A, M, L, M); }

/* Gaussian elimination with partial pivoting on [A | b]; x is M x m. */
int orc_gepp_solve(int M, int m, const double *A, const double *b, double *x) {
  int W = M + m;
  double *T = (double *)malloc((size_t)M * W * sizeof(double));
  for (int i = 0; i < M; ++i) {
    for (int j = 0; j < M; ++j) T[(size_t)i * W + j] = A[(size_t)i * M + j];
    for (int j = 0; j < m; ++j) T[(size_t)i * W + M + j] = b[(size_t)i * m + j];
  }
  for (int k = 0; k < M; ++k) {
    int p = k;
    for (int i = k + 1; i < M; ++i)
      if (fabs(T[(size_t)i * W + k]) > fabs(T[(size_t)p * W + k])) p = i;
    if (T[(size_t)p * W + k] == 0.0) { free(T); return k + 1; }
    if (p != k)
      for (int j = 0; j < W; ++j) {
        double t = T[(size_t)k * W + j];
        T[(size_t)k * W + j] = T[(size_t)p * W + j];
        T[(size_t)p * W + j] = t;
      }
    for (int i = k + 1; i < M; ++i) {
      double f = T[(size_t)i * W + k] / T[(size_t)k * W + k];
      for (int j = k; j < W; ++j) T[(size_t)i * W + j] -= f * T[(size_t)k * W + j];
    }
  }
  for (int c = 0; c < m; ++c)
    for (int i = M - 1; i >= 0; --i) {
      double v = T[(size_t)i * W + M + c];
      for (int j = i + 1; j < M; ++j) v -= T[(size_t)i * W + j] * x[(size_t)j * m + c];
      x[(size_t)i * m + c] = v / T[(size_t)i * W + i];
    }
  free(T);
  return 0;
}

/*
 * Multi-stage permutation P_inf (Sec. 4.3): eliminate, for s = 1, 2, 4, ...,
 * the 1-based nodes s, 3s, 5s, ... <= N. Writes the 0-based node of each
 * elimination step into order[0..N-1]; returns the number of levels.
 */
int orc_nd_order(int N, int *order) {
  int pos = 0, levels = 0;
  for (long s = 1; s <= N; s *= 2) {
    for (long i = s; i <= N; i += 2 * s) order[pos++] = (int)(i - 1);
    ++levels;
  }
  return levels;
}

/*
 * Block-sparse right-looking Cholesky of P Psi P^T for an arbitrary
 * elimination order (order[t] = node eliminated at step t, 0-based).
 * Working storage is an N x N table of block pointers in *elimination
 * position* space, lower triangle only (row position > column position);
 * a NULL entry is a structural zero. For each step k (Fig. 1, left):
 *     A_kk <- chol(A_kk)
 *     A_ik <- A_ik A_kk^{-T}             for every nonzero A_ik, i > k
 *     A_ij <- A_ij - A_ik A_jk^T         for every pair of nonzeros i >= j > k
 *                                        (allocating A_ij if it was zero: fill)
 * Outputs, indexed by NODE: Ldiag[node] = L(node, node). Off-diagonal nonzero
 * blocks are listed as (row node, column node) pairs with the block
 * L(row, col) (row eliminated after col), at most `cap` of them.
 * Returns: number of off-diagonal blocks (>= 0); -1 if cap is too small;
 * -(2 + step*65536 + col) for a non-positive pivot.
 */
int orc_bs_chol(int N, int n, const int *order, const double *D, const double *B, double *Ldiag, int cap,
                int *pairs, double *Loff) {
  size_t bs = (size_t)n * n;
  int *pos = (int *)malloc(N * sizeof(int));
  double **T = (double **)calloc((size_t)N * N, sizeof(double *));
  double *tmp = (double *)malloc(bs * sizeof(double));
  for (int t = 0; t < N; ++t) pos[order[t]] = t;
  /* scatter Psi into position space */
  for (int i = 0; i < N; ++i) {
    double *blk = (double *)malloc(bs * sizeof(double));
    for (int r = 0; r < n; ++r)
      for (int c = 0; c < n; ++c) blk[r * n + c] = sym_lower(D + i * bs, n, r, c);
    T[(size_t)pos[i] * N + pos[i]] = blk;
  }
  for (int i = 0; i + 1 < N; ++i) {
    /* B_i = Psi(i+1, i); stored at (max pos, min pos) in the orientation of that position pair */
    int p = pos[i + 1], q = pos[i];
    double *blk = (double *)malloc(bs * sizeof(double));
    for (int r = 0; r < n; ++r)
      for (int c = 0; c < n; ++c) blk[r * n + c] = p > q ? B[i * bs + r * n + c] : B[i * bs + c * n + r];
    if (p > q) T[(size_t)p * N + q] = blk;
    else T[(size_t)q * N + p] = blk;
  }
  int ret = 0;
  int *nz = (int *)malloc(N * sizeof(int));
  for (int k = 0; k < N && ret == 0; ++k) {
    double *Akk = T[(size_t)k * N + k];
    int info = orc_chol(n, Akk, n, tmp, n);
    if (info) { ret = -(2 + k * 65536 + (info - 1)); break; }
    memcpy(Akk, tmp, bs * sizeof(double));
    int cnt = 0;
    for (int i = k + 1; i < N; ++i)
      if (T[(size_t)i * N + k]) {
        trsm_right_lower_t(n, n, Akk, T[(size_t)i * N + k]);
        nz[cnt++] = i;
      }
    for (int a = 0; a < cnt; ++a)
      for (int b = 0; b <= a; ++b) {
        int i = nz[a], j = nz[b]; /* i >= j since nz is increasing */
        double **slot = &T[(size_t)i * N + j];
        if (!*slot) *slot = (double *)calloc(bs, sizeof(double));
        gemm_nt_sub(n, T[(size_t)i * N + k], T[(size_t)j * N + k], *slot);
      }
  }
  if (ret == 0) {
    int cntoff = 0;
    for (int t = 0; t < N; ++t) memcpy(Ldiag + (size_t)order[t] * bs, T[(size_t)t * N + t], bs * sizeof(double));
    for (int i = 0; i < N && ret == 0; ++i)
      for (int j = 0; j < i; ++j)
        if (T[(size_t)i * N + j]) {
          if (cntoff >= cap) { ret = -1; break; }
          pairs[2 * cntoff] = order[i];
          pairs[2 * cntoff + 1] = order[j];
          memcpy(Loff + (size_t)cntoff * bs, T[(size_t)i * N + j], bs * sizeof(double));
          ++cntoff;
        }
    if (ret == 0) ret = cntoff;
  }
  for (size_t e = 0; e < (size_t)N * N; ++e) free(T[e]);
  free(T); free(pos); free(tmp); free(nz);
  return ret;
}

/*
 * ||P Psi P^T - L L^T||_F / ||Psi||_F for a block-sparse factor given as
 * (Ldiag by node, list of (row node, col node, block)), with `order` the
 * elimination order. (L L^T)(p, q) = sum over columns c of L(p,c) L(q,c)^T.
 */
double orc_bs_reconstruct(int N, int n, const int *order, const double *D, const double *B, const double *Ldiag,
                          int nnz, const int *pairs, const double *Loff) {
  size_t bs = (size_t)n * n;
  int *pos = (int *)malloc(N * sizeof(int));
  for (int t = 0; t < N; ++t) pos[order[t]] = t;
  /* column lists in position space: for each column position, the (row pos, block ptr) entries incl. diagonal */
  int *colcnt = (int *)calloc(N, sizeof(int));
  for (int e = 0; e < nnz; ++e) colcnt[pos[pairs[2 * e + 1]]]++;
  int *colstart = (int *)malloc((N + 1) * sizeof(int));
  colstart[0] = 0;
  for (int c = 0; c < N; ++c) colstart[c + 1] = colstart[c] + colcnt[c] + 1;
  int *rowpos = (int *)malloc(colstart[N] * sizeof(int));
  const double **blk = (const double **)malloc(colstart[N] * sizeof(double *));
  int *fillp = (int *)calloc(N, sizeof(int));
  for (int t = 0; t < N; ++t) {
    rowpos[colstart[t]] = t;
    blk[colstart[t]] = Ldiag + (size_t)order[t] * bs;
    fillp[t] = 1;
  }
  for (int e = 0; e < nnz; ++e) {
    int c = pos[pairs[2 * e + 1]];
    int k = colstart[c] + fillp[c]++;
    rowpos[k] = pos[pairs[2 * e]];
    blk[k] = Loff + (size_t)e * bs;
  }
  /* accumulate LL^T into a hash-free dense-by-block map of the lower part: use an N x N pointer table */
  double **P = (double **)calloc((size_t)N * N, sizeof(double *));
  for (int c = 0; c < N; ++c)
    for (int a = colstart[c]; a < colstart[c + 1]; ++a)
      for (int b = colstart[c]; b < colstart[c + 1]; ++b) {
        int p = rowpos[a], q = rowpos[b];
        if (p < q) continue;
        double **slot = &P[(size_t)p * N + q];
        if (!*slot) *slot = (double *)calloc(bs, sizeof(double));
        for (int r = 0; r < n; ++r)
          for (int s = 0; s < n; ++s) {
            double v = 0.0;
            for (int k = 0; k < n; ++k) v += blk[a][r * n + k] * blk[b][s * n + k];
            (*slot)[r * n + s] += v;
          }
      }
  /* subtract P Psi P^T on the lower part, accumulate Frobenius norms (off-diagonal blocks counted twice) */
  double num = 0.0, den = 0.0;
  double *ref = (double *)malloc(bs * sizeof(double));
  for (int p = 0; p < N; ++p)
    for (int q = 0; q <= p; ++q) {
      int i = order[p], j = order[q];
      int have = 0;
      if (i == j) {
        for (int r = 0; r < n; ++r)
          for (int s = 0; s < n; ++s) ref[r * n + s] = sym_lower(D + i * bs, n, r, s);
        have = 1;
      } else if (i == j + 1) {
        memcpy(ref, B + j * bs, bs * sizeof(double));
        have = 1;
      } else if (j == i + 1) {
        for (int r = 0; r < n; ++r)
          for (int s = 0; s < n; ++s) ref[r * n + s] = B[i * bs + s * n + r];
        have = 1;
      }
      const double *got = P[(size_t)p * N + q];
      if (!have && !got) continue;
      double w = (p == q) ? 1.0 : 2.0;
      for (int e = 0; e < (int)bs; ++e) {
        double a = have ? ref[e] : 0.0;
        double g = got ? got[e] : 0.0;
        num += w * (a - g) * (a - g);
        den += w * a * a;
      }
    }
  for (size_t e = 0; e < (size_t)N * N; ++e) free(P[e]);
  free(P); free(ref); free(pos); free(colcnt); free(colstart); free(rowpos); free(blk); free(fillp);
  return sqrt(num) / sqrt(den);
}

/*
 * out[0] = ||b - Psi x||_inf, out[1] = ||Psi||_inf (max absolute row sum),
 * out[2] = ||x||_inf; x and b are (N n) x m row-major; the infinity norms of
 * the m-column blocks are the maxima over columns.
 */
void orc_resid(int N, int n, int m, const double *D, const double *B, const double *x, const double *b,
               double *out) {
  size_t bs = (size_t)n * n;
  double rmax = 0.0, amax = 0.0, xmax = 0.0;
  for (int i = 0; i < N; ++i)
    for (int r = 0; r < n; ++r) {
      double rowsum = 0.0;
      for (int c = 0; c < n; ++c) rowsum += fabs(sym_lower(D + i * bs, n, r, c));
      if (i > 0)
        for (int c = 0; c < n; ++c) rowsum += fabs(B[(i - 1) * bs + r * n + c]);
      if (i + 1 < N)
        for (int c = 0; c < n; ++c) rowsum += fabs(B[i * bs + c * n + r]);
      if (rowsum > amax) amax = rowsum;
      for (int col = 0; col < m; ++col) {
        double v = b[((size_t)i * n + r) * m + col];
        for (int c = 0; c < n; ++c) v -= sym_lower(D + i * bs, n, r, c) * x[((size_t)i * n + c) * m + col];
        if (i > 0)
          for (int c = 0; c < n; ++c) v -= B[(i - 1) * bs + r * n + c] * x[((size_t)(i - 1) * n + c) * m + col];
        if (i + 1 < N)
          for (int c = 0; c < n; ++c) v -= B[i * bs + c * n + r] * x[((size_t)(i + 1) * n + c) * m + col];
        if (fabs(v) > rmax) rmax = fabs(v);
        double xv = fabs(x[((size_t)i * n + r) * m + col]);
        if (xv > xmax) xmax = xv;
      }
    }
  out[0] = rmax;
  out[1] = amax;
  out[2] = xmax;
}

/*
 * Dense bordered matrix of size (N n + m): Psi (orc_assemble) in the leading
 * block, C (m x N n, row-major) in the last m rows, C^T in the last m columns
 * and A (lower triangle read, mirrored) in the trailing m x m block.
 */
void orc_arrow_assemble(int N, int n, int m, const double *D, const double *B, const double *C, const double *A,
                        double *out) {
  const int L = N * n, M = L + m;
  double *T = (double *)calloc((size_t)L * L, sizeof(double));
  orc_assemble(N, n, D, B, T);
  memset(out, 0, sizeof(double) * (size_t)M * M);
  for (int i = 0; i < L; ++i)
    for (int j = 0; j < L; ++j) out[(size_t)i * M + j] = T[(size_t)i * L + j];
  for (int r = 0; r < m; ++r)
    for (int j = 0; j < L; ++j) {
      out[(size_t)(L + r) * M + j] = C[(size_t)r * L + j];
      out[(size_t)j * M + L + r] = C[(size_t)r * L + j];
    }
  for (int r = 0; r < m; ++r)
    for (int c = 0; c < m; ++c) out[(size_t)(L + r) * M + L + c] = sym_lower(A, m, r, c);
  free(T);
}

/*
 * out[0] = ||b - Psi_a x||_inf, out[1] = ||Psi_a||_inf, out[2] = ||x||_inf for
 * the bordered matrix, one right-hand side of length N n + m, without forming
 * it: the block-tridiagonal rows add the coupling columns C^T, the last m rows
 * are C and A.
 */
void orc_arrow_resid(int N, int n, int m, const double *D, const double *B, const double *C, const double *A,
                     const double *x, const double *b, double *out) {
  const int L = N * n;
  size_t bs = (size_t)n * n;
  double rmax = 0.0, amax = 0.0, xmax = 0.0;
  for (int i = 0; i < N; ++i)
    for (int r = 0; r < n; ++r) {
      const int row = i * n + r;
      double rowsum = 0.0, v = b[row];
      for (int c = 0; c < n; ++c) {
        const double a = sym_lower(D + i * bs, n, r, c);
        rowsum += fabs(a);
        v -= a * x[i * n + c];
      }
      if (i > 0)
        for (int c = 0; c < n; ++c) {
          const double a = B[(i - 1) * bs + r * n + c];
          rowsum += fabs(a);
          v -= a * x[(i - 1) * n + c];
        }
      if (i + 1 < N)
        for (int c = 0; c < n; ++c) {
          const double a = B[i * bs + c * n + r];
          rowsum += fabs(a);
          v -= a * x[(i + 1) * n + c];
        }
      for (int q = 0; q < m; ++q) {
        const double a = C[(size_t)q * L + row];
        rowsum += fabs(a);
        v -= a * x[L + q];
      }
      if (rowsum > amax) amax = rowsum;
      if (fabs(v) > rmax) rmax = fabs(v);
      if (fabs(x[row]) > xmax) xmax = fabs(x[row]);
    }
  for (int q = 0; q < m; ++q) {
    double rowsum = 0.0, v = b[L + q];
    for (int j = 0; j < L; ++j) {
      rowsum += fabs(C[(size_t)q * L + j]);
      v -= C[(size_t)q * L + j] * x[j];
    }
    for (int c = 0; c < m; ++c) {
      const double a = sym_lower(A, m, q, c);
      rowsum += fabs(a);
      v -= a * x[L + c];
    }
    if (rowsum > amax) amax = rowsum;
    if (fabs(v) > rmax) rmax = fabs(v);
    if (fabs(x[L + q]) > xmax) xmax = fabs(x[L + q]);
  }
  out[0] = rmax;
  out[1] = amax;
  out[2] = xmax;
}

/*
 * Block-banded Psi: Nb block rows of size b, lower block bandwidth w. The band
 * is A [w+1][Nb][b][b] with A_k[i] = Psi(i+k, i); blocks with i + k >= Nb are
 * outside the matrix and not read, and of A_0 only the lower triangles are
 * read. Element (row, col) of block (I, J) with |I - J| <= w.
 */
static double band_elem(int Nb, int b, const double *A, int I, int J, int r, int c) {
  const size_t bb = (size_t)b * b;
  if (I == J) return sym_lower(A + (size_t)I * bb, b, r, c);
  if (I > J) return A[((size_t)(I - J) * Nb + J) * bb + (size_t)r * b + c];
  return A[((size_t)(J - I) * Nb + I) * bb + (size_t)c * b + r]; /* Psi(I, J) = Psi(J, I)^T */
}

/* The dense (Nb b) x (Nb b) matrix. */
void orc_band_assemble(int Nb, int b, int w, const double *A, double *out) {
  const size_t L = (size_t)Nb * b;
  for (size_t q = 0; q < L * L; ++q) out[q] = 0.0;
  for (int I = 0; I < Nb; ++I)
    for (int J = I - w; J <= I + w; ++J) {
      if (J < 0 || J >= Nb) continue;
      for (int r = 0; r < b; ++r)
        for (int c = 0; c < b; ++c) out[((size_t)I * b + r) * L + (size_t)J * b + c] = band_elem(Nb, b, A, I, J, r, c);
    }
}

/* out = (||b - Psi x||_inf, ||Psi||_inf, ||x||_inf), maxima over the m columns
 * of x and b ([Nb b][m], row-major). */
void orc_band_resid(int Nb, int b, int w, int m, const double *A, const double *x, const double *rhs, double *out) {
  double rmax = 0.0, amax = 0.0, xmax = 0.0;
  for (int I = 0; I < Nb; ++I)
    for (int r = 0; r < b; ++r) {
      const size_t row = (size_t)I * b + r;
      double rowsum = 0.0;
      for (int J = I - w; J <= I + w; ++J) {
        if (J < 0 || J >= Nb) continue;
        for (int c = 0; c < b; ++c) rowsum += fabs(band_elem(Nb, b, A, I, J, r, c));
      }
      if (rowsum > amax) amax = rowsum;
      for (int q = 0; q < m; ++q) {
        double v = rhs[row * m + q];
        for (int J = I - w; J <= I + w; ++J) {
          if (J < 0 || J >= Nb) continue;
          for (int c = 0; c < b; ++c) v -= band_elem(Nb, b, A, I, J, r, c) * x[((size_t)J * b + c) * m + q];
        }
        if (fabs(v) > rmax) rmax = fabs(v);
        if (fabs(x[row * m + q]) > xmax) xmax = fabs(x[row * m + q]);
      }
    }
  out[0] = rmax;
  out[1] = amax;
  out[2] = xmax;
}
