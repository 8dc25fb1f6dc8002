// FP64 n x n dense routines run by one CTA inside the Gram methods' epilogues (paper
// Sec. 3.1): Cholesky (Algorithm 1, steps 2 and 4), the inverse of an upper triangle (the
// R1^{-1} applied on the fly in the second pass), the product of two upper triangles
// (R = R2 R1), the symmetric eigendecomposition of SVQB, and a Householder QR of a small
// square matrix (the R of X = Q Z).  All matrices live in shared memory, row-major with
// leading dimension ld; T is the CTA size.
#pragma once

#include "common.cuh"

namespace ql {

// Right-looking Cholesky of the upper triangle of C (in place: C <- R with R^T R = C).
// Returns 0 or the 1-based index of the first non-positive pivot (to every thread).
template <int T>
QL_DEV int chol_upper_inplace(double* C, int ld, int n, int* s_flag) {
  if (threadIdx.x == 0) *s_flag = 0;
  __syncthreads();
  for (int j = 0; j < n; ++j) {
    double d = C[j * ld + j];
    if (!(d > 0.0)) {
      __syncthreads();
      if (threadIdx.x == 0) *s_flag = j + 1;
      __syncthreads();
      return *s_flag;
    }
    double rjj = sqrt(d);
    double inv = 1.0 / rjj;
    __syncthreads();
    for (int c = j + 1 + threadIdx.x; c < n; c += T) C[j * ld + c] *= inv;
    if (threadIdx.x == 0) C[j * ld + j] = rjj;
    __syncthreads();
    int w = n - j - 1;
    int pairs = w * w;
    for (int t = threadIdx.x; t < pairs; t += T) {
      int p = j + 1 + t / w, q = j + 1 + t % w;
      if (p <= q) C[p * ld + q] = fma(-C[j * ld + p], C[j * ld + q], C[p * ld + q]);
    }
    __syncthreads();
  }
  for (int t = threadIdx.x; t < n * n; t += T)
    if (t / n > t % n) C[(t / n) * ld + t % n] = 0.0;
  __syncthreads();
  return 0;
}

// Minv <- R^{-1} for an upper triangular R with nonzero diagonal (one column per thread).
template <int T>
QL_DEV void tri_upper_inverse(const double* R, int ldr, double* Minv, int ldm, int n) {
  for (int t = threadIdx.x; t < n * n; t += T) Minv[(t / n) * ldm + t % n] = 0.0;
  __syncthreads();
  for (int c = threadIdx.x; c < n; c += T) {
    Minv[c * ldm + c] = 1.0 / R[c * ldr + c];
    for (int i = c - 1; i >= 0; --i) {
      double s = 0.0;
      for (int k = i + 1; k <= c; ++k) s = fma(R[i * ldr + k], Minv[k * ldm + c], s);
      Minv[i * ldm + c] = -s / R[i * ldr + i];
    }
  }
  __syncthreads();
}

// P <- A B for upper triangular A, B (P may not alias).
template <int T>
QL_DEV void upper_times_upper(const double* A, int lda, const double* B, int ldb, double* P, int ldp, int n) {
  for (int t = threadIdx.x; t < n * n; t += T) {
    int i = t / n, j = t % n;
    double s = 0.0;
    for (int k = i; k <= j; ++k) s = fma(A[i * lda + k], B[k * ldb + j], s);
    P[i * ldp + j] = i <= j ? s : 0.0;
  }
  __syncthreads();
}

// P <- A B for full n x n matrices.
template <int T>
QL_DEV void full_times_full(const double* A, int lda, const double* B, int ldb, double* P, int ldp, int n) {
  for (int t = threadIdx.x; t < n * n; t += T) {
    int i = t / n, j = t % n;
    double s = 0.0;
    for (int k = 0; k < n; ++k) s = fma(A[i * lda + k], B[k * ldb + j], s);
    P[i * ldp + j] = s;
  }
  __syncthreads();
}

// Cyclic two-sided Jacobi on a symmetric matrix A (full storage, overwritten): on return
// A's diagonal holds the eigenvalues and U (n x n) the eigenvectors, A_in = U diag U^T.
// Rounds follow the round-robin ("chess tournament") ordering, so the n/2 rotations of a
// round touch disjoint row/column pairs and run concurrently.  A round applies J^T A J by
// 2 x 2 blocks: block (k1, k2), k1 <= k2, holds rows {p1, q1} and columns {p2, q2} of the
// pairs k1 and k2, is rotated on both sides at once and is written together with its
// mirror image, so only half of the blocks are computed (about 2/3 of the FP64 work of
// rotating all columns, then all rows) and a round needs two barriers.  A rotated pair's
// diagonal block takes the closed form a_pp - t a_pq, a_qq + t a_pq, 0.  For odd n the
// matrix is bordered by a zero row and column (the dummy player of the ordering), which no
// rotation touches, so A and U need n + 1 rows and columns of storage then.  A pair is
// skipped when |a_pq| <= 1e-17 sqrt(|a_pp a_qq|); the loop stops after a sweep without
// rotations or after max_sweeps.  Returns the number of sweeps used.
template <int T>
QL_DEV int jacobi_eig(double* A, int ld, double* U, int ldu, int n, double* sc, int* s_flag, int max_sweeps = 30) {
  if (n < 2) {
    if (threadIdx.x == 0 && n == 1) U[0] = 1.0;
    __syncthreads();
    return 0;
  }
  const int N = (n + 1) & ~1;  // players (one dummy when n is odd)
  const int half = N / 2;
  const int nb = half * (half + 1) / 2;  // blocks k1 <= k2
  for (int e = threadIdx.x; e < N * N; e += T) {
    const int i = e / N, j = e % N;
    U[i * ldu + j] = (i == j) ? 1.0 : 0.0;
    if (i == n || j == n) A[i * ld + j] = 0.0;  // the border of odd n
  }
  int sweep = 0;
  __syncthreads();
  for (; sweep < max_sweeps; ++sweep) {
    if (threadIdx.x == 0) *s_flag = 0;
    __syncthreads();
    for (int r = 0; r < N - 1; ++r) {
      // rotation parameters, one thread per pair: c, s, t and the pair (p << 8 | q)
      for (int k = threadIdx.x; k < half; k += T) {
        const int a = (k == 0) ? 0 : 1 + (k - 1 + r) % (N - 1);
        const int b = 1 + (N - 2 - k + r) % (N - 1);
        const int p = a < b ? a : b, q = a < b ? b : a;
        double c = 1.0, s = 0.0, t = 0.0;
        const double apq = A[p * ld + q], app = A[p * ld + p], aqq = A[q * ld + q];
        if (apq != 0.0 && fabs(apq) > 1e-17 * sqrt(fabs(app * aqq))) {
          const double tau = (aqq - app) / (2.0 * apq);
          t = (tau >= 0.0 ? 1.0 : -1.0) / (fabs(tau) + sqrt(1.0 + tau * tau));
          c = 1.0 / sqrt(1.0 + t * t);
          s = t * c;
          *s_flag = 1;
        }
        sc[4 * k + 0] = c;
        sc[4 * k + 1] = s;
        sc[4 * k + 2] = t;
        sc[4 * k + 3] = (double)((p << 8) | q);
      }
      __syncthreads();
      // A <- J^T A J by blocks (first nb work items), U <- U J by (pair, row) (the rest)
      for (int w = threadIdx.x; w < nb + half * N; w += T) {
        if (w < nb) {
          int k2 = (int)((sqrtf(8.0f * (float)w + 1.0f) - 1.0f) * 0.5f);
          while (k2 * (k2 + 1) / 2 > w) --k2;
          while ((k2 + 1) * (k2 + 2) / 2 <= w) ++k2;
          const int k1 = w - k2 * (k2 + 1) / 2;
          const double s1 = sc[4 * k1 + 1], s2 = sc[4 * k2 + 1];
          const int pq1 = (int)sc[4 * k1 + 3], pq2 = (int)sc[4 * k2 + 3];
          const int p1 = pq1 >> 8, q1 = pq1 & 255, p2 = pq2 >> 8, q2 = pq2 & 255;
          if (k1 == k2) {
            if (s1 != 0.0) {
              const double t1 = sc[4 * k1 + 2], apq = A[p1 * ld + q1];
              A[p1 * ld + p1] = fma(-t1, apq, A[p1 * ld + p1]);
              A[q1 * ld + q1] = fma(t1, apq, A[q1 * ld + q1]);
              A[p1 * ld + q1] = 0.0;
              A[q1 * ld + p1] = 0.0;
            }
          } else if (s1 != 0.0 || s2 != 0.0) {
            double b00 = A[p1 * ld + p2], b01 = A[p1 * ld + q2], b10 = A[q1 * ld + p2], b11 = A[q1 * ld + q2];
            if (s2 != 0.0) {  // columns p2, q2
              const double c2 = sc[4 * k2];
              const double x0 = b00, x1 = b10;
              b00 = c2 * x0 - s2 * b01;
              b01 = s2 * x0 + c2 * b01;
              b10 = c2 * x1 - s2 * b11;
              b11 = s2 * x1 + c2 * b11;
            }
            if (s1 != 0.0) {  // rows p1, q1
              const double c1 = sc[4 * k1];
              const double y0 = b00, y1 = b01;
              b00 = c1 * y0 - s1 * b10;
              b10 = s1 * y0 + c1 * b10;
              b01 = c1 * y1 - s1 * b11;
              b11 = s1 * y1 + c1 * b11;
            }
            A[p1 * ld + p2] = b00;
            A[p2 * ld + p1] = b00;
            A[p1 * ld + q2] = b01;
            A[q2 * ld + p1] = b01;
            A[q1 * ld + p2] = b10;
            A[p2 * ld + q1] = b10;
            A[q1 * ld + q2] = b11;
            A[q2 * ld + q1] = b11;
          }
        } else {
          const int v = w - nb, k = v / N, i = v % N;
          const double s = sc[4 * k + 1];
          if (s != 0.0) {
            const double c = sc[4 * k];
            const int pq = (int)sc[4 * k + 3], p = pq >> 8, q = pq & 255;
            const double u = U[i * ldu + p], x = U[i * ldu + q];
            U[i * ldu + p] = c * u - s * x;
            U[i * ldu + q] = s * u + c * x;
          }
        }
      }
      __syncthreads();
    }
    const int any = *s_flag;
    __syncthreads();
    if (!any) break;
  }
  return sweep;
}

// Householder QR of a square n x n matrix Z (row-major, overwritten): on return the upper
// triangle of Z holds R (beta = -sign(x_1) ||x|| convention, zero columns skipped).
template <int T>
QL_DEV void householder_square(double* Z, int ld, int n, double* sd) {
  double* cnm = sd + n;  // sum over finished rows i < j of Z(i, c)^2
  for (int c = threadIdx.x; c < n; c += T) cnm[c] = 0.0;
  __syncthreads();
  for (int j = 0; j < n; ++j) {
    for (int c = j + threadIdx.x; c < n; c += T) {
      double s = 0.0;
      for (int i = j + 1; i < n; ++i) s = fma(Z[i * ld + j], Z[i * ld + c], s);
      sd[c] = s;
    }
    double x1 = Z[j * ld + j];
    __syncthreads();
    double nr = sd[j];
    double rem = fma(x1, x1, nr);
    bool skip = nr == 0.0 || rem <= 0x1p-92 * (cnm[j] + rem);  // residue below 2^-46 of the column
    if (!skip) {
      double nrm = sqrt(rem);
      double beta = x1 < 0.0 ? nrm : -nrm;
      double v1 = x1 - beta;
      double g = -1.0 / (beta * v1);
      for (int c = j + 1 + threadIdx.x; c < n; c += T) {
        double f = fma(v1, Z[j * ld + c], sd[c]) * g;
        double rn = fma(-v1, f, Z[j * ld + c]);
        Z[j * ld + c] = rn;
        cnm[c] = fma(rn, rn, cnm[c]);
        for (int i = j + 1; i < n; ++i) Z[i * ld + c] = fma(-Z[i * ld + j], f, Z[i * ld + c]);
      }
      if (threadIdx.x == 0) Z[j * ld + j] = beta;
    } else {
      for (int c = j + 1 + threadIdx.x; c < n; c += T) cnm[c] = fma(Z[j * ld + c], Z[j * ld + c], cnm[c]);
    }
    __syncthreads();
  }
  for (int t = threadIdx.x; t < n * n; t += T)
    if (t / n > t % n) Z[(t / n) * ld + t % n] = 0.0;
  __syncthreads();
}

}  // namespace ql
