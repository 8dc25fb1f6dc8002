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
// round touch disjoint row/column pairs and run concurrently.  A pair is skipped when
// |a_pq| <= 1e-17 sqrt(|a_pp a_qq|); the loop stops after a sweep without rotations or
// after max_sweeps.  Returns the number of sweeps used.
template <int T>
QL_DEV int jacobi_eig(double* A, int ld, double* U, int ldu, int n, double* sc, int* s_flag, int max_sweeps = 30) {
  for (int t = threadIdx.x; t < n * n; t += T) U[(t / n) * ldu + t % n] = (t / n == t % n) ? 1.0 : 0.0;
  const int N = (n + 1) & ~1;  // players (one dummy when n is odd)
  const int half = N / 2;
  int sweep = 0;
  __syncthreads();
  for (; sweep < max_sweeps; ++sweep) {
    if (threadIdx.x == 0) *s_flag = 0;
    __syncthreads();
    for (int r = 0; r < N - 1; ++r) {
      // rotation parameters, one thread per pair
      for (int k = threadIdx.x; k < half; k += T) {
        int a = (k == 0) ? 0 : 1 + (k - 1 + r) % (N - 1);
        int b = 1 + (N - 2 - k + r) % (N - 1);
        int p = a < b ? a : b, q = a < b ? b : a;
        double c = 1.0, s = 0.0;
        if (q < n) {
          double apq = A[p * ld + q], app = A[p * ld + p], aqq = A[q * ld + q];
          if (apq != 0.0 && fabs(apq) > 1e-17 * sqrt(fabs(app * aqq))) {
            double tau = (aqq - app) / (2.0 * apq);
            double t = (tau >= 0.0 ? 1.0 : -1.0) / (fabs(tau) + sqrt(1.0 + tau * tau));
            c = 1.0 / sqrt(1.0 + t * t);
            s = t * c;
            *s_flag = 1;
          }
        }
        sc[4 * k + 0] = c;
        sc[4 * k + 1] = s;
        sc[4 * k + 2] = (double)p;
        sc[4 * k + 3] = (double)q;
      }
      __syncthreads();
      // columns p, q of A and U:  X <- X J
      for (int t = threadIdx.x; t < half * n; t += T) {
        int k = t / n, i = t % n;
        double c = sc[4 * k], s = sc[4 * k + 1];
        int p = (int)sc[4 * k + 2], q = (int)sc[4 * k + 3];
        if (q < n && s != 0.0) {
          double x = A[i * ld + p], y = A[i * ld + q];
          A[i * ld + p] = c * x - s * y;
          A[i * ld + q] = s * x + c * y;
          double u = U[i * ldu + p], v = U[i * ldu + q];
          U[i * ldu + p] = c * u - s * v;
          U[i * ldu + q] = s * u + c * v;
        }
      }
      __syncthreads();
      // rows p, q of A:  A <- J^T A
      for (int t = threadIdx.x; t < half * n; t += T) {
        int k = t / n, i = t % n;
        double c = sc[4 * k], s = sc[4 * k + 1];
        int p = (int)sc[4 * k + 2], q = (int)sc[4 * k + 3];
        if (q < n && s != 0.0) {
          double x = A[p * ld + i], y = A[q * ld + i];
          A[p * ld + i] = c * x - s * y;
          A[q * ld + i] = s * x + c * y;
        }
      }
      __syncthreads();
      for (int k = threadIdx.x; k < half; k += T) {
        int p = (int)sc[4 * k + 2], q = (int)sc[4 * k + 3];
        if (q < n && sc[4 * k + 1] != 0.0) {
          A[p * ld + q] = 0.0;
          A[q * ld + p] = 0.0;
        }
      }
      __syncthreads();
    }
    int any = *s_flag;
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
