/*
 * Oracle for the Q-less QR of a tall, skinny matrix -- TEST INFRASTRUCTURE ONLY.
 *
 * Plain, slow, obviously-correct CPU code that the tests, the smoke check and the
 * CPU-baseline leg of the benchmark compare the CUDA library against.  It shares no
 * code, header, table or helper with the CUDA path, and the product path never calls it.
 *
 * Storage is IEEE double; every norm, dot product and update is accumulated in
 * `long double` (80-bit extended on x86-64, binary128 on aarch64).  Matrices are
 * column-major with a leading dimension, exactly like the library's boundary.
 *
 * What each routine follows (paper: "Implementation of QR factorization of tall and very
 * skinny matrices on current GPUs"):
 *   qo_householder_r   the problem statement of Sec. 1 (X = QR, Q^T Q = I, R upper
 *                      triangular), computed by textbook column-by-column Householder QR;
 *                      R is returned with a nonnegative diagonal, which makes it unique
 *                      when rank(X) = n.
 *   qo_gram            C = X^T X, the first step of Algorithm 1.
 *   qo_cholesky_upper  R^T R = C (the "chol" of Algorithm 1, steps 2 and 4).
 *   qo_cholqr2         Algorithm 1 (Q-less Cholesky-QR2), step by step.
 *   qo_scholqr3        shifted Cholesky-QR3, the ill-conditioned variant Sec. 1 cites, in the
 *                      published form: chol(X^T X + s I), then Cholesky-QR twice.
 *   qo_q_from_r        Q = X R^{-1}, the orthonormal factor of X = QR (Sec. 1), by row-wise
 *                      forward substitution.
 *   qo_project_out     the two-phase problem (I - Y Y^T) X with re-orthogonalisation (Sec. 2):
 *                      two projection passes, coefficients accumulated.
 *   qo_jacobi_eig      C = U diag(lambda) U^T (the eigendecomposition that SVQB uses in
 *                      place of chol, Sec. 3.1).
 *   qo_svqb2           SVQB applied twice (Sec. 3.1): B = U Lambda^{-1/2}, X B = Q, and the
 *                      QZ form X = Q Z of Sec. 1, turned into R by a QR of Z.
 *   qo_lstsq           least squares through the Q-less QR of [A b] (Sec. 1).
 *   qo_singular_values one-sided Jacobi SVD of a small square matrix (condition numbers).
 *
 * Return values: 0 on success, a positive LAPACK-style index on numerical breakdown,
 * -1 on bad arguments or allocation failure.
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

typedef long double acc_t;

#define AT(a, ld, i, j) ((a)[(size_t)(j) * (size_t)(ld) + (size_t)(i)])

static double* copy_matrix(int64_t m, int64_t n, const double* x, int64_t ldx) {
  size_t cnt = (size_t)(m > 0 ? m : 1) * (size_t)(n > 0 ? n : 1);
  double* a = (double*)malloc(cnt * sizeof(double));
  if (!a) return NULL;
  for (int64_t j = 0; j < n; ++j)
    for (int64_t i = 0; i < m; ++i) AT(a, m, i, j) = AT(x, ldx, i, j);
  return a;
}

/* Multiply every row of the upper triangle with a negative diagonal entry by -1. */
static void sign_normalise(int64_t n, double* r, int64_t ldr) {
  for (int64_t i = 0; i < n; ++i)
    if (AT(r, ldr, i, i) < 0.0)
      for (int64_t j = i; j < n; ++j) AT(r, ldr, i, j) = -AT(r, ldr, i, j);
}

/*
 * Householder QR, R only.  For column j the reflector H = I - 2 v v^T / (v^T v) maps
 * x = A[j:m, j] onto beta e_1 with beta = -sign(x_1) ||x||, sign(0) = +1, so that
 * v_1 = x_1 - beta never cancels.  A zero column gets no reflector (R_jj = 0), which
 * is how rank deficiency shows up as a zero diagonal entry.
 */
int qo_householder_r(int64_t m, int64_t n, const double* X, int64_t ldx, double* R, int64_t ldr) {
  if (m < 0 || n < 0 || ldx < (m > 1 ? m : 1) || ldr < (n > 1 ? n : 1)) return -1;
  for (int64_t j = 0; j < n; ++j)
    for (int64_t i = 0; i < n; ++i) AT(R, ldr, i, j) = 0.0;
  if (m == 0 || n == 0) return 0;
  double* a = copy_matrix(m, n, X, ldx);
  if (!a) return -1;
  int64_t steps = m < n ? m : n;
  for (int64_t j = 0; j < steps; ++j) {
    acc_t s2 = 0.0L;
    for (int64_t i = j; i < m; ++i) s2 += (acc_t)AT(a, m, i, j) * (acc_t)AT(a, m, i, j);
    if (s2 == 0.0L) continue;
    acc_t nrm = sqrtl(s2);
    acc_t x1 = AT(a, m, j, j);
    acc_t beta = (x1 >= 0.0L) ? -nrm : nrm;
    acc_t v1 = x1 - beta;
    acc_t vtv = -2.0L * beta * v1; /* = 2 beta (beta - x1) > 0 */
    for (int64_t c = j + 1; c < n; ++c) {
      acc_t s = v1 * (acc_t)AT(a, m, j, c);
      for (int64_t i = j + 1; i < m; ++i) s += (acc_t)AT(a, m, i, j) * (acc_t)AT(a, m, i, c);
      acc_t f = 2.0L * s / vtv;
      AT(a, m, j, c) = (double)((acc_t)AT(a, m, j, c) - f * v1);
      for (int64_t i = j + 1; i < m; ++i)
        AT(a, m, i, c) = (double)((acc_t)AT(a, m, i, c) - f * (acc_t)AT(a, m, i, j));
    }
    AT(a, m, j, j) = (double)beta;
  }
  for (int64_t j = 0; j < n; ++j)
    for (int64_t i = 0; i <= j && i < steps; ++i) AT(R, ldr, i, j) = AT(a, m, i, j);
  sign_normalise(n, R, ldr);
  free(a);
  return 0;
}

/* C = X^T X (full symmetric matrix). */
int qo_gram(int64_t m, int64_t n, const double* X, int64_t ldx, double* C, int64_t ldc) {
  if (m < 0 || n < 0 || ldx < (m > 1 ? m : 1) || ldc < (n > 1 ? n : 1)) return -1;
  for (int64_t p = 0; p < n; ++p)
    for (int64_t q = p; q < n; ++q) {
      acc_t s = 0.0L;
      for (int64_t i = 0; i < m; ++i) s += (acc_t)AT(X, ldx, i, p) * (acc_t)AT(X, ldx, i, q);
      AT(C, ldc, p, q) = (double)s;
      AT(C, ldc, q, p) = (double)s;
    }
  return 0;
}

/*
 * Upper Cholesky factor: R^T R = C, reading only the upper triangle of C.  Returns j+1
 * when the j-th pivot is not positive (LAPACK's info); R's rows before j are valid.
 */
int qo_cholesky_upper(int64_t n, const double* C, int64_t ldc, double* R, int64_t ldr) {
  if (n < 0 || ldc < (n > 1 ? n : 1) || ldr < (n > 1 ? n : 1)) return -1;
  for (int64_t j = 0; j < n; ++j)
    for (int64_t i = 0; i < n; ++i) AT(R, ldr, i, j) = 0.0;
  for (int64_t j = 0; j < n; ++j) {
    acc_t d = AT(C, ldc, j, j);
    for (int64_t k = 0; k < j; ++k) d -= (acc_t)AT(R, ldr, k, j) * (acc_t)AT(R, ldr, k, j);
    if (!(d > 0.0L)) return (int)(j + 1);
    acc_t rjj = sqrtl(d);
    AT(R, ldr, j, j) = (double)rjj;
    for (int64_t c = j + 1; c < n; ++c) {
      acc_t s = AT(C, ldc, j, c);
      for (int64_t k = 0; k < j; ++k) s -= (acc_t)AT(R, ldr, k, j) * (acc_t)AT(R, ldr, k, c);
      AT(R, ldr, j, c) = (double)(s / rjj);
    }
  }
  return 0;
}

/* Solve Y R = X row by row (Y = X R^{-1}, the "X / R" of Algorithm 1), R upper triangular. */
static void right_upper_solve(int64_t m, int64_t n, const double* X, int64_t ldx, const double* R,
                              int64_t ldr, double* Y) {
  for (int64_t i = 0; i < m; ++i)
    for (int64_t c = 0; c < n; ++c) {
      acc_t s = AT(X, ldx, i, c);
      for (int64_t k = 0; k < c; ++k) s -= (acc_t)AT(Y, m, i, k) * (acc_t)AT(R, ldr, k, c);
      AT(Y, m, i, c) = (double)(s / (acc_t)AT(R, ldr, c, c));
    }
}

/* P = A B for n x n upper triangular A and B (the product is upper triangular). */
static void upper_product(int64_t n, const double* A, int64_t lda, const double* B, int64_t ldb,
                          double* P, int64_t ldp) {
  for (int64_t j = 0; j < n; ++j)
    for (int64_t i = 0; i < n; ++i) {
      acc_t s = 0.0L;
      for (int64_t k = i; k <= j; ++k) s += (acc_t)AT(A, lda, i, k) * (acc_t)AT(B, ldb, k, j);
      AT(P, ldp, i, j) = (i <= j) ? (double)s : 0.0;
    }
}

/*
 * Algorithm 1, Q-less Cholesky-QR2:
 *   C <- X^T X;  R1 <- chol(C);  C <- (X/R1)^T (X/R1);  R2 <- chol(C);  R <- R2 R1.
 * Optional R1 output (ldr).  Returns the chol info of the failing step: j+1 for the first
 * Cholesky, 1000 + j + 1 for the second.
 */
int qo_cholqr2(int64_t m, int64_t n, const double* X, int64_t ldx, double* R, int64_t ldr,
               double* R1_out) {
  if (m < 0 || n < 1 || ldx < (m > 1 ? m : 1) || ldr < n) return -1;
  size_t nn = (size_t)n * (size_t)n;
  double* C = (double*)malloc(nn * sizeof(double));
  double* R1 = (double*)malloc(nn * sizeof(double));
  double* R2 = (double*)malloc(nn * sizeof(double));
  double* Y = (double*)malloc((size_t)(m > 0 ? m : 1) * (size_t)n * sizeof(double));
  int info = -1;
  if (!C || !R1 || !R2 || !Y) goto done;
  qo_gram(m, n, X, ldx, C, n);
  info = qo_cholesky_upper(n, C, n, R1, n);
  if (info) goto done;
  right_upper_solve(m, n, X, ldx, R1, n, Y);
  qo_gram(m, n, Y, (m > 1 ? m : 1), C, n);
  info = qo_cholesky_upper(n, C, n, R2, n);
  if (info) { info += 1000; goto done; }
  upper_product(n, R2, n, R1, n, R, ldr);
  if (R1_out)
    for (size_t k = 0; k < nn; ++k) R1_out[k] = R1[k];
done:
  free(C); free(R1); free(R2); free(Y);
  return info;
}

/*
 * Q = X R^{-1} for an upper triangular R with nonzero diagonal: row i of Q solves
 * q R = x_i (forward substitution over the columns).  Returns j+1 when R(j, j) = 0.
 */
int qo_q_from_r(int64_t m, int64_t n, const double* X, int64_t ldx, const double* R, int64_t ldr, double* Q,
                int64_t ldq) {
  if (m < 0 || n < 1 || ldx < (m > 1 ? m : 1) || ldr < n || ldq < (m > 1 ? m : 1)) return -1;
  for (int64_t j = 0; j < n; ++j)
    if (AT(R, ldr, j, j) == 0.0) return (int)(j + 1);
  for (int64_t i = 0; i < m; ++i)
    for (int64_t c = 0; c < n; ++c) {
      acc_t s = AT(X, ldx, i, c);
      for (int64_t k = 0; k < c; ++k) s -= (acc_t)AT(Q, ldq, i, k) * (acc_t)AT(R, ldr, k, c);
      AT(Q, ldq, i, c) = (double)(s / (acc_t)AT(R, ldr, c, c));
    }
  return 0;
}

/*
 * Two projections against Y (m x k, orthonormal columns):  C1 = Y^T X;  W1 = X - Y C1;
 * C2 = Y^T W1;  W = W1 - Y C2;  C = C1 + C2 (k x n, ld ldc).  W (m x n, ld ldw).
 */
static void project_once(int64_t m, int64_t k, const double* Y, int64_t ldy, int64_t n, const double* V,
                         int64_t ldv, double* Cp, double* W, int64_t ldw) {
  for (int64_t j = 0; j < n; ++j)
    for (int64_t i = 0; i < k; ++i) {
      acc_t s = 0.0L;
      for (int64_t r = 0; r < m; ++r) s += (acc_t)AT(Y, ldy, r, i) * (acc_t)AT(V, ldv, r, j);
      AT(Cp, k, i, j) = (double)s;
    }
  for (int64_t j = 0; j < n; ++j)
    for (int64_t r = 0; r < m; ++r) {
      acc_t w = AT(V, ldv, r, j);
      for (int64_t i = 0; i < k; ++i) w -= (acc_t)AT(Y, ldy, r, i) * (acc_t)AT(Cp, k, i, j);
      AT(W, ldw, r, j) = (double)w;
    }
}

int qo_project_out(int64_t m, int64_t k, const double* Y, int64_t ldy, int64_t n, const double* X, int64_t ldx,
                   double* W, int64_t ldw, double* C, int64_t ldc) {
  int64_t lmin = m > 1 ? m : 1;
  if (m < 0 || k < 1 || n < 1 || ldy < lmin || ldx < lmin || ldw < lmin || ldc < k) return -1;
  double* C1 = (double*)malloc((size_t)k * (size_t)n * sizeof(double));
  double* C2 = (double*)malloc((size_t)k * (size_t)n * sizeof(double));
  double* W1 = (double*)malloc((size_t)lmin * (size_t)n * sizeof(double));
  int info = -1;
  if (!C1 || !C2 || !W1) goto done;
  project_once(m, k, Y, ldy, n, X, ldx, C1, W1, lmin);
  project_once(m, k, Y, ldy, n, W1, lmin, C2, W, ldw);
  for (int64_t j = 0; j < n; ++j)
    for (int64_t i = 0; i < k; ++i) AT(C, ldc, i, j) = AT(C1, k, i, j) + AT(C2, k, i, j);
  info = 0;
done:
  free(C1); free(C2); free(W1);
  return info;
}

/*
 * Shifted Cholesky-QR3:
 *   C <- X^T X;  s <- 11 (m n + n (n + 1)) u ||X||_F^2 with u = 2^-53 and ||X||_F^2 =
 *   trace(C) (an upper bound of ||X||_2^2);  R1 <- chol(C + s I);  Y1 <- X / R1;
 *   R2 <- chol(Y1^T Y1);  Y2 <- Y1 / R2;  R3 <- chol(Y2^T Y2);  R <- R3 R2 R1.
 * Returns the chol info of the failing step: j+1, 1000 + j+1 or 2000 + j+1.
 */
int qo_scholqr3(int64_t m, int64_t n, const double* X, int64_t ldx, double* R, int64_t ldr) {
  if (m < 0 || n < 1 || ldx < (m > 1 ? m : 1) || ldr < n) return -1;
  size_t nn = (size_t)n * (size_t)n, mn = (size_t)(m > 0 ? m : 1) * (size_t)n;
  int64_t ldy = m > 1 ? m : 1;
  double* C = (double*)malloc(nn * sizeof(double));
  double* R1 = (double*)malloc(nn * sizeof(double));
  double* R2 = (double*)malloc(nn * sizeof(double));
  double* R3 = (double*)malloc(nn * sizeof(double));
  double* T = (double*)malloc(nn * sizeof(double));
  double* Y1 = (double*)malloc(mn * sizeof(double));
  double* Y2 = (double*)malloc(mn * sizeof(double));
  int info = -1;
  if (!C || !R1 || !R2 || !R3 || !T || !Y1 || !Y2) goto done;
  qo_gram(m, n, X, ldx, C, n);
  {
    acc_t tr = 0.0L;
    for (int64_t j = 0; j < n; ++j) tr += AT(C, n, j, j);
    double shift = (double)(11.0L * ((acc_t)m * (acc_t)n + (acc_t)n * (acc_t)(n + 1)) * ldexpl(1.0L, -53) * tr);
    for (int64_t j = 0; j < n; ++j) AT(C, n, j, j) += shift;
  }
  info = qo_cholesky_upper(n, C, n, R1, n);
  if (info) goto done;
  right_upper_solve(m, n, X, ldx, R1, n, Y1);
  qo_gram(m, n, Y1, ldy, C, n);
  info = qo_cholesky_upper(n, C, n, R2, n);
  if (info) { info += 1000; goto done; }
  right_upper_solve(m, n, Y1, ldy, R2, n, Y2);
  qo_gram(m, n, Y2, ldy, C, n);
  info = qo_cholesky_upper(n, C, n, R3, n);
  if (info) { info += 2000; goto done; }
  upper_product(n, R2, n, R1, n, T, n);
  upper_product(n, R3, n, T, n, R, ldr);
done:
  free(C); free(R1); free(R2); free(R3); free(T); free(Y1); free(Y2);
  return info;
}

/*
 * Cyclic two-sided Jacobi for a symmetric n x n matrix: C = U diag(lambda) U^T.
 * Rotation angles follow the textbook symmetric Schur step (tau, t, c, s); a pair is
 * skipped when |c_pq| is below 1e-18 * sqrt(|c_pp c_qq|) (a relative test, so small
 * eigenvalues keep their relative accuracy), and the sweep loop ends after a sweep
 * with no rotation.  Eigenvalues come back in ascending order with U's columns.
 */
int qo_jacobi_eig(int64_t n, const double* Cin, int64_t ldc, double* lambda, double* U, int64_t ldu) {
  if (n < 1 || ldc < n || ldu < n) return -1;
  size_t nn = (size_t)n * (size_t)n;
  acc_t* a = (acc_t*)malloc(nn * sizeof(acc_t));
  acc_t* u = (acc_t*)malloc(nn * sizeof(acc_t));
  if (!a || !u) { free(a); free(u); return -1; }
  for (int64_t j = 0; j < n; ++j)
    for (int64_t i = 0; i < n; ++i) {
      a[j * n + i] = AT(Cin, ldc, (i < j ? i : j), (i < j ? j : i)); /* upper triangle */
      u[j * n + i] = (i == j) ? 1.0L : 0.0L;
    }
  for (int sweep = 0; sweep < 100; ++sweep) {
    int rotated = 0;
    for (int64_t p = 0; p < n - 1; ++p)
      for (int64_t q = p + 1; q < n; ++q) {
        acc_t apq = a[q * n + p];
        acc_t app = a[p * n + p], aqq = a[q * n + q];
        if (apq == 0.0L) continue;
        if (fabsl(apq) <= 1e-18L * sqrtl(fabsl(app * aqq))) continue;
        rotated = 1;
        acc_t tau = (aqq - app) / (2.0L * apq);
        acc_t t = (tau >= 0.0L ? 1.0L : -1.0L) / (fabsl(tau) + sqrtl(1.0L + tau * tau));
        acc_t c = 1.0L / sqrtl(1.0L + t * t), s = t * c;
        for (int64_t k = 0; k < n; ++k) { /* columns p, q: A <- A J */
          acc_t akp = a[p * n + k], akq = a[q * n + k];
          a[p * n + k] = c * akp - s * akq;
          a[q * n + k] = s * akp + c * akq;
        }
        for (int64_t k = 0; k < n; ++k) { /* rows p, q: A <- J^T A */
          acc_t apk = a[k * n + p], aqk = a[k * n + q];
          a[k * n + p] = c * apk - s * aqk;
          a[k * n + q] = s * apk + c * aqk;
        }
        a[q * n + p] = 0.0L;
        a[p * n + q] = 0.0L;
        for (int64_t k = 0; k < n; ++k) { /* U <- U J */
          acc_t ukp = u[p * n + k], ukq = u[q * n + k];
          u[p * n + k] = c * ukp - s * ukq;
          u[q * n + k] = s * ukp + c * ukq;
        }
      }
    if (!rotated) break;
  }
  /* ascending order (selection sort keeps it plain) */
  int64_t* idx = (int64_t*)malloc((size_t)n * sizeof(int64_t));
  if (!idx) { free(a); free(u); return -1; }
  for (int64_t i = 0; i < n; ++i) idx[i] = i;
  for (int64_t i = 0; i < n; ++i) {
    int64_t best = i;
    for (int64_t k = i + 1; k < n; ++k)
      if (a[idx[k] * n + idx[k]] < a[idx[best] * n + idx[best]]) best = k;
    int64_t t = idx[i]; idx[i] = idx[best]; idx[best] = t;
  }
  for (int64_t i = 0; i < n; ++i) {
    lambda[i] = (double)a[idx[i] * n + idx[i]];
    for (int64_t k = 0; k < n; ++k) AT(U, ldu, k, i) = (double)u[idx[i] * n + k];
  }
  free(idx); free(a); free(u);
  return 0;
}

/*
 * One SVQB step on the Gram matrix C: eigendecomposition C = U Lambda U^T, then
 * B = U Lambda^{-1/2} and the factor S = Lambda^{1/2} U^T (so that B = S^{-1} on the kept
 * subspace).  Eigenvalues below n * eps * lambda_max are treated as zero: their entries of
 * Lambda^{-1/2} and Lambda^{1/2} are set to 0 (the truncation of Sec. 3.1).
 */
static int svqb_step(int64_t n, const double* C, double* B, double* S) {
  size_t nn = (size_t)n * (size_t)n;
  double* lam = (double*)malloc((size_t)n * sizeof(double));
  double* U = (double*)malloc(nn * sizeof(double));
  if (!lam || !U) { free(lam); free(U); return -1; }
  int info = qo_jacobi_eig(n, C, n, lam, U, n);
  if (info) { free(lam); free(U); return info; }
  double lmax = 0.0;
  for (int64_t i = 0; i < n; ++i) if (lam[i] > lmax) lmax = lam[i];
  double cut = (double)n * 2.220446049250313e-16 * lmax;
  for (int64_t i = 0; i < n; ++i) {
    int keep = lam[i] > cut && lam[i] > 0.0;
    acc_t sq = keep ? sqrtl((acc_t)lam[i]) : 0.0L;
    acc_t inv = keep ? 1.0L / sq : 0.0L;
    for (int64_t k = 0; k < n; ++k) {
      AT(B, n, k, i) = (double)((acc_t)AT(U, n, k, i) * inv);
      AT(S, n, i, k) = (double)(sq * (acc_t)AT(U, n, k, i));
    }
  }
  free(lam); free(U);
  return 0;
}

/* Y = X B for X m x n, B n x n (full). */
static void right_multiply(int64_t m, int64_t n, const double* X, int64_t ldx, const double* B, double* Y) {
  for (int64_t i = 0; i < m; ++i)
    for (int64_t c = 0; c < n; ++c) {
      acc_t s = 0.0L;
      for (int64_t k = 0; k < n; ++k) s += (acc_t)AT(X, ldx, i, k) * (acc_t)AT(B, n, k, c);
      AT(Y, m, i, c) = (double)s;
    }
}

/*
 * SVQB applied twice, Q-less (Sec. 3.1): C1 = X^T X -> (B1, S1); C2 = (X B1)^T (X B1) ->
 * (B2, S2).  Then X B1 B2 = Q and X = Q Z with Z = S2 S1.  R = qr_r(Z), so that
 * R^T R = Z^T Z = X^T X.  Z (n x n, optional) is returned before the QR.
 */
int qo_svqb2(int64_t m, int64_t n, const double* X, int64_t ldx, double* R, int64_t ldr, double* Z_out) {
  if (m < 0 || n < 1 || ldx < (m > 1 ? m : 1) || ldr < n) return -1;
  size_t nn = (size_t)n * (size_t)n;
  double *C = malloc(nn * 8), *B1 = malloc(nn * 8), *S1 = malloc(nn * 8), *B2 = malloc(nn * 8),
         *S2 = malloc(nn * 8), *Z = malloc(nn * 8);
  double* Y = (double*)malloc((size_t)(m > 0 ? m : 1) * (size_t)n * sizeof(double));
  int info = -1;
  if (!C || !B1 || !S1 || !B2 || !S2 || !Z || !Y) goto done;
  qo_gram(m, n, X, ldx, C, n);
  if ((info = svqb_step(n, C, B1, S1))) goto done;
  right_multiply(m, n, X, ldx, B1, Y);
  qo_gram(m, n, Y, (m > 1 ? m : 1), C, n);
  if ((info = svqb_step(n, C, B2, S2))) goto done;
  for (int64_t j = 0; j < n; ++j)
    for (int64_t i = 0; i < n; ++i) {
      acc_t s = 0.0L;
      for (int64_t k = 0; k < n; ++k) s += (acc_t)AT(S2, n, i, k) * (acc_t)AT(S1, n, k, j);
      AT(Z, n, i, j) = (double)s;
    }
  if (Z_out)
    for (size_t k = 0; k < nn; ++k) Z_out[k] = Z[k];
  info = qo_householder_r(n, n, Z, n, R, ldr);
done:
  free(C); free(B1); free(S1); free(B2); free(S2); free(Z); free(Y);
  return info;
}

/* Solve R x = z by back-substitution; returns i+1 if R_ii == 0. */
int qo_back_substitution(int64_t n, const double* R, int64_t ldr, const double* z, double* x) {
  for (int64_t i = n - 1; i >= 0; --i) {
    acc_t s = z[i];
    for (int64_t k = i + 1; k < n; ++k) s -= (acc_t)AT(R, ldr, i, k) * (acc_t)x[k];
    if (AT(R, ldr, i, i) == 0.0) return (int)(i + 1);
    x[i] = (double)(s / (acc_t)AT(R, ldr, i, i));
  }
  return 0;
}

/*
 * min_x ||A x - b||_2 through the Q-less QR of the extended matrix [A b] (Sec. 1):
 * R_ext = [[R, z], [0, rho]], x = R^{-1} z, ||b - A x|| = rho.  R_ext ((n+1) x (n+1),
 * ld n+1) is optional.
 */
int qo_lstsq(int64_t m, int64_t n, const double* A, int64_t lda, const double* b, double* x,
             double* resnorm, double* Rext_out) {
  if (m < 0 || n < 1 || lda < (m > 1 ? m : 1)) return -1;
  int64_t n1 = n + 1;
  double* Ab = (double*)malloc((size_t)(m > 0 ? m : 1) * (size_t)n1 * sizeof(double));
  double* Re = (double*)malloc((size_t)n1 * (size_t)n1 * sizeof(double));
  double* z = (double*)malloc((size_t)n * sizeof(double));
  int info = -1;
  if (!Ab || !Re || !z) goto done;
  for (int64_t j = 0; j < n; ++j)
    for (int64_t i = 0; i < m; ++i) AT(Ab, m, i, j) = AT(A, lda, i, j);
  for (int64_t i = 0; i < m; ++i) AT(Ab, m, i, n) = b[i];
  if ((info = qo_householder_r(m, n1, Ab, (m > 1 ? m : 1), Re, n1))) goto done;
  for (int64_t i = 0; i < n; ++i) z[i] = AT(Re, n1, i, n);
  *resnorm = AT(Re, n1, n, n);
  info = qo_back_substitution(n, Re, n1, z, x);
  if (Rext_out)
    for (size_t k = 0; k < (size_t)n1 * (size_t)n1; ++k) Rext_out[k] = Re[k];
done:
  free(Ab); free(Re); free(z);
  return info;
}

/*
 * Singular values of a square n x n matrix by one-sided (Hestenes) Jacobi: rotate column
 * pairs until all are mutually orthogonal; the column norms are the singular values
 * (descending).  Used to state kappa_2 for the tolerance when X is not built with a known
 * spectrum.
 */
int qo_singular_values(int64_t n, const double* Ain, int64_t lda, double* sigma) {
  if (n < 1 || lda < n) return -1;
  acc_t* a = (acc_t*)malloc((size_t)n * (size_t)n * sizeof(acc_t));
  if (!a) return -1;
  for (int64_t j = 0; j < n; ++j)
    for (int64_t i = 0; i < n; ++i) a[j * n + i] = AT(Ain, lda, i, j);
  for (int sweep = 0; sweep < 100; ++sweep) {
    int rotated = 0;
    for (int64_t p = 0; p < n - 1; ++p)
      for (int64_t q = p + 1; q < n; ++q) {
        acc_t alpha = 0, beta = 0, gamma = 0;
        for (int64_t k = 0; k < n; ++k) {
          alpha += a[p * n + k] * a[p * n + k];
          beta += a[q * n + k] * a[q * n + k];
          gamma += a[p * n + k] * a[q * n + k];
        }
        if (gamma == 0.0L || fabsl(gamma) <= 1e-18L * sqrtl(alpha * beta)) continue;
        rotated = 1;
        acc_t zeta = (beta - alpha) / (2.0L * gamma);
        acc_t t = (zeta >= 0.0L ? 1.0L : -1.0L) / (fabsl(zeta) + sqrtl(1.0L + zeta * zeta));
        acc_t c = 1.0L / sqrtl(1.0L + t * t), s = c * t;
        for (int64_t k = 0; k < n; ++k) {
          acc_t ap = a[p * n + k], aq = a[q * n + k];
          a[p * n + k] = c * ap - s * aq;
          a[q * n + k] = s * ap + c * aq;
        }
      }
    if (!rotated) break;
  }
  for (int64_t j = 0; j < n; ++j) {
    acc_t s = 0;
    for (int64_t k = 0; k < n; ++k) s += a[j * n + k] * a[j * n + k];
    sigma[j] = (double)sqrtl(s);
  }
  for (int64_t i = 0; i < n; ++i) /* descending */
    for (int64_t k = i + 1; k < n; ++k)
      if (sigma[k] > sigma[i]) { double t = sigma[i]; sigma[i] = sigma[k]; sigma[k] = t; }
  free(a);
  return 0;
}
