// FP64 epilogues run by the single CTA that owns the final triangle (the R-tree root, or
// the last CTA of a Gram pass): sign normalisation and output of R (Sec. 1: R with a
// nonnegative diagonal), and the least-squares solve of the extended factor
// R_ext = [[R, z], [0, rho]] of [A b] (x = R^{-1} z, ||b - A x|| = rho).
#pragma once

#include "common.cuh"

namespace ql {

// Ra: n x n upper triangle in shared memory, row-major with leading dimension lds.
// Rows with a negative diagonal entry are negated; the strict lower triangle of R is
// written as zero.  Returns (to every thread) whether a non-finite entry was seen.
template <int T>
QL_DEV bool write_r_normalised(double* Ra, int lds, int n, double* R, int64_t ldr, int* s_flag) {
  if (threadIdx.x == 0) *s_flag = 0;
  __syncthreads();
  for (int i = threadIdx.x; i < n * n; i += T) {
    int c = i / n, r = i % n;
    double v = 0.0;
    if (r <= c) {
      v = Ra[r * lds + c];
      if (Ra[r * lds + r] < 0.0) v = -v;
      if (!isfinite(v)) *s_flag = 1;
    }
    if (R) R[(int64_t)c * ldr + r] = v;
  }
  __syncthreads();
  bool bad = *s_flag != 0;
  __syncthreads();
  // normalise in place as well (later epilogue stages read it)
  for (int i = threadIdx.x; i < n * n; i += T) {
    int r = i / n, c = i % n;
    if (r < c && Ra[r * lds + r] < 0.0) Ra[r * lds + c] = -Ra[r * lds + c];
  }
  __syncthreads();
  for (int r = threadIdx.x; r < n; r += T)
    if (Ra[r * lds + r] < 0.0) Ra[r * lds + r] = -Ra[r * lds + r];
  __syncthreads();
  return bad;
}

QL_DEV void write_info(int32_t* info, int status, int index) {
  if (info && threadIdx.x == 0) {
    info[0] = status;
    info[1] = index;
  }
}

// Status of a finished factorisation: a non-finite R first; otherwise a bounded wait that
// gave up earlier in the call (the call was completed by the FP64 kernels, R is valid)
// reports {QL_ERR_TIMEOUT, where}; otherwise QL_OK.
QL_DEV void write_final_info(int32_t* info, bool nonfinite, int timeout_where) {
  if (nonfinite)
    write_info(info, QL_ERR_NONFINITE, 0);
  else if (timeout_where)
    write_info(info, QL_ERR_TIMEOUT, timeout_where);
  else
    write_info(info, QL_OK, 0);
}

// Root epilogue for a plain factorisation: R out, info.
template <int T>
QL_DEV void epilogue_r(double* Ra, int lds, int n, double* R, int64_t ldr, int32_t* info, int* s_flag,
                       int timeout_where = 0) {
  bool bad = write_r_normalised<T>(Ra, lds, n, R, ldr, s_flag);
  write_final_info(info, bad, timeout_where);
}

// Root epilogue for least squares: Ra holds R_ext (n1 x n1, n1 = n + 1).
template <int T>
QL_DEV void epilogue_lstsq(double* Ra, int lds, int n1, double* x, double* resnorm, double* Rext,
                           int32_t* info, double* zz, int* s_flag, int timeout_where = 0) {
  int n = n1 - 1;
  bool bad = write_r_normalised<T>(Ra, lds, n1, Rext, n1, s_flag);
  // zero diagonal entry of R -> rank deficient: report the first one
  if (threadIdx.x == 0) {
    int zi = 0;
    for (int i = 0; i < n; ++i)
      if (Ra[i * lds + i] == 0.0) {
        zi = i + 1;
        break;
      }
    s_flag[1] = zi;
  }
  for (int i = threadIdx.x; i < n; i += T) zz[i] = Ra[i * lds + n];
  __syncthreads();
  int zi = s_flag[1];
  if (zi) {
    for (int i = threadIdx.x; i < n; i += T) x[i] = __longlong_as_double(0x7ff8000000000000ll);
    if (threadIdx.x == 0) *resnorm = Ra[n * lds + n];
    write_info(info, QL_ERR_NOT_SPD, zi);
    return;
  }
  // back-substitution, column oriented: x_i = zz_i / R_ii, then zz_k -= R_ki x_i (k < i)
  for (int i = n - 1; i >= 0; --i) {
    double xi = zz[i] / Ra[i * lds + i];
    for (int k = threadIdx.x; k < i; k += T) zz[k] = fma(-Ra[k * lds + i], xi, zz[k]);
    if (threadIdx.x == 0) x[i] = xi;
    __syncthreads();
  }
  if (threadIdx.x == 0) *resnorm = Ra[n * lds + n];
  write_final_info(info, bad, timeout_where);
}

}  // namespace ql
