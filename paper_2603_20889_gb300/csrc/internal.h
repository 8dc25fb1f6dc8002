// Host-side internal interfaces between the C ABI (api.cu) and the kernel translation
// units.  Not part of the public boundary.
#pragma once

#include <cstddef>
#include <cstdint>
#include <cuda.h>
#include <cuda_runtime.h>

#include "../../include/qless.h"

namespace ql {

// Epilogue selected for the root of a TSQR / the last CTA of a Gram pass.
enum Epilogue : int { kEpiR = 0, kEpiLstsq = 1 };

struct TsqrCall {
  int64_t m = 0;
  int n = 0;            // columns factored (n + 1 for least squares)
  int nA = 0;           // columns taken from A; column nA (if < n) comes from b
  const void* A = nullptr;
  int64_t lda = 0;
  const void* b = nullptr;
  ql_dtype dtype = QL_F64;
  int epilogue = kEpiR;
  double* R = nullptr;  // kEpiR: n x n output (ldr)
  int64_t ldr = 0;
  double* x = nullptr;  // kEpiLstsq: solution (n - 1 entries)
  double* resnorm = nullptr;
  double* Rext = nullptr;  // kEpiLstsq: optional n x n R_ext (ld n)
  int32_t* info = nullptr;
  void* ws = nullptr;
  size_t ws_bytes = 0;
  cudaStream_t stream = nullptr;
  int ctas_per_sm = 0;  // 0: occupancy maximum
  int max_ctas = 0;     // 0: no limit (testing the R-tree with few leaves)
  int variant = -1;     // thread layout (row-block height) for n > 8: -1 environment default, 0..2
  int arity = 0;        // R-tree arity: 0 the column class's default, else 2 .. default
};

// Upper bound of the TSQR workspace for n columns (any m).
size_t tsqr_workspace_bytes(int n);
// Launch the double-float TSQR (or FP64 when arith == QL_ARITH_F64) and, after a
// double-float launch, the gated FP64 fallback.
ql_status tsqr_launch(const TsqrCall& c, ql_arith arith);

struct GramCall {
  int64_t m = 0;
  int n = 0;
  int nA = 0;
  const void* A = nullptr;
  int64_t lda = 0;
  const void* b = nullptr;
  ql_dtype dtype = QL_F64;
  int method = QL_CHOLQR2;  // QL_CHOLQR2 or QL_SVQB2
  int epilogue = kEpiR;
  double* R = nullptr;
  int64_t ldr = 0;
  double* Z = nullptr;
  double rank_tol = 0.0;
  double* x = nullptr;
  double* resnorm = nullptr;
  double* Rext = nullptr;
  int32_t* info = nullptr;
  void* ws = nullptr;
  size_t ws_bytes = 0;
  cudaStream_t stream = nullptr;
};
size_t gram_workspace_bytes(int n);
ql_status gram_launch(const GramCall& c, ql_arith arith);

// SM count of the current device (cached per device).
int device_sm_count();
ql_arith current_arith();

// Largest n any entry point accepts.
constexpr int kApiMaxN = 64;
// Argument checks shared by the entry points (no device work): m >= 0, 1 <= n <= nmax, a
// known dtype, ld >= max(m, 1), X non-null when m > 0 (QL_ERR_ARG), X aligned to its
// element size (QL_ERR_ALIGN).
bool elem_aligned(const void* p, ql_dtype dt);
ql_status check_matrix(int64_t m, int64_t n, const void* X, ql_dtype dt, int64_t ld, int nmax);
// Output triangle R: non-null with ldr >= n (QL_ERR_ARG), 8-byte aligned (QL_ERR_ALIGN).
ql_status check_r(const double* R, int64_t ldr, int64_t n);
// Whether the Gram passes use the tensor-core kernels (double-float mode, n >= 9);
// the environment variable QL_GRAM_SIMT=1 selects the SIMT kernels instead.
bool tc_gram_enabled();
// First Gram pass of the 16-, 32- and 64-column classes on the pipelined tcgen05 kernel
// (default; QL_GRAM_PIPE=0 selects the per-tile kernels, for comparison).
bool pipe_gram_enabled();
// QL_GRAM_PIPE2=0: the later Gram passes of n <= 32 run on the per-tile mma.sync kernel instead
// of the pipelined one (A/B comparisons).
bool pipe_gram2_enabled();
// Tensor maps of the columns of [A b] for the pipelined Gram pass: A as a rank-2 tensor (rows
// innermost, stride lda; boxes of 128 bytes of rows x all its columns, 128-byte swizzle) and
// b as one unswizzled column; rows past m read as zeros.  tmB may be null (no b).  False, with the maps left
// unset, if the data does not allow tensor copies (a column not 16-byte aligned, m >= 2^31)
// or the driver offers no encoder; the caller then reads X without them.
bool pipe_tensor_maps(CUtensorMap* tmA, CUtensorMap* tmB, const void* A, const void* b, int dtype, int64_t m, int nA,
                      int64_t lda);

// Thread-layout variant of the TSQR kernels (environment QL_TSQR_CFG, 0 = default).
int tsqr_variant();

// Counts every kernel this library launches (reported by ql_launch_count()).
void count_launch();
// dst = the first nonzero {status, index} pair among src[0 .. count) (one tiny launch).
ql_status first_status_async(int32_t* dst, const int32_t* src, int count, cudaStream_t stream);

// Autotune table lookup for an (m, n, dtype, kappa) class: method, TSQR CTAs per SM, thread
// layout and R-tree arity (null outputs are skipped).
bool tune_lookup(int64_t m, int64_t n, ql_dtype dt, double kappa, int* method, int* ctas, int* variant = nullptr,
                 int* arity = nullptr);

// Batched path, asynchronous plan upload through pinned staging (serving loop).
ql_status batch_prepare_async(int32_t count, const ql_problem* probs, void* ws, size_t ws_bytes, cudaStream_t st,
                              unsigned char* pinned, size_t pinned_bytes);
size_t batch_plan_upload_bytes(int32_t count, const ql_problem* probs);

}  // namespace ql
