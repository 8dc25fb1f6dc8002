/*
 * qless -- Q-less QR of tall, very skinny matrices on GB300 (sm_103a).
 *
 * Given a real dense X (m x n, m >> n, n <= 64), every entry point here computes the n x n
 * upper triangular factor R of X = QR, Q^T Q = I, with a nonnegative diagonal, and never
 * writes Q (the "Q-less QR" of the paper "Implementation of QR factorization of tall and
 * very skinny matrices on current GPUs", Sec. 1).  Three methods reach the same R:
 *   - Householder TSQR (Sec. 3.2, Algorithms 2-4): one pass over X;
 *   - Cholesky-QR2 (Sec. 3.1, Algorithm 1): two passes, Cholesky of the Gram matrix;
 *   - SVQB2 (Sec. 3.1): two passes, eigendecomposition of the Gram matrix.
 *
 * Conventions shared by every call:
 *   - X (and A, b) are column-major with leading dimension ld >= max(m, 1), stored as
 *     IEEE double (QL_F64) or float (QL_F32).  X is read, never written.
 *   - All matrix/vector pointers are DEVICE pointers unless stated otherwise; the caller
 *     owns them.  R is always double, column-major, leading dimension ldr >= n; its strict
 *     lower triangle is written as zero.
 *   - `stream` is a cudaStream_t passed as void* (NULL = legacy default stream).  Calls are
 *     asynchronous on that stream and need no host synchronisation between them.
 *   - `ws` is a device workspace of at least ql_workspace_bytes(...) bytes, 256-byte
 *     aligned, owned by the caller, and must not be shared by calls in flight at once.
 *   - `info` (nullable device pointer to int32[2]) receives {status, index} when the
 *     call's last kernel finishes: {QL_OK, 0}, {QL_ERR_NOT_SPD, pivot (1-based)},
 *     {QL_ERR_NONFINITE, 0}, {QL_ERR_TIMEOUT, where}.  It is written on every call.
 *   - The return value reports only synchronous errors (argument checks, launch errors).
 *     64-bit sizes are used throughout; m * ld may exceed 2^31.
 *
 * Arithmetic.  The m-proportional loops run in "double-float" arithmetic (an unevaluated
 * sum of two floats, about 48 significant bits) on the FP32 pipes by default, because the
 * FP64 pipe of this GPU is about 60x slower than its FP32 pipes; the n x n steps (R-tree,
 * Cholesky, eigensolve, back-substitution) always run in FP64.  Inputs whose magnitudes
 * fall outside the double-float range (see ql_set_arith) are detected on the device and
 * recomputed by the FP64 kernels inside the same call, with no host round trip.
 */
#ifndef QLESS_H
#define QLESS_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef int32_t ql_status;
enum {
  QL_OK = 0,
  QL_ERR_ARG = 1,        /* bad size, leading dimension, dtype or null pointer */
  QL_ERR_ALIGN = 2,      /* a pointer is not aligned to its element size */
  QL_ERR_WORKSPACE = 3,  /* workspace missing or smaller than ql_workspace_bytes() */
  QL_ERR_CUDA = 4,       /* a CUDA runtime call or kernel launch failed */
  QL_ERR_NOT_SPD = 5,    /* device info: Cholesky pivot <= 0; info[1] = pivot (1-based) */
  QL_ERR_TIMEOUT = 6,    /* device info: a bounded wait gave up */
  QL_ERR_NONFINITE = 7,  /* device info: R is not finite (NaN/Inf in X or overflow) */
  QL_ERR_BUDGET = 8,     /* server: request does not fit the HBM admission budget */
  QL_ERR_BUSY = 9,       /* server: result not ready yet / queue full */
  QL_ERR_UNKNOWN = 10    /* server: unknown ticket */
};

typedef int32_t ql_dtype;
enum { QL_F64 = 0, QL_F32 = 1 };

typedef int32_t ql_method;
enum { QL_TSQR = 0, QL_CHOLQR2 = 1, QL_SVQB2 = 2, QL_AUTO = 3, QL_SCHOLQR3 = 4 };

/* Arithmetic of the m-proportional loops.
 *   QL_ARITH_DF  (default) double-float on the FP32 pipes; the kernels check that every
 *                block-column maximum |x| lies in [2^-40, 2^50] (or is 0) and otherwise
 *                recompute the whole call in FP64 on the device.
 *   QL_ARITH_F64 native FP64 throughout (the baseline; about 10x slower on GB300). */
typedef int32_t ql_arith;
enum { QL_ARITH_DF = 0, QL_ARITH_F64 = 1 };

/* Process-wide arithmetic selection for subsequent calls (not for calls already queued).
 * Returns the previous setting.  Not synchronised with calls running on other threads. */
ql_arith ql_set_arith(ql_arith mode);

/* Library version and build identity, e.g. "qless 0.1 sm_103a". Static string. */
const char* ql_version(void);

/* Number of kernels this library has launched in this process (instrumentation for
 * benchmarks: every launch of every entry point, gated fallback launches included). */
uint64_t ql_launch_count(void);

/*
 * Measured compute-pipe throughput of the current device (measurement support for the
 * roofline of the arithmetic-bound kernels; the paper has no counterpart).  Fills out[5]
 * (host memory) with TFLOP/s: [0] FP32 FMA, [1] FP64 FMA, [2] FP64 tensor-core MMA
 * (mma.sync m8n8k4), [3] the library's double-float multiply-accumulate in FP64-equivalent
 * flops (2 per operation), [4] packed FP32 FMA (fma.rn.f32x2, two lanes per instruction).
 * Synchronous: launches five timed kernels (a few tens of ms
 * each) on `stream`, allocates and frees one small device buffer.  QL_ERR_ARG for a null
 * out, QL_ERR_CUDA if a launch or the timing fails.
 */
ql_status ql_measure_peaks(double* out, void* stream);

/*
 * Self-check of the device-side failure reporting (test support; the paper has no
 * counterpart).  One warp initialises an mbarrier and waits on it with the same bounded
 * wait the tensor-core kernels use, giving up after limit_clocks (0 < limit <= 2^34) SM
 * clocks.  arrive != 0: a thread arrives first and info = {QL_OK, 0}; arrive == 0: nothing
 * arrives, the wait runs out and info = {QL_ERR_TIMEOUT, 1}.  Nothing asynchronous is in
 * flight during the wait.  info: device int32[2] (required).  Asynchronous on stream.
 */
ql_status ql_check_bounded_wait(int32_t arrive, int64_t limit_clocks, int32_t* info, void* stream);

/* Device workspace bytes for one call of `method` on an m x n problem of `dtype`
 * (QL_AUTO: the maximum over the methods).  0 on bad arguments. */
size_t ql_workspace_bytes(ql_method method, int64_t m, int64_t n, ql_dtype dtype);

/*
 * Q-less Householder TSQR (Sec. 3.2, Algorithms 2-4).  One persistent launch: every CTA
 * streams its row blocks of X through shared memory, factors [R; W] in place with
 * Householder reflectors (Algorithm 4), and the per-CTA triangles are merged by a binary
 * "last CTA done" R-tree (Algorithm 2, stage 2) inside the same launch.  An FP64 fallback
 * launch follows that exits at once unless the range check fired.
 * Arguments: m >= 0 rows, 1 <= n <= 64 columns, X device (F64 or F32), ldx >= max(m,1),
 * R device double n x n (ldr >= n), info nullable device int32[2], ws/ws_bytes workspace.
 */
ql_status ql_tsqr_qless(int64_t m, int64_t n, const void* X, ql_dtype dtype, int64_t ldx, double* R,
                        int64_t ldr, int32_t* info, void* ws, size_t ws_bytes, void* stream);

/*
 * TSQR for callers that cannot allocate device memory (the paper has no counterpart: it is
 * an interface addition of this library).  Same computation, arguments, argument and
 * alignment checks (QL_ERR_ARG, QL_ERR_ALIGN before any device work) and tuned grid as
 * ql_tsqr_qless, without the workspace: code running while its stream is captured into a
 * CUDA graph may not call cudaMalloc, host callbacks must not, and extensions of
 * frameworks that route every device allocation through their own pools often have no
 * allocator to call.  The scratch lives in a fixed 4 MiB array inside the library that
 * every GPU loading the library keeps until the process exits; n <= 16 is supported (any
 * m), larger n returns QL_ERR_WORKSPACE (the capacity check uses the SM count of the device
 * current at the call).  No cudaMalloc, cudaFree or other allocating
 * call is made.  The first call on a device looks up the array's device address (with that
 * device current) and should come before any stream capture.  All calls share the one
 * array: calls that overlap on the GPU (different streams, or different host threads)
 * race and must be serialised by the caller.
 */
ql_status ql_tsqr_qless_noalloc(int64_t m, int64_t n, const void* X, ql_dtype dtype, int64_t ldx, double* R,
                                int64_t ldr, int32_t* info, void* stream);

/*
 * Q-less Cholesky-QR2 (Sec. 3.1, Algorithm 1): C = X^T X; R1 = chol(C); C = (X R1^{-1})^T
 * (X R1^{-1}) with X R1^{-1} formed tile by tile and never stored; R2 = chol(C); R = R2 R1.
 * Both Cholesky factorisations, R1^{-1} and R2 R1 run on the device in FP64.  A
 * non-positive pivot sets info = {QL_ERR_NOT_SPD, pivot} (+1000 for the second pass) and
 * fills R with NaN.  Reliable for kappa_2(X) up to about 1e6 (the Gram squares kappa).
 */
ql_status ql_cholqr2_qless(int64_t m, int64_t n, const void* X, ql_dtype dtype, int64_t ldx, double* R,
                           int64_t ldr, int32_t* info, void* ws, size_t ws_bytes, void* stream);

/*
 * Q-less shifted Cholesky-QR3 (the variant Sec. 1 cites for ill-conditioned X, robust for
 * kappa(X) up to about u^{-1/2}): three Gram passes over X.
 *   pass 1: C1 = X^T X, s = 11 (m n + n (n + 1)) u ||X||_F^2 with u = 2^-53 and
 *           ||X||_F^2 = trace(C1) standing in for ||X||_2^2 (an upper bound), R1 = chol(C1 + s I);
 *   pass 2: Y = X R1^{-1} formed tile by tile, R2 = chol(Y^T Y);
 *   pass 3: Y = X (R2 R1)^{-1}, R3 = chol(Y^T Y);  R = R3 R2 R1.
 * Arguments, workspace and outputs as ql_cholqr2_qless.  A non-positive pivot sets info =
 * {QL_ERR_NOT_SPD, pivot + 1000 (pass - 1)} and R = NaN.
 */
ql_status ql_scholqr3_qless(int64_t m, int64_t n, const void* X, ql_dtype dtype, int64_t ldx, double* R,
                            int64_t ldr, int32_t* info, void* ws, size_t ws_bytes, void* stream);

/*
 * Q-less SVQB2 (Sec. 3.1, SVQB applied twice): C = X^T X = U L U^T (FP64 Jacobi on the
 * device), B1 = U L^{-1/2} with eigenvalues below rank_tol * lambda_max treated as zero
 * (rank_tol <= 0 selects n * 2^-52); second pass on X B1 (formed tile by tile); then
 * X = Q Z with Z = L2^{1/2} U2^T L1^{1/2} U1^T and R = qr_r(Z) (FP64 Householder on the
 * device).  Z (nullable device double n x n, ld n) receives Z.
 */
ql_status ql_svqb_qless(int64_t m, int64_t n, const void* X, ql_dtype dtype, int64_t ldx, double* R,
                        int64_t ldr, double* Z, double rank_tol, int32_t* info, void* ws, size_t ws_bytes,
                        void* stream);

/*
 * Least squares min_x ||A x - b||_2 with one pass over the data (Sec. 1): the Q-less QR of
 * the extended matrix [A b] gives R_ext = [[R, z], [0, rho]], then x = R^{-1} z (FP64
 * back-substitution on the device) and ||b - A x|| = rho.  A is m x n (lda >= m), b has m
 * entries (contiguous), both of `dtype`; [A b] is read in place, never copied.  method is
 * QL_TSQR, QL_CHOLQR2 or QL_SCHOLQR3 (QL_AUTO: the tuner's choice, TSQR without a table).  x (device double[n]), resnorm (device double[1]);
 * Rext (nullable device double (n+1) x (n+1), ld n+1).  1 <= n <= 63.  A zero diagonal
 * entry of R sets info = {QL_ERR_NOT_SPD, i} and x = NaN.
 */
ql_status ql_lstsq_qless(int64_t m, int64_t n, const void* A, int64_t lda, const void* b, ql_dtype dtype,
                         ql_method method, double* x, double* resnorm, double* Rext, int32_t* info, void* ws,
                         size_t ws_bytes, void* stream);

/*
 * Q reconstruction: Q = X R^{-1}, the orthonormal factor of X = Q R (the explicit Q of
 * Sec. 1 that block iterative solvers need), for the R returned by any of the Q-less
 * calls above (n x n upper triangular, FP64, device, ld ldr >= n).  X is m x n of `dtype`
 * (ldx >= m); Q (device, m x n, ldq >= m) receives Q in the same dtype; X and Q may not
 * overlap.  One launch, no workspace: every CTA inverts R in FP64 and forms its rows of Q
 * in double-float, or in FP64 for row tiles outside the double-float exponent range.  A zero
 * diagonal entry of R sets info = {QL_ERR_NOT_SPD, i} (1-based) and Q = NaN.
 */
ql_status ql_q_from_r(int64_t m, int64_t n, const void* X, ql_dtype dtype, int64_t ldx, const double* R,
                      int64_t ldr, void* Q, int64_t ldq, int32_t* info, void* stream);

/*
 * Two-phase orthogonalisation: the "two-phase problem" QR = (I - Y Y^T) X with
 * re-orthogonalisation that Sec. 2 discusses, for Y (m x k, orthonormal columns, 1 <= k <=
 * 64, ld ldy) and X (m x n, 1 <= n <= 64, ld ldx), both of `dtype`:
 *   C1 = Y^T X,  W1 = X - Y C1,  C2 = Y^T W1,  W = W1 - Y C2,
 * W (device, m x n of dtype, ld ldw; may be X itself) receives the projected block and C
 * (device double k x n, ld ldc >= k) the coefficients C1 + C2, so X = Y C + W.  The R of the
 * orthogonalised block is any Q-less call on W.  Four launches; the Y^T V products are
 * reduced in a fixed order (reproducible).  ws: ql_project_workspace_bytes(k, n) bytes.
 */
size_t ql_project_workspace_bytes(int64_t k, int64_t n);
ql_status ql_project_out(int64_t m, int64_t k, const void* Y, int64_t ldy, int64_t n, const void* X, int64_t ldx,
                         ql_dtype dtype, void* W, int64_t ldw, double* C, int64_t ldc, void* ws, size_t ws_bytes,
                         void* stream);

/*
 * QR of wider matrices (65 <= n <= 4096; any n >= 1 works): the hybrid of block
 * Gram-Schmidt and TSQR panels that the paper's outlook names beyond the very-skinny
 * regime.  Panels of 64 columns, left to right: each is projected twice against all earlier
 * panels' Q (ql_project_out; the coefficients are R's off-diagonal blocks), factored by TSQR
 * (R's diagonal block) and turned into its Q by ql_q_from_r.  R (device double n x n, ld
 * ldr, lower triangle zeroed); Q (device m x n of dtype, ld ldq) receives the orthonormal
 * factor; info (nullable) the first failing call's {status, index}.  No allocation:
 * ws of ql_qr_wide_workspace_bytes(m, n, dtype) bytes.  Every step runs on `stream`.
 */
size_t ql_qr_wide_workspace_bytes(int64_t m, int64_t n, ql_dtype dtype);
ql_status ql_qr_wide(int64_t m, int64_t n, const void* X, ql_dtype dtype, int64_t ldx, double* R, int64_t ldr,
                     void* Q, int64_t ldq, int32_t* info, void* ws, size_t ws_bytes, void* stream);

/* ------------------------------------------------------------------ batched form */

/* One problem of a batch.  All pointers are device pointers. */
typedef struct {
  int64_t m, n, ld;      /* 0 <= m, 1 <= n <= 64, ld >= max(m, 1) */
  const void* X;         /* column-major m x n */
  ql_dtype dtype;        /* QL_F64 or QL_F32 */
  int32_t kind;          /* 0: R only; 1: least squares on [X b] with b = `b` */
  const void* b;         /* kind 1: right-hand side (m entries, dtype) */
  double* R;             /* n x n (kind 0) or (n+1) x (n+1) (kind 1), ld = rows */
  double* x;             /* kind 1: solution (n entries) and x[n] = residual norm */
  int32_t* info;         /* nullable int32[2] */
  int32_t method_hint;   /* QL_AUTO (0 in a zeroed struct is QL_TSQR; set QL_AUTO to let the
                            tuner choose), QL_TSQR or QL_CHOLQR2 */
  double kappa_hint;     /* estimate of kappa_2(X); <= 0: unknown (the Gram method is only
                            chosen automatically for a known kappa_hint <= 1e6) */
} ql_problem;

/*
 * Many uneven problems, each by its own method (Householder TSQR, Sec. 3.2, or
 * Cholesky-QR2, Sec. 3.1, Algorithm 1).  probs: HOST array of `count` problems.  The method
 * of a problem is its method_hint, or for QL_AUTO the autotune table entry of its
 * (m, n, dtype, kappa) class (ql_autotune), else Cholesky-QR2 from 24 columns when
 * 0 < kappa_hint <= 1e6 and TSQR otherwise; the Gram method needs n (+1 for least squares)
 * >= 9, narrower problems always run TSQR.  All TSQR problems run in ONE persistent launch
 * (work list of row-tile chunks, per-problem R-trees); the Cholesky-QR2 problems run as
 * work items of one persistent launch per (column class, storage, pass) of the
 * tensor-core Gram kernels.  A problem that leaves the double-float range, or (QL_AUTO)
 * whose Cholesky breaks down, is redone by a final gated FP64 TSQR launch.  The plan lives
 * in `ws` (ql_batch_workspace_bytes) and is rebuilt on every call.  Equivalent, problem by
 * problem, to the single-call entry points up to rounding order.
 */
size_t ql_batch_workspace_bytes(int32_t count, const ql_problem* probs);
ql_status ql_batch_qless(int32_t count, const ql_problem* probs, void* ws, size_t ws_bytes, void* stream);

/* The two halves of ql_batch_qless.  ql_batch_prepare builds the plan on the host, uploads
 * it into `ws` and waits for the upload (not capturable).  ql_batch_launch clears the
 * counters and launches the persistent kernel(s) of the plan last prepared in `ws`; it
 * makes no host synchronisation and allocates nothing, so it can be captured in a CUDA
 * graph and replayed (the first launch of the process should happen before capture). */
ql_status ql_batch_prepare(int32_t count, const ql_problem* probs, void* ws, size_t ws_bytes, void* stream);
ql_status ql_batch_launch(void* ws, void* stream);
/* The method chosen for each problem of the plan last prepared in `ws` (QL_TSQR or
 * QL_CHOLQR2, in the caller's order; count must equal the batch's).  Host only. */
ql_status ql_batch_methods(void* ws, int32_t* methods, int32_t count);

/*
 * Autotuner: times the candidate configurations (rows per CTA tile, CTAs per SM, method)
 * for an m x n problem of `dtype` on the current device using scratch inputs in `ws`
 * (ql_autotune_workspace_bytes), records the fastest one that meets the accuracy model
 * for kappa_hint (CholQR2 only when kappa_hint <= 1e6), and returns the chosen method in
 * *method_out and its time in *ms_out.  Results stay in a process-wide table that later
 * calls consult; ql_autotune_save/load persist it as JSON text.
 */
size_t ql_autotune_workspace_bytes(int64_t m, int64_t n, ql_dtype dtype);
ql_status ql_autotune(int64_t m, int64_t n, ql_dtype dtype, double kappa_hint, void* ws, size_t ws_bytes,
                      void* stream, ql_method* method_out, double* ms_out);
ql_status ql_autotune_save(const char* path);
ql_status ql_autotune_load(const char* path);
/* Method the tuner picks for (m, n, dtype, kappa_hint) without timing (table or model). */
ql_method ql_autotune_choose(int64_t m, int64_t n, ql_dtype dtype, double kappa_hint);

/* ------------------------------------------------------------------ serving loop */

typedef struct ql_server ql_server;

typedef struct {
  int64_t m, n, ld;
  const void* X;      /* device, stays valid until the result is polled */
  ql_dtype dtype;
  int32_t kind;       /* 0: R only; 1: least squares on [X b] */
  const void* b;      /* kind 1 */
  double kappa_hint;  /* <= 0: unknown */
  int32_t method_hint; /* as ql_problem::method_hint */
} ql_request;

typedef struct {
  ql_status status;   /* QL_OK or the device info status */
  int32_t index;      /* device info index */
  double latency_ms;  /* submit -> result ready on the device (host clock) */
  double* R;          /* device pointer owned by the server until ql_server_release */
  double* x;          /* kind 1: device solution (n entries) then the residual norm */
} ql_result;

typedef struct {
  int64_t submitted, completed, rejected, in_flight;
  double p50_ms, p99_ms, mean_ms, solves_per_s;
  double hbm_in_use_bytes, hbm_peak_bytes;
} ql_stats;

/*
 * A continuous-batching server on the current device: a scheduler thread admits queued
 * requests while the HBM budget (request data is not counted: it belongs to the caller;
 * the budget covers the server's workspaces and outputs) and `max_slots` allow, launches
 * each admitted group as one batched persistent kernel on one of `streams` CUDA streams,
 * so groups overlap on the device, and completes them as their events fire.
 *
 * The server's streams are non-blocking and wait on nothing of the caller's: a request's
 * X and b must be complete in device memory when it is submitted (synchronise the stream
 * that produced them first), and must stay unchanged until the request completes.
 */
ql_server* ql_server_create(size_t hbm_budget_bytes, int32_t max_slots, int32_t streams);
ql_status ql_server_submit(ql_server* s, const ql_request* req, uint64_t* ticket);
/* QL_OK with *out filled when done, QL_ERR_BUSY while pending, QL_ERR_UNKNOWN otherwise. */
ql_status ql_server_poll(ql_server* s, uint64_t ticket, ql_result* out);
/* Frees the result's device buffers (returns them to the budget). */
ql_status ql_server_release(ql_server* s, uint64_t ticket);
/* Withdraws a request that is still queued (not yet admitted to a group): QL_OK, and the
 * ticket becomes unknown; QL_ERR_BUSY once it has been launched (it then completes and is
 * polled and released as usual); QL_ERR_UNKNOWN for an unknown ticket. */
ql_status ql_server_cancel(ql_server* s, uint64_t ticket);
ql_status ql_server_drain(ql_server* s, double timeout_s);
ql_status ql_server_stats(ql_server* s, ql_stats* out);
void ql_server_destroy(ql_server* s);

#ifdef __cplusplus
}
#endif
#endif /* QLESS_H */
