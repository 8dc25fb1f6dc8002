// The C ABI of include/qless.h: argument checks, workspace sizing and dispatch to the
// kernel launchers.  No computation happens here; every step of the path runs on the GPU.
#include <atomic>
#include <cstdint>
#include <cstring>

#include "internal.h"

namespace ql {

static std::atomic<int> g_arith{QL_ARITH_DF};
static std::atomic<unsigned long long> g_launches{0};
void count_launch() { g_launches.fetch_add(1, std::memory_order_relaxed); }
ql_arith current_arith() { return (ql_arith)g_arith.load(); }

bool elem_aligned(const void* p, ql_dtype dt) {
  uintptr_t a = (uintptr_t)p;
  return dt == QL_F64 ? (a % 8 == 0) : (a % 4 == 0);
}

ql_status check_matrix(int64_t m, int64_t n, const void* X, ql_dtype dt, int64_t ld, int nmax) {
  if (m < 0 || n < 1 || n > nmax) return QL_ERR_ARG;
  if (dt != QL_F64 && dt != QL_F32) return QL_ERR_ARG;
  if (ld < (m > 1 ? m : 1)) return QL_ERR_ARG;
  if (m > 0 && !X) return QL_ERR_ARG;
  if (X && !elem_aligned(X, dt)) return QL_ERR_ALIGN;
  return QL_OK;
}

ql_status check_r(const double* R, int64_t ldr, int64_t n) {
  if (!R || ldr < n) return QL_ERR_ARG;
  return ((uintptr_t)R % 8) ? QL_ERR_ALIGN : QL_OK;
}

}  // namespace ql

using namespace ql;

extern "C" {

ql_arith ql_set_arith(ql_arith mode) {
  if (mode != QL_ARITH_DF && mode != QL_ARITH_F64) return current_arith();
  return (ql_arith)g_arith.exchange(mode);
}

const char* ql_version(void) { return "qless 0.1 sm_103a"; }

uint64_t ql_launch_count(void) { return g_launches.load(); }

size_t ql_workspace_bytes(ql_method method, int64_t m, int64_t n, ql_dtype dtype) {
  (void)m;
  if (n < 1 || n > kApiMaxN || (dtype != QL_F64 && dtype != QL_F32)) return 0;
  size_t t = tsqr_workspace_bytes((int)(n + 1 <= kApiMaxN ? n + 1 : n));
  size_t g = gram_workspace_bytes((int)(n + 1 <= kApiMaxN ? n + 1 : n));
  switch (method) {
    case QL_TSQR: return n == 1 && g > t ? g : t;  // n = 1 runs the one-column streaming pass
    case QL_CHOLQR2:
    case QL_SCHOLQR3:
    case QL_SVQB2: return g;
    case QL_AUTO: return t > g ? t : g;
    default: return 0;
  }
}

ql_status ql_tsqr_qless(int64_t m, int64_t n, const void* X, ql_dtype dtype, int64_t ldx, double* R,
                        int64_t ldr, int32_t* info, void* ws, size_t ws_bytes, void* stream) {
  ql_status st = check_matrix(m, n, X, dtype, ldx, kApiMaxN);
  if (st) return st;
  if ((st = check_r(R, ldr, n))) return st;
  if (n == 1) {
    // one column: R = ||x||, the norm that the Householder reflector of x is built from,
    // streamed by the one-column Gram pass (no tiles, reflectors or R-tree needed)
    GramCall g;
    g.m = m;
    g.n = 1;
    g.nA = 1;
    g.A = X;
    g.lda = ldx;
    g.b = X;
    g.dtype = dtype;
    g.method = QL_TSQR;
    g.epilogue = kEpiR;
    g.R = R;
    g.ldr = ldr;
    g.info = info;
    g.ws = ws;
    g.ws_bytes = ws_bytes;
    g.stream = (cudaStream_t)stream;
    return gram_launch(g, current_arith());
  }
  TsqrCall c;
  c.m = m;
  c.n = (int)n;
  c.nA = (int)n;
  c.A = X;
  c.lda = ldx;
  c.b = X;
  c.dtype = dtype;
  c.epilogue = kEpiR;
  c.R = R;
  c.ldr = ldr;
  c.info = info;
  c.ws = ws;
  c.ws_bytes = ws_bytes;
  c.stream = (cudaStream_t)stream;
  int ctas = 0;
  int var = -1, ar = 0;
  if (tune_lookup(m, n, dtype, 1.0, nullptr, &ctas, &var, &ar)) {
    c.ctas_per_sm = ctas;
    c.variant = var;
    c.arity = ar;
  }
  return tsqr_launch(c, current_arith());
}

static ql_status gram_entry(int method, int64_t m, int64_t n, const void* X, ql_dtype dtype, int64_t ldx,
                            double* R, int64_t ldr, double* Z, double rank_tol, int32_t* info, void* ws,
                            size_t ws_bytes, void* stream) {
  ql_status st = check_matrix(m, n, X, dtype, ldx, kApiMaxN);
  if (st) return st;
  if ((st = check_r(R, ldr, n))) return st;
  GramCall c;
  c.m = m;
  c.n = (int)n;
  c.nA = (int)n;
  c.A = X;
  c.lda = ldx;
  c.b = X;
  c.dtype = dtype;
  c.method = method;
  c.epilogue = kEpiR;
  c.R = R;
  c.ldr = ldr;
  c.Z = Z;
  c.rank_tol = rank_tol;
  c.info = info;
  c.ws = ws;
  c.ws_bytes = ws_bytes;
  c.stream = (cudaStream_t)stream;
  return gram_launch(c, current_arith());
}

ql_status ql_cholqr2_qless(int64_t m, int64_t n, const void* X, ql_dtype dtype, int64_t ldx, double* R,
                           int64_t ldr, int32_t* info, void* ws, size_t ws_bytes, void* stream) {
  return gram_entry(QL_CHOLQR2, m, n, X, dtype, ldx, R, ldr, nullptr, 0.0, info, ws, ws_bytes, stream);
}

ql_status ql_scholqr3_qless(int64_t m, int64_t n, const void* X, ql_dtype dtype, int64_t ldx, double* R,
                            int64_t ldr, int32_t* info, void* ws, size_t ws_bytes, void* stream) {
  return gram_entry(QL_SCHOLQR3, m, n, X, dtype, ldx, R, ldr, nullptr, 0.0, info, ws, ws_bytes, stream);
}

ql_status ql_svqb_qless(int64_t m, int64_t n, const void* X, ql_dtype dtype, int64_t ldx, double* R,
                        int64_t ldr, double* Z, double rank_tol, int32_t* info, void* ws, size_t ws_bytes,
                        void* stream) {
  return gram_entry(QL_SVQB2, m, n, X, dtype, ldx, R, ldr, Z, rank_tol, info, ws, ws_bytes, stream);
}

ql_status ql_lstsq_qless(int64_t m, int64_t n, const void* A, int64_t lda, const void* b, ql_dtype dtype,
                         ql_method method, double* x, double* resnorm, double* Rext, int32_t* info, void* ws,
                         size_t ws_bytes, void* stream) {
  ql_status st = check_matrix(m, n, A, dtype, lda, kApiMaxN - 1);
  if (st) return st;
  if ((m > 0 && !b) || !x || !resnorm) return QL_ERR_ARG;
  if (b && !elem_aligned(b, dtype)) return QL_ERR_ALIGN;
  if (method == QL_AUTO) method = ql_autotune_choose(m, n + 1, dtype, 1.0);
  if (method == QL_TSQR) {
    TsqrCall c;
    c.m = m;
    c.n = (int)n + 1;
    c.nA = (int)n;
    c.A = A;
    c.lda = lda;
    c.b = b;
    c.dtype = dtype;
    c.epilogue = kEpiLstsq;
    c.x = x;
    c.resnorm = resnorm;
    c.Rext = Rext;
    c.info = info;
    c.ws = ws;
    c.ws_bytes = ws_bytes;
    c.stream = (cudaStream_t)stream;
    return tsqr_launch(c, current_arith());
  }
  if (method == QL_CHOLQR2 || method == QL_SVQB2 || method == QL_SCHOLQR3) {
    GramCall c;
    c.m = m;
    c.n = (int)n + 1;
    c.nA = (int)n;
    c.A = A;
    c.lda = lda;
    c.b = b;
    c.dtype = dtype;
    c.method = method;
    c.epilogue = kEpiLstsq;
    c.x = x;
    c.resnorm = resnorm;
    c.Rext = Rext;
    c.info = info;
    c.ws = ws;
    c.ws_bytes = ws_bytes;
    c.stream = (cudaStream_t)stream;
    return gram_launch(c, current_arith());
  }
  return QL_ERR_ARG;
}

}  // extern "C"
