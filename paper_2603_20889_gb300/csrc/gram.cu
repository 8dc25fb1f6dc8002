// Host launcher of the Q-less Gram methods (paper Sec. 3.1): Cholesky-QR2 (Algorithm 1)
// and SVQB2.  Two launches per call (first pass, second pass); after the double-float
// pair, two gated FP64 launches follow that run only if the range check fired.
#include "gram_launch.cuh"

#include <cstdlib>

namespace ql {

bool tc_gram_enabled() {
  static const bool on = [] {
    const char* v = std::getenv("QL_GRAM_SIMT");
    return !(v && v[0] == '1');
  }();
  return on;
}

bool pipe_gram_enabled() {
  static const bool on = [] {
    const char* v = std::getenv("QL_GRAM_PIPE");
    return !(v && v[0] == '0');
  }();
  return on;
}

static int nc_of(int n) { return n <= 1 ? 1 : n <= 2 ? 2 : n <= 4 ? 4 : n <= 8 ? 8 : n <= 16 ? 16 : n <= 32 ? 32 : 64; }

static size_t gram_layout(int n, GramWs* w, void* base) {
  const int nc = nc_of(n);
  const size_t head = 512;  // flags, counters and the first pass's column exponents
  const size_t keep = ((size_t)3 * nc * nc * sizeof(double) + 255) / 256 * 256;  // 3 n x n blocks (ld n)
  // one NC x NC partial per CTA (the streaming kernel for nc <= 4 runs up to 8 CTAs per SM)
  const size_t parts = (size_t)device_sm_count() * (nc <= 4 ? 8 : kGramMaxCtasPerSm) * nc * nc * sizeof(double);
  // FP64 accumulators of the tcgen05 kernels (16 to 64 columns, one CTA per SM)
  const size_t fbuf = nc >= 16 ? (size_t)device_sm_count() * nc * 128 * sizeof(double) : 0;
  if (w && base) {
    unsigned char* b = static_cast<unsigned char*>(base);
    w->flags = reinterpret_cast<int*>(b);
    w->keep = reinterpret_cast<double*>(b + head);
    w->partials = reinterpret_cast<double*>(b + head + keep);
    w->fbuf = reinterpret_cast<double*>(b + head + keep + parts);
  }
  return head + keep + parts + fbuf;
}

size_t gram_workspace_bytes(int n) {
  if (n < 1 || n > kMaxN) return 0;
  return gram_layout(n, nullptr, nullptr);
}

ql_status gram_launch(const GramCall& c, ql_arith arith) {
  if (c.n < 1 || c.n > kMaxN) return QL_ERR_ARG;
  if (c.method != QL_CHOLQR2 && c.method != QL_SVQB2 && c.method != QL_SCHOLQR3 &&
      !(c.method == QL_TSQR && c.n == 1 && c.epilogue == kEpiR))
    return QL_ERR_ARG;
  if (!c.ws || c.ws_bytes < gram_layout(c.n, nullptr, nullptr)) return QL_ERR_WORKSPACE;
  GramWs w;
  gram_layout(c.n, &w, c.ws);
  if (cudaMemsetAsync(w.flags, 0, 512, c.stream) != cudaSuccess) return QL_ERR_CUDA;
  ql_status st;
  if (c.dtype == QL_F64) {
    if (arith == QL_ARITH_F64) return gram_dispatch<double, ArithF64>(c, w, 0);
    if ((st = gram_dispatch<double, ArithDF>(c, w, 0))) return st;
    return gram_dispatch<double, ArithF64>(c, w, 1);
  }
  if (arith == QL_ARITH_F64) return gram_dispatch<float, ArithF64>(c, w, 0);
  if ((st = gram_dispatch<float, ArithDF>(c, w, 0))) return st;
  return gram_dispatch<float, ArithF64>(c, w, 1);
}

}  // namespace ql
