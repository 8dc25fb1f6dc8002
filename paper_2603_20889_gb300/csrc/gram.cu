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

bool pipe_gram2_enabled() {
  static const bool on = [] {
    const char* v = std::getenv("QL_GRAM_PIPE2");
    return !(v && v[0] == '0');
  }();
  return on;
}

bool pipe_tensor_maps(CUtensorMap* tmA, CUtensorMap* tmB, const void* A, const void* b, int dtype, int64_t m, int nA,
                      int64_t lda) {
  using Encode = CUresult (*)(CUtensorMap*, CUtensorMapDataType, cuuint32_t, void*, const cuuint64_t*,
                              const cuuint64_t*, const cuuint32_t*, const cuuint32_t*, CUtensorMapInterleave,
                              CUtensorMapSwizzle, CUtensorMapL2promotion, CUtensorMapFloatOOBfill);
  static const Encode encode = [] {
    void* fn = nullptr;
    cudaDriverEntryPointQueryResult q{};
    if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &fn, 12000, cudaEnableDefault, &q) != cudaSuccess ||
        q != cudaDriverEntryPointSuccess)
      return (Encode) nullptr;
    return reinterpret_cast<Encode>(fn);
  }();
  const size_t es = dtype == QL_F64 ? 8 : 4;
  auto aligned = [](const void* p) { return (reinterpret_cast<uintptr_t>(p) & 15u) == 0; };
  if (!encode || m < 1 || m >= (int64_t(1) << 31) || nA < 1 || nA > 256 || !aligned(A) || ((size_t)lda * es) % 16 ||
      (tmB && !aligned(b)))
    return false;
  const CUtensorMapDataType dt = dtype == QL_F64 ? CU_TENSOR_MAP_DATA_TYPE_FLOAT64 : CU_TENSOR_MAP_DATA_TYPE_FLOAT32;
  const cuuint32_t box_rows = (cuuint32_t)(128 / es), es1[2] = {1, 1};
  {
    const cuuint64_t dims[2] = {(cuuint64_t)m, (cuuint64_t)nA}, strides[1] = {(cuuint64_t)lda * es};
    const cuuint32_t box[2] = {box_rows, (cuuint32_t)nA};
    if (encode(tmA, dt, 2, const_cast<void*>(A), dims, strides, box, es1, CU_TENSOR_MAP_INTERLEAVE_NONE,
               CU_TENSOR_MAP_SWIZZLE_128B, CU_TENSOR_MAP_L2_PROMOTION_L2_256B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) !=
        CUDA_SUCCESS)
      return false;
  }
  if (tmB) {
    const cuuint64_t dims[2] = {(cuuint64_t)m, 1}, strides[1] = {((cuuint64_t)m * es + 15) / 16 * 16};
    const cuuint32_t box[2] = {box_rows, 1};
    // unswizzled: its box lands at line kb NC + nA, 128-byte but not 1024-byte aligned
    if (encode(tmB, dt, 2, const_cast<void*>(b), dims, strides, box, es1, CU_TENSOR_MAP_INTERLEAVE_NONE,
               CU_TENSOR_MAP_SWIZZLE_NONE, CU_TENSOR_MAP_L2_PROMOTION_L2_256B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) !=
        CUDA_SUCCESS)
      return false;
  }
  return true;
}

static int nc_of(int n) { return n <= 1 ? 1 : n <= 2 ? 2 : n <= 4 ? 4 : n <= 8 ? 8 : n <= 16 ? 16 : n <= 32 ? 32 : 64; }

static size_t gram_layout(int n, GramWs* w, void* base) {
  const int nc = nc_of(n);
  const size_t head = 512;  // flags, counters and the first pass's column exponents
  const size_t keep = ((size_t)3 * nc * nc * sizeof(double) + 255) / 256 * 256;  // 3 n x n blocks (ld n)
  // one NC x NC partial per CTA (the streaming kernel for nc <= 4 runs up to 8 CTAs per SM)
  const size_t parts = (size_t)device_sm_count() * (nc <= 4 ? 8 : kGramMaxCtasPerSm) * nc * nc * sizeof(double);
  // accumulators of the tcgen05 kernels (16 to 64 columns, one CTA per SM): an FP64 and a
  // double-float level per CTA (the per-tile kernel of the later passes uses the first)
  const size_t fbuf = nc >= 16 ? (size_t)device_sm_count() * nc * 128 * 2 * sizeof(double) : 0;
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
