// Q-less TSQR for callers that cannot allocate device memory.
//
// The regular entry point takes a caller-allocated workspace (R-tree triangles, arrival
// counters, flags).  Some callers cannot obtain one: code that runs while a stream is
// being captured into a CUDA graph (cudaMalloc is not allowed during capture), host
// callbacks, and plugins of frameworks that own every device allocation through their own
// pool and expose no allocator to their extensions.  This variant keeps its scratch in a
// file-scope device array of fixed size instead, so it calls no cudaMalloc, cudaFree or
// allocating library routine.  The array is loaded with the library and stays resident on
// every GPU that loads it until the process exits.
#include <mutex>

#include "internal.h"

namespace ql {

// Scratch capacity: enough for the R-tree of up to kMaxCtasPerSm CTAs per SM on 152 SMs
// with n <= 16 columns (1216 triangle slots of 16 x 16 doubles plus counters and flags).
constexpr size_t kNoAllocScratchBytes = 4u << 20;  // 4 MiB
constexpr int kNoAllocMaxN = 16;

static __device__ __align__(256) unsigned char g_tsqr_scratch[kNoAllocScratchBytes];

// Device address of the scratch array, looked up once per device with that device current.
// In host code the array's name is only a host-side stand-in, never a device address.
static constexpr int kMaxDevices = 64;
static void* g_scratch_addr[kMaxDevices] = {};
static std::mutex g_scratch_mu;

static ql_status scratch_for_current_device(void** out) {
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= kMaxDevices) return QL_ERR_CUDA;
  std::lock_guard<std::mutex> lk(g_scratch_mu);
  if (!g_scratch_addr[dev]) {
    void* p = nullptr;
    if (cudaGetSymbolAddress(&p, g_tsqr_scratch) != cudaSuccess || !p) return QL_ERR_CUDA;
    g_scratch_addr[dev] = p;
  }
  *out = g_scratch_addr[dev];
  return QL_OK;
}

}  // namespace ql

using namespace ql;

extern "C" ql_status ql_tsqr_qless_noalloc(int64_t m, int64_t n, const void* X, ql_dtype dtype, int64_t ldx,
                                           double* R, int64_t ldr, int32_t* info, void* stream) {
  // the same argument and alignment checks as ql_tsqr_qless, before any device work
  ql_status st = check_matrix(m, n, X, dtype, ldx, kApiMaxN);
  if (st) return st;
  if ((st = check_r(R, ldr, n))) return st;
  if (n > kNoAllocMaxN) return QL_ERR_WORKSPACE;  // beyond what the fixed scratch array holds
  // the R-tree is sized for the SM count of the current device
  if (tsqr_workspace_bytes((int)n) > kNoAllocScratchBytes) return QL_ERR_WORKSPACE;
  void* scratch = nullptr;
  st = scratch_for_current_device(&scratch);
  if (st != QL_OK) return st;
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
  c.ws = scratch;
  c.ws_bytes = kNoAllocScratchBytes;
  c.stream = (cudaStream_t)stream;
  int ctas = 0;  // the autotuned grid, as the regular entry point uses (a table lookup, no allocation)
  int var = -1, ar = 0;
  if (tune_lookup(m, n, dtype, 1.0, nullptr, &ctas, &var, &ar)) {
    c.ctas_per_sm = ctas;
    c.variant = var;
    c.arity = ar;
  }
  // tsqr_launch clears the counters and flags of the scratch on the stream before the
  // kernels run; the triangle slots are fully written before they are read.
  return tsqr_launch(c, current_arith());
}
