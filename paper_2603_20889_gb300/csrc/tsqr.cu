// Host launcher of the Q-less Householder TSQR (paper Sec. 3.2, Algorithms 2-4).
//
// One persistent launch per call: CTA i factors tiles [t0_i, t1_i) of X into its triangle
// (tsqr.cuh), stores it as leaf i of a binary R-tree and climbs the tree; the CTA that
// completes the root writes R (or solves the least-squares problem of [A b]).  When the
// double-float launch finds data outside its exponent range it leaves R unwritten and
// raises a flag; the FP64 launch queued behind it runs only in that case.
#include <atomic>
#include <cstdlib>

#include "tsqr_launch.cuh"

namespace ql {

int tsqr_variant() {
  static const int v = [] {
    const char* e = std::getenv("QL_TSQR_CFG");
    return e ? std::atoi(e) : 0;
  }();
  return v;
}

int device_sm_count() {
  // cached per device: a process may drive GPUs with different SM counts
  constexpr int kMaxDev = 64;
  static std::atomic<int> sms[kMaxDev] = {};
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= kMaxDev) dev = 0;
  int v = sms[dev].load(std::memory_order_relaxed);
  if (v > 0) return v;
  if (cudaDeviceGetAttribute(&v, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess || v <= 0) v = 1;
  sms[dev].store(v, std::memory_order_relaxed);
  return v;
}

size_t tsqr_workspace_bytes(int n) {
  if (n < 1 || n > kMaxN) return 0;
  size_t leaves = (size_t)device_sm_count() * kMaxCtasPerSm;
  size_t cnt = tree_counters((int)leaves);
  size_t head = 256 + (cnt * sizeof(int) + 255) / 256 * 256;
  return head + tree_slots((int)leaves) * (size_t)n * n * sizeof(double);
}

ql_status tsqr_launch(const TsqrCall& c, ql_arith arith) {
  if (c.n < 1 || c.n > kMaxN) return QL_ERR_ARG;
  const int sms = device_sm_count();
  size_t leaves_max = (size_t)sms * kMaxCtasPerSm;
  size_t cnt = tree_counters((int)leaves_max);
  size_t head = 256 + (cnt * sizeof(int) + 255) / 256 * 256;
  size_t need = head + tree_slots((int)leaves_max) * (size_t)c.n * c.n * sizeof(double);
  if (!c.ws || c.ws_bytes < need) return QL_ERR_WORKSPACE;
  unsigned char* ws = static_cast<unsigned char*>(c.ws);
  TreeView tv;
  tv.flags = reinterpret_cast<int*>(ws);
  tv.counters = reinterpret_cast<int*>(ws + 256);
  tv.slots = reinterpret_cast<double*>(ws + head);
  tv.leaves = 0;
  if (cudaMemsetAsync(ws, 0, head, c.stream) != cudaSuccess) return QL_ERR_CUDA;
  ql_status st;
  if (c.dtype == QL_F64) {
    if (arith == QL_ARITH_F64) return dispatch<double, ArithF64>(c, tv, 0);
    st = dispatch<double, ArithDF>(c, tv, 0);
    if (st != QL_OK) return st;
    return dispatch<double, ArithF64>(c, tv, 1);
  } else {
    if (arith == QL_ARITH_F64) return dispatch<float, ArithF64>(c, tv, 0);
    st = dispatch<float, ArithDF>(c, tv, 0);
    if (st != QL_OK) return st;
    return dispatch<float, ArithF64>(c, tv, 1);
  }
}

}  // namespace ql
