// Device-side check of the library's failure reporting: the bounded mbarrier wait that the
// tensor-core kernels use gives up after its limit and the kernel reports
// {QL_ERR_TIMEOUT, where} through `info` instead of hanging.  Test support, not part of the
// paper's method.  No copy, MMA or other asynchronous operation is in flight while it waits,
// so giving up leaves nothing behind.
#include "gram_umma.cuh"
#include "epilogue.cuh"
#include "internal.h"

namespace ql {

// One warp.  arrive = 1: thread 0 arrives on the barrier before the wait (the phase
// completes, QL_OK); arrive = 0: nothing arrives and the wait runs out after `limit` clocks.
__global__ void bounded_wait_check_kernel(int arrive, long long limit, int32_t* info) {
  __shared__ __align__(8) uint64_t mbar;
  if (threadIdx.x == 0) mbar_init(&mbar, 1);
  __syncthreads();
  if (arrive && threadIdx.x == 0) mbar_arrive(&mbar);
  const bool done = mbar_wait_bounded(&mbar, 0, limit);
  const bool all = __syncthreads_and(done);
  if (all)
    write_info(info, QL_OK, 0);
  else
    write_info(info, QL_ERR_TIMEOUT, 1);
}

}  // namespace ql

using namespace ql;

extern "C" ql_status ql_check_bounded_wait(int32_t arrive, int64_t limit_clocks, int32_t* info, void* stream) {
  if (!info || limit_clocks < 0 || limit_clocks > (1ll << 34)) return QL_ERR_ARG;
  count_launch();
  bounded_wait_check_kernel<<<1, 32, 0, (cudaStream_t)stream>>>(arrive ? 1 : 0, limit_clocks, info);
  return cudaPeekAtLastError() == cudaSuccess ? QL_OK : QL_ERR_CUDA;
}
