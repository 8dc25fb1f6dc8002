// Grouped Gram passes of the batched form: the Cholesky-QR2 problems of a batch with at
// least 9 columns run on the tensor-core Gram kernels (the first pass on gram_pipe_body;
// the second on gram_tc_body for column classes 16 and 32, gram_umma_body for 64), one
// persistent launch per (column class, storage, pass).
// Every CTA claims (problem, chunk) work items from one atomic counter and runs the same
// body as the single-call kernels on that chunk's row tiles, as partial `chunk` of the
// problem's `nchunks`; the last chunk of a problem to finish runs its epilogue (the FP64
// n x n work of the pass) exactly as the last CTA of a single call does.
#include "batch_gram.h"
#include "gram_launch.cuh"

namespace ql {

// Claim the next work item: (item index, chunk) or false when the list is exhausted.  The
// two shared slots live past the body's shared memory.
template <typename Item>
QL_DEV bool claim(int* counter, const Item* items, int count, int64_t total, int64_t* s_work, int* s_item,
                  int64_t& w, int& idx) {
  if (threadIdx.x == 0) {
    const int64_t v = atomicAdd(counter, 1);
    int lo = 0, hi = count - 1;
    while (lo < hi) {  // last item whose work_begin <= v (items ordered by work_begin)
      const int mid = (lo + hi + 1) >> 1;
      if (items[mid].work_begin <= v)
        lo = mid;
      else
        hi = mid - 1;
    }
    *s_work = v;
    *s_item = lo;
  }
  __syncthreads();
  w = *s_work;
  idx = *s_item;
  __syncthreads();
  return w < total;
}

template <int NC, typename S, int XF>
__global__ void __launch_bounds__(256, 1)
    gram_tc_group_kernel(int* counter, const GramGroupItem* items, int count, int64_t total, int pass) {
  using Sm = TcSmem<NC, S>;
  extern __shared__ __align__(16) unsigned char smem[];
  int64_t* s_work = reinterpret_cast<int64_t*>(smem + (Sm::kBytes + 15) / 16 * 16);
  int* s_item = reinterpret_cast<int*>(s_work + 1);
  int64_t w;
  int idx;
  while (claim(counter, items, count, total, s_work, s_item, w, idx)) {
    GramArgs<S> a = *reinterpret_cast<const GramArgs<S>*>(&items[idx].args);
    a.pass = pass;
    gram_tc_body<NC, S, XF>(a, (int)(w - items[idx].work_begin), items[idx].nchunks);
    __syncthreads();
  }
}

template <int NC, typename S, int XF>
__global__ void __launch_bounds__(umma_threads<XF>(), 1)
    gram_umma_group_kernel(int* counter, const GramGroupItem* items, int count, int64_t total, int pass) {
  using Sh = UmmaShape<NC>;
  using Sm = UmmaSmem<NC, S>;
  extern __shared__ __align__(1024) unsigned char smem_umma[];
  int64_t* s_work = reinterpret_cast<int64_t*>(smem_umma + (Sm::kBytes + 15) / 16 * 16);
  int* s_item = reinterpret_cast<int*>(s_work + 1);
  uint32_t* tslot = reinterpret_cast<uint32_t*>(s_item + 1);
  // tensor memory and the barriers once per CTA: a CTA gives up its allocation permit after
  // its first alloc, and a used barrier is not initialised again
  const uint32_t tbase = umma_cta_begin<NC, S>(smem_umma, tslot);
  UmmaBars bars;
  int64_t w;
  int idx;
  // a CTA whose bounded wait gave up takes no more work (the others drain the list)
  while (bars.ok && claim(counter, items, count, total, s_work, s_item, w, idx)) {
    GramArgs<S> a = *reinterpret_cast<const GramArgs<S>*>(&items[idx].args);
    a.pass = pass;
    gram_umma_body<NC, S, XF>(a, (int)(w - items[idx].work_begin), items[idx].nchunks, tbase, bars);
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
  }
  tc_fence_before();
  __syncthreads();
  if ((threadIdx.x >> 5) == 0) tmem_dealloc(tbase, Sh::TCOLS);
}

template <int NC, typename S>
__global__ void __launch_bounds__(PipeShape<NC>::T, 1)
    gram_pipe_group_kernel(int* counter, const GramGroupItem* items, int count, int64_t total, int pass) {
  using Sm = PipeSmem<NC, S>;
  extern __shared__ __align__(1024) unsigned char smem_umma[];
  int64_t* s_work = reinterpret_cast<int64_t*>(smem_umma + (Sm::kBytes + 15) / 16 * 16);
  int* s_item = reinterpret_cast<int*>(s_work + 1);
  // tensor memory and the barriers once per CTA (see gram_umma_group_kernel)
  const uint32_t tbase = pipe_cta_begin<NC, S>(smem_umma);
  PipeBars bars;
  int64_t w;
  int idx;
  while (bars.ok && claim(counter, items, count, total, s_work, s_item, w, idx)) {
    GramArgs<S> a = *reinterpret_cast<const GramArgs<S>*>(&items[idx].args);
    a.pass = pass;
    a.bulk = items[idx].tma;
    gram_pipe_body<NC, S>(a, (int)(w - items[idx].work_begin), items[idx].nchunks, tbase, bars, &items[idx].tmA,
                          items[idx].tma && a.src.nA < a.n ? &items[idx].tmB : nullptr);
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
  }
  tc_fence_before();
  __syncthreads();
  if ((threadIdx.x >> 5) == 0) tmem_dealloc(tbase, PipeShape<NC>::TCOLS);
}

template <typename K>
static ql_status launch_group(K kern, int threads, size_t smem, int* counter, const GramGroupItem* items, int count,
                              int64_t total, int pass, cudaStream_t st) {
  static std::mutex mu;
  {
    std::lock_guard<std::mutex> lk(mu);
    if (cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem) != cudaSuccess)
      return QL_ERR_CUDA;
  }
  int64_t grid = device_sm_count();  // one CTA per SM (the bodies' shared memory allows no second)
  if (grid > total) grid = total;
  if (grid < 1) grid = 1;
  count_launch();
  kern<<<(int)grid, threads, smem, st>>>(counter, items, count, total, pass);
  return cudaPeekAtLastError() == cudaSuccess ? QL_OK : QL_ERR_CUDA;
}

template <int NC, typename S>
static ql_status launch_class(int* counter, const GramGroupItem* items, int count, int64_t total, int pass,
                              cudaStream_t st) {
  if (pass == 1 && pipe_gram_enabled()) {
    constexpr size_t smem = (PipeSmem<NC, S>::kBytes + 15) / 16 * 16 + 32;
    return launch_group(gram_pipe_group_kernel<NC, S>, PipeShape<NC>::T, smem, counter, items, count, total, pass,
                        st);
  }
  if constexpr (NC == 64) {
    constexpr size_t smem = (UmmaSmem<NC, S>::kBytes + 15) / 16 * 16 + 32;
    if (pass == 1)
      return launch_group(gram_umma_group_kernel<NC, S, kXNone>, umma_threads<kXNone>(), smem, counter, items, count,
                          total, pass, st);
    return launch_group(gram_umma_group_kernel<NC, S, kXUpper>, umma_threads<kXUpper>(), smem, counter, items, count,
                        total, pass, st);
  } else {
    constexpr size_t smem = (TcSmem<NC, S>::kBytes + 15) / 16 * 16 + 32;
    if (pass == 1)
      return launch_group(gram_tc_group_kernel<NC, S, kXNone>, 256, smem, counter, items, count, total, pass, st);
    return launch_group(gram_tc_group_kernel<NC, S, kXUpper>, 256, smem, counter, items, count, total, pass, st);
  }
}

ql_status gram_group_launch(int nc, int dtype, int pass, int* counter, const GramGroupItem* items, int count,
                            int64_t total, cudaStream_t st) {
  if (count < 1 || total < 1) return QL_OK;
  if (dtype == QL_F64) {
    if (nc == 16) return launch_class<16, double>(counter, items, count, total, pass, st);
    if (nc == 32) return launch_class<32, double>(counter, items, count, total, pass, st);
    return launch_class<64, double>(counter, items, count, total, pass, st);
  }
  if (nc == 16) return launch_class<16, float>(counter, items, count, total, pass, st);
  if (nc == 32) return launch_class<32, float>(counter, items, count, total, pass, st);
  return launch_class<64, float>(counter, items, count, total, pass, st);
}

int gram_group_tile_rows(int nc) { return nc == 64 ? UmmaShape<64>::KT : (nc == 32 ? TcShape<32>::KT : TcShape<16>::KT); }

}  // namespace ql
