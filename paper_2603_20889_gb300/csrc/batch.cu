// Batched Q-less QR: many uneven problems, each by the method chosen for it.
//
// Method per problem: the caller's method_hint, or for QL_AUTO the autotune table entry of
// its (m, n, dtype, kappa) class, else a model (Cholesky-QR2 from 24 columns when
// 0 < kappa_hint <= 1e6, where the tensor-core Gram passes outrun the Householder tiles;
// TSQR otherwise).  The Gram method covers n >= 9 (tensor-core kernels); narrower problems
// always run TSQR.
//
// TSQR problems run in ONE persistent launch.  The host plan splits every problem into
// chunks of row tiles (the leaves of that problem's R-tree) and orders the problems by
// decreasing work.  A fixed grid of persistent CTAs claims chunks through one atomic
// counter; a CTA factors its chunk with the single-problem tile machinery (tsqr.cuh) of
// the problem's column class, stores the leaf triangle and climbs that problem's tree;
// whoever completes a root writes R (or the least-squares solution).
//
// Cholesky-QR2 problems run as work items of grouped persistent Gram launches, one per
// (column class, storage, pass) (batch_gram.cu).  Stream order: the Gram first passes, the
// TSQR launch, the Gram second passes, then a gated FP64 TSQR launch that redoes every
// flagged problem -- TSQR problems whose data leave the double-float range, and Gram
// problems that left it or (method chosen automatically) whose Cholesky broke down.
#include <algorithm>
#include <cstddef>
#include <cstring>
#include <mutex>
#include <vector>

#include "batch_gram.h"
#include "epilogue.cuh"
#include "internal.h"
#include "tsqr.cuh"

namespace ql {

// Column classes of the batched TSQR kernel: NC, TC, RPT at T = 256 threads (for n > 8 the
// layouts of the single-call kernel, measured fastest there).
template <int NC> struct BatchCls;
template <> struct BatchCls<4> { static constexpr int TC = 1, RPT = 8; };
template <> struct BatchCls<8> { static constexpr int TC = 1, RPT = 8; };
template <> struct BatchCls<16> { static constexpr int TC = 4, RPT = 16; };
template <> struct BatchCls<32> { static constexpr int TC = 8, RPT = 16; };
template <> struct BatchCls<64> { static constexpr int TC = 16, RPT = 16; };
constexpr int kBatchT = 256;

static int class_of(int n) { return n <= 4 ? 4 : n <= 8 ? 8 : n <= 16 ? 16 : n <= 32 ? 32 : 64; }
template <int NC>
__host__ __device__ constexpr int rows_per_tile() {
  return (kBatchT / BatchCls<NC>::TC) * BatchCls<NC>::RPT;
}
static int rows_per_tile_rt(int nc) {
  switch (nc) {
    case 4: return rows_per_tile<4>();
    case 8: return rows_per_tile<8>();
    case 16: return rows_per_tile<16>();
    case 32: return rows_per_tile<32>();
    default: return rows_per_tile<64>();
  }
}

// Per-problem plan entry (device copy lives in the workspace).
struct BatchItem {
  const void* A;
  const void* b;
  int64_t m, lda;
  int n;       // columns factored (n + 1 for least squares)
  int nA;      // columns from A
  int nc;      // column class
  int dtype;
  int kind;    // 0 R, 1 lstsq
  int chunks;  // leaves
  int64_t tiles, tiles_per_chunk;
  int64_t work_begin;  // prefix of chunks over the ordered problems
  int64_t slot_off;    // in doubles
  int64_t cnt_off;     // in ints
  double* R;
  double* x;
  int32_t* info;
  int flag_idx;
  int method;  // QL_TSQR, or QL_CHOLQR2 (TSQR items of such problems run only when flagged)
};

constexpr int kMaxGramGroups = 6;  // column classes 16, 32, 64 x storage F64, F32
struct BatchHeader {
  int work_counter[2];  // [0] double-float launch, [1] gated FP64 launch
  int count;
  int pad;
  int64_t total_work;     // chunks of every problem (the gated FP64 launch)
  int64_t total_work_df;  // chunks of the TSQR problems, which come first
  int gram_counter[2 * kMaxGramGroups];  // per group and pass
};

template <int NC, typename S, typename Ar>
QL_DEV void batch_chunk(const BatchItem& it, int64_t chunk, unsigned char* smem, double* slots, int* counters,
                        int* flags) {
  constexpr int TC = BatchCls<NC>::TC, RPT = BatchCls<NC>::RPT, T = kBatchT;
  using Cta = TsqrCta<NC, TC, RPT, T, S, Ar>;
  Cta cta;
  cta.init(smem);
  cta.reset_r();
  if (threadIdx.x == 0) cta.misc[0] = 0;
  __syncthreads();
  TsqrProblem<S> p;
  p.src.A = static_cast<const S*>(it.A);
  p.src.lda = it.lda;
  p.src.b = static_cast<const S*>(it.b);
  p.src.nA = it.nA;
  p.m = it.m;
  p.n = it.n;
  p.vec16 = 0;
  const int64_t t0 = chunk * it.tiles_per_chunk;
  const int64_t t1 = min(it.tiles, t0 + it.tiles_per_chunk);
  cta.run(p, 0, t0, t1);
  const int n = it.n;
  if (threadIdx.x == 0 && cta.out_of_range(n, it.m)) {
    atomicOr(&flags[it.flag_idx], 1);
    atomicOr(&flags[-1], 1);  // any_flag lives just before the per-problem flags
  }
  TreeView tv;
  tv.slots = slots + it.slot_off;
  tv.counters = counters + it.cnt_off;
  tv.flags = flags + it.flag_idx;
  tv.leaves = it.chunks;
  double* slot = tv.slots + (size_t)chunk * n * n;
  for (int i = threadIdx.x; i < n * n; i += T) {
    int c = i / n, r = i % n;
    __stcg(slot + i, r <= c ? Ar::r_to_double(cta.R[r * NC + c]) : 0.0);
  }
  double* Ra = cta.arena;
  if (!climb_tree<NC, T>(tv, (int)chunk, n, cta.arena, cta.sd, &cta.misc[1], tree_arity<NC>())) return;
  __threadfence();
  if (Ar::kRangeChecked && *(volatile int*)&flags[it.flag_idx] != 0) return;
  // a Gram pass whose bounded wait gave up put the place into bits 8.. of the redo flag
  const int tmo = Ar::kRangeChecked ? 0 : (*(volatile int*)&flags[it.flag_idx] >> 8) & 0xff;
  if (it.kind == 0)
    epilogue_r<T>(Ra, NC, n, it.R, n, it.info, &cta.misc[2], tmo);
  else
    epilogue_lstsq<T>(Ra, NC, n, it.x, it.x + (n - 1), it.R, it.info, cta.sd, &cta.misc[2], tmo);
  __syncthreads();
}

template <typename S, typename Ar>
QL_DEV void batch_dispatch(const BatchItem& it, int64_t chunk, unsigned char* smem, double* slots, int* counters,
                           int* flags) {
  switch (it.nc) {
    case 4: batch_chunk<4, S, Ar>(it, chunk, smem, slots, counters, flags); break;
    case 8: batch_chunk<8, S, Ar>(it, chunk, smem, slots, counters, flags); break;
    case 16: batch_chunk<16, S, Ar>(it, chunk, smem, slots, counters, flags); break;
    case 32: batch_chunk<32, S, Ar>(it, chunk, smem, slots, counters, flags); break;
    default: batch_chunk<64, S, Ar>(it, chunk, smem, slots, counters, flags); break;
  }
}

template <typename Ar>
__global__ void __launch_bounds__(kBatchT, 1)
    batch_kernel(BatchHeader* hdr, const BatchItem* items, int count, double* slots, int* counters, int* flags,
                 int gated) {
  extern __shared__ __align__(16) unsigned char smem[];
  __shared__ int64_t s_work;
  __shared__ int s_item;
  if (gated && *(volatile int*)&flags[-1] == 0) return;  // no problem left the range
  const int64_t total = gated ? hdr->total_work : hdr->total_work_df;
  for (;;) {
    if (threadIdx.x == 0) {
      s_work = atomicAdd(&hdr->work_counter[gated ? 1 : 0], 1);
      // last problem whose work_begin <= s_work (items ordered by work_begin)
      int lo = 0, hi = count - 1;
      while (lo < hi) {
        int mid = (lo + hi + 1) >> 1;
        if (items[mid].work_begin <= s_work) lo = mid;
        else hi = mid - 1;
      }
      s_item = lo;
    }
    __syncthreads();
    const int64_t w = s_work;
    const int idx = s_item;
    __syncthreads();
    if (w >= total) break;
    const BatchItem it = items[idx];
    if (gated && *(volatile int*)&flags[it.flag_idx] == 0) continue;
    const int64_t chunk = w - it.work_begin;
    if (it.dtype == QL_F64)
      batch_dispatch<double, Ar>(it, chunk, smem, slots, counters, flags);
    else
      batch_dispatch<float, Ar>(it, chunk, smem, slots, counters, flags);
    __syncthreads();
  }
}

template <int NC, typename S, typename Ar>
static size_t cls_smem() {
  return TsqrSmem<NC, BatchCls<NC>::TC, BatchCls<NC>::RPT, kBatchT, S, Ar>::kBytes;
}
template <typename Ar>
static size_t batch_smem_bytes() {
  size_t b = 0;
  b = std::max({b, cls_smem<4, float, Ar>(), cls_smem<8, float, Ar>(), cls_smem<16, float, Ar>(),
                cls_smem<32, float, Ar>(), cls_smem<64, float, Ar>()});
  b = std::max({b, cls_smem<4, double, Ar>(), cls_smem<8, double, Ar>(), cls_smem<16, double, Ar>(),
                cls_smem<32, double, Ar>(), cls_smem<64, double, Ar>()});
  return b;
}

// ---------------------------------------------------------------------------------------
// Host plan
// ---------------------------------------------------------------------------------------

struct GramGroupPlan {
  int nc = 0, dtype = 0;
  std::vector<GramGroupItem> items;
  int64_t total = 0;
  size_t off_items = 0;
};

struct BatchPlan {
  std::vector<BatchItem> items;        // TSQR plan of every problem, TSQR problems first
  std::vector<int32_t> method;         // chosen method per problem, in the caller's order
  std::vector<GramGroupPlan> groups;   // Cholesky-QR2 problems by (column class, storage)
  size_t off_items = 0, off_flags = 0, off_counters = 0, off_gflags = 0, off_slots = 0, off_gram = 0,
         off_groups = 0, bytes = 0;
  int64_t total_work = 0, total_work_df = 0;
  size_t gram_flag_blocks = 0;  // Gram problems (512-byte flag block each, zeroed per launch)
};

// Tiles per chunk: aim for chunks of about kTargetRows rows (fewer, longer chunks for
// wide problems keep their FP64 tree merges cheap), overridable by the tuner.
static int64_t g_target_rows = 1 << 15;

static int gram_class_of(int ncols) { return ncols <= 8 ? 0 : ncols <= 16 ? 16 : ncols <= 32 ? 32 : 64; }

// The method of one problem (see the file comment).
static int choose_method(const ql_problem& pr, int ncols) {
  if (gram_class_of(ncols) == 0 || !tc_gram_enabled() || current_arith() == QL_ARITH_F64) return QL_TSQR;
  if (pr.method_hint == QL_CHOLQR2) return QL_CHOLQR2;
  if (pr.method_hint != QL_AUTO) return QL_TSQR;
  int m = QL_TSQR;
  if (tune_lookup(pr.m, ncols, pr.dtype, pr.kappa_hint > 0.0 ? pr.kappa_hint : 1e300, &m, nullptr))
    return m == QL_CHOLQR2 ? QL_CHOLQR2 : QL_TSQR;
  return (pr.kappa_hint > 0.0 && pr.kappa_hint <= 1e6 && ncols >= 24) ? QL_CHOLQR2 : QL_TSQR;
}

// Build the plan; with `ws` non-null the Gram items' device pointers point into it.
static bool make_plan(int32_t count, const ql_problem* probs, BatchPlan& P, unsigned char* ws = nullptr) {
  P = BatchPlan();
  P.method.assign(count, QL_TSQR);
  for (int i = 0; i < count; ++i) {
    const ql_problem& pr = probs[i];
    if (pr.m < 0 || pr.n < 1 || pr.n > 64 || (pr.kind == 1 && pr.n > 63)) return false;
    if (pr.ld < (pr.m > 1 ? pr.m : 1) || (pr.dtype != QL_F64 && pr.dtype != QL_F32)) return false;
    if (!pr.R || (pr.kind == 1 && (!pr.x || !pr.b)) || (pr.m > 0 && !pr.X)) return false;
    P.method[i] = choose_method(pr, (int)pr.n + (pr.kind == 1 ? 1 : 0));
  }
  std::vector<int> order(count);
  for (int i = 0; i < count; ++i) order[i] = i;
  auto work = [&](int i) { return (double)probs[i].m * probs[i].n * probs[i].n; };
  // TSQR problems first (the double-float TSQR launch covers a prefix of the work list),
  // each part by decreasing work
  std::stable_sort(order.begin(), order.end(), [&](int a, int b) {
    const bool ta = P.method[a] == QL_TSQR, tb = P.method[b] == QL_TSQR;
    if (ta != tb) return ta;
    return work(a) > work(b);
  });
  // chunk height: the batch's rows split into at least ~4 chunks per persistent CTA
  // (so a small batch still fills the GPU), between 2048 rows and g_target_rows
  int64_t total_rows = 0;
  for (int i = 0; i < count; ++i) total_rows += probs[i].m > 0 ? probs[i].m : 0;
  const int64_t ctas = (int64_t)device_sm_count();
  const int64_t target = std::max<int64_t>(2048, std::min<int64_t>(g_target_rows, total_rows / (4 * ctas)));
  int64_t slots = 0, cnts = 0, wb = 0;
  for (int k = 0; k < count; ++k) {
    const ql_problem& pr = probs[order[k]];
    BatchItem it{};
    it.A = pr.X;
    it.b = pr.kind == 1 ? pr.b : pr.X;
    it.m = pr.m;
    it.lda = pr.ld;
    it.nA = (int)pr.n;
    it.n = (int)pr.n + (pr.kind == 1 ? 1 : 0);
    it.nc = class_of(it.n);
    it.dtype = pr.dtype;
    it.kind = pr.kind;
    const int B = rows_per_tile_rt(it.nc);
    it.tiles = (pr.m + B - 1) / B;
    int64_t tpc = std::max<int64_t>(1, target / B);
    it.chunks = (int)std::max<int64_t>(1, (it.tiles + tpc - 1) / tpc);
    if (it.chunks > 4096) {  // keep trees shallow
      it.chunks = 4096;
      tpc = (it.tiles + 4095) / 4096;
    }
    it.tiles_per_chunk = tpc;
    it.work_begin = wb;
    wb += it.chunks;
    if (P.method[order[k]] == QL_TSQR) P.total_work_df = wb;
    it.slot_off = slots;
    slots += (int64_t)tree_slots(it.chunks) * it.n * it.n;
    it.cnt_off = cnts;
    cnts += (int64_t)tree_counters(it.chunks);
    it.R = pr.R;
    it.x = pr.x;
    it.info = pr.info;
    it.flag_idx = k;
    it.method = P.method[order[k]];
    P.items.push_back(it);
  }
  P.total_work = wb;
  size_t off = (sizeof(BatchHeader) + 255) / 256 * 256;
  P.off_items = off;
  off += (count * sizeof(BatchItem) + 255) / 256 * 256;
  P.off_flags = off;  // any_flag at [0], per-problem flags from [1]
  off += ((count + 1) * sizeof(int) + 255) / 256 * 256;
  P.off_counters = off;
  off += (cnts * sizeof(int) + 255) / 256 * 256;
  // Gram problems: flag blocks (cleared with the counters), then carried blocks, partials
  // and FP64 accumulator blocks, then the group item arrays
  P.off_gflags = off;
  std::vector<int> gram_probs;
  for (int k = 0; k < count; ++k)
    if (P.items[k].method == QL_CHOLQR2) gram_probs.push_back(k);
  P.gram_flag_blocks = gram_probs.size();
  off += gram_probs.size() * 512;
  P.off_slots = off;
  off += ((size_t)slots * sizeof(double) + 255) / 256 * 256;
  P.off_gram = off;
  int gidx[3][2];
  for (auto& r : gidx) r[0] = r[1] = -1;
  int fb = 0;
  for (int k : gram_probs) {
    const BatchItem& it = P.items[k];
    const int nc = gram_class_of(it.n), ci = nc == 16 ? 0 : (nc == 32 ? 1 : 2), di = it.dtype == QL_F64 ? 0 : 1;
    if (gidx[ci][di] < 0) {
      gidx[ci][di] = (int)P.groups.size();
      P.groups.emplace_back();
      P.groups.back().nc = nc;
      P.groups.back().dtype = it.dtype;
    }
    GramGroupPlan& G = P.groups[gidx[ci][di]];
    const int KT = gram_group_tile_rows(nc);
    const int64_t tiles = (it.m + KT - 1) / KT;
    const int64_t tpc = std::max<int64_t>(1, target / KT);
    const int nch = (int)std::max<int64_t>(1, std::min<int64_t>(4096, (tiles + tpc - 1) / tpc));
    GramGroupItem gi{};
    GramArgs<double>& a = gi.args;
    const size_t keep_b = ((size_t)3 * nc * nc * sizeof(double) + 255) / 256 * 256;
    const size_t part_b = (size_t)nch * nc * nc * sizeof(double);
    const size_t fbuf_b = (size_t)nch * nc * 128 * 2 * sizeof(double);  // accumulator levels of the tcgen05 kernels
    const size_t flags_off = P.off_gflags + (size_t)fb * 512, keep_off = off, part_off = off + keep_b,
                 fbuf_off = off + keep_b + part_b;
    off += keep_b + part_b + fbuf_b;
    ++fb;
    auto at = [&](size_t o) { return ws ? ws + o : nullptr; };
    a.src.A = static_cast<const double*>(it.A);
    a.src.lda = it.lda;
    a.src.b = static_cast<const double*>(it.b);
    a.src.nA = it.nA;
    a.m = it.m;
    a.n = it.n;
    a.tiles = tiles;
    a.pass = 1;
    a.method = QL_CHOLQR2;
    a.gated = 0;
    a.epilogue = it.kind == 1 ? kEpiLstsq : kEpiR;
    a.w.flags = reinterpret_cast<int*>(at(flags_off));
    a.w.keep = reinterpret_cast<double*>(at(keep_off));
    a.w.partials = reinterpret_cast<double*>(at(part_off));
    a.w.fbuf = reinterpret_cast<double*>(at(fbuf_off));
    if (it.kind == 1) {  // R_ext into R (ld n + 1), x and the residual norm into x
      a.x = it.x;
      a.resnorm = it.x + (it.n - 1);
      a.Rext = it.R;
    } else {
      a.R = it.R;
      a.ldr = it.n;
    }
    a.info = it.info;
    {
      auto al16 = [](const void* q) { return (reinterpret_cast<uintptr_t>(q) & 15u) == 0; };
      const size_t es = it.dtype == QL_F64 ? 8 : 4;
      bool b = al16(it.A) && ((size_t)it.lda * es) % 16 == 0;
      if (it.kind == 1) b = b && al16(it.b);
      a.bulk = b ? 1 : 0;
    }
    gi.tma = pipe_tensor_maps(&gi.tmA, it.kind == 1 ? &gi.tmB : nullptr, it.A, it.b, it.dtype, it.m, it.nA, it.lda)
                 ? 1
                 : 0;
    a.mround = 2;
    a.redo = reinterpret_cast<int*>(at(P.off_flags)) + 1 + k;
    a.redo_any = reinterpret_cast<int*>(at(P.off_flags));
    a.redo_on_breakdown = probs[order[k]].method_hint == QL_AUTO ? 1 : 0;
    gi.work_begin = G.total;
    gi.nchunks = nch;
    G.total += nch;
    G.items.push_back(gi);
  }
  P.off_groups = off = (off + 255) / 256 * 256;
  for (auto& G : P.groups) {
    G.off_items = off;
    off += (G.items.size() * sizeof(GramGroupItem) + 255) / 256 * 256;
  }
  P.bytes = off;
  return true;
}

template <typename Ar>
static ql_status launch_batch(unsigned char* ws, const BatchPlan& P, int count, cudaStream_t stream, int gated) {
  static int occ = 0;
  static size_t smem = 0;
  static std::mutex mu;
  auto kern = batch_kernel<Ar>;
  {
    std::lock_guard<std::mutex> lk(mu);
    if (occ == 0) {
      smem = batch_smem_bytes<Ar>();
      if (cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem) != cudaSuccess)
        return QL_ERR_CUDA;
      int o = 0;
      if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&o, kern, kBatchT, smem) != cudaSuccess) return QL_ERR_CUDA;
      occ = o < 1 ? 1 : o;
    }
  }
  int grid = device_sm_count() * occ;
  if (P.total_work < grid) grid = (int)std::max<int64_t>(1, P.total_work);
  count_launch();
  kern<<<grid, kBatchT, smem, stream>>>(reinterpret_cast<BatchHeader*>(ws),
                                         reinterpret_cast<const BatchItem*>(ws + P.off_items), count,
                                         reinterpret_cast<double*>(ws + P.off_slots),
                                         reinterpret_cast<int*>(ws + P.off_counters),
                                         reinterpret_cast<int*>(ws + P.off_flags) + 1, gated);
  return cudaPeekAtLastError() == cudaSuccess ? QL_OK : QL_ERR_CUDA;
}

// The plan of the last ql_batch_prepare per workspace pointer (for ql_batch_launch).
struct PlanCache {
  std::mutex mu;
  std::vector<std::pair<void*, BatchPlan>> plans;
  void put(void* ws, const BatchPlan& p) {
    std::lock_guard<std::mutex> lk(mu);
    for (auto& e : plans)
      if (e.first == ws) {
        e.second = p;
        return;
      }
    plans.emplace_back(ws, p);
  }
  bool get(void* ws, BatchPlan& p) {
    std::lock_guard<std::mutex> lk(mu);
    for (auto& e : plans)
      if (e.first == ws) {
        p = e.second;
        return true;
      }
    return false;
  }
};
static PlanCache g_plans;

void set_batch_target_rows(int64_t rows) { g_target_rows = rows < 256 ? 256 : rows; }
int64_t batch_target_rows() { return g_target_rows; }

// The host image of what the device needs of a plan: [header, TSQR items] (uploaded to
// offset 0) followed by the Gram group item arrays (uploaded to off_groups).
static size_t upload_bytes(const BatchPlan& P) { return P.off_flags + (P.bytes - P.off_groups); }
static void fill_upload(const BatchPlan& P, int32_t count, unsigned char* dst) {
  BatchHeader h{};
  h.count = count;
  h.total_work = P.total_work;
  h.total_work_df = P.total_work_df;
  std::memset(dst, 0, upload_bytes(P));
  std::memcpy(dst, &h, sizeof(h));
  std::memcpy(dst + P.off_items, P.items.data(), P.items.size() * sizeof(BatchItem));
  for (const auto& G : P.groups)
    std::memcpy(dst + P.off_flags + (G.off_items - P.off_groups), G.items.data(), G.items.size() * sizeof(GramGroupItem));
}

// Asynchronous plan upload through a caller-owned pinned staging buffer (the serving
// loop's path: no host synchronisation).  The staging bytes must stay untouched until the
// stream has passed the copy.
ql_status batch_prepare_async(int32_t count, const ql_problem* probs, void* ws, size_t ws_bytes, cudaStream_t st,
                              unsigned char* pinned, size_t pinned_bytes) {
  if (count < 1 || !probs) return QL_ERR_ARG;
  BatchPlan P;
  if (!make_plan(count, probs, P, static_cast<unsigned char*>(ws))) return QL_ERR_ARG;
  if (!ws || ws_bytes < P.bytes) return QL_ERR_WORKSPACE;
  if (!pinned || pinned_bytes < upload_bytes(P)) return QL_ERR_WORKSPACE;
  fill_upload(P, count, pinned);
  unsigned char* w = static_cast<unsigned char*>(ws);
  if (cudaMemcpyAsync(w, pinned, P.off_flags, cudaMemcpyHostToDevice, st) != cudaSuccess) return QL_ERR_CUDA;
  if (P.bytes > P.off_groups &&
      cudaMemcpyAsync(w + P.off_groups, pinned + P.off_flags, P.bytes - P.off_groups, cudaMemcpyHostToDevice, st) !=
          cudaSuccess)
    return QL_ERR_CUDA;
  g_plans.put(ws, P);
  return QL_OK;
}

size_t batch_plan_upload_bytes(int32_t count, const ql_problem* probs) {
  BatchPlan P;
  if (count < 1 || !probs || !make_plan(count, probs, P)) return 0;
  return upload_bytes(P);
}

}  // namespace ql

using namespace ql;

extern "C" {

size_t ql_batch_workspace_bytes(int32_t count, const ql_problem* probs) {
  if (count < 1 || !probs) return 0;
  BatchPlan P;
  if (!make_plan(count, probs, P)) return 0;
  return P.bytes;
}

ql_status ql_batch_prepare(int32_t count, const ql_problem* probs, void* ws, size_t ws_bytes, void* stream) {
  if (count < 1 || !probs) return QL_ERR_ARG;
  BatchPlan P;
  if (!make_plan(count, probs, P, static_cast<unsigned char*>(ws))) return QL_ERR_ARG;
  if (!ws || ws_bytes < P.bytes) return QL_ERR_WORKSPACE;
  cudaStream_t st = (cudaStream_t)stream;
  unsigned char* w = static_cast<unsigned char*>(ws);
  std::vector<unsigned char> img(upload_bytes(P));
  fill_upload(P, count, img.data());
  if (cudaMemcpyAsync(w, img.data(), P.off_flags, cudaMemcpyHostToDevice, st) != cudaSuccess) return QL_ERR_CUDA;
  if (P.bytes > P.off_groups && cudaMemcpyAsync(w + P.off_groups, img.data() + P.off_flags, P.bytes - P.off_groups,
                                                cudaMemcpyHostToDevice, st) != cudaSuccess)
    return QL_ERR_CUDA;
  if (cudaStreamSynchronize(st) != cudaSuccess) return QL_ERR_CUDA;  // img is freed on return
  g_plans.put(ws, P);
  return QL_OK;
}

ql_status ql_batch_launch(void* ws, void* stream) {
  BatchPlan P;
  if (!ws || !g_plans.get(ws, P)) return QL_ERR_ARG;
  cudaStream_t st = (cudaStream_t)stream;
  unsigned char* w = static_cast<unsigned char*>(ws);
  const int count = (int)P.items.size();
  // work counters, tree counters and every flag (TSQR and Gram) start at zero on every launch
  if (cudaMemsetAsync(w, 0, offsetof(BatchHeader, count), st) != cudaSuccess) return QL_ERR_CUDA;
  if (cudaMemsetAsync(w + offsetof(BatchHeader, gram_counter), 0, sizeof(int) * 2 * kMaxGramGroups, st) !=
      cudaSuccess)
    return QL_ERR_CUDA;
  if (cudaMemsetAsync(w + P.off_flags, 0, P.off_slots - P.off_flags, st) != cudaSuccess) return QL_ERR_CUDA;
  BatchHeader* hdr = reinterpret_cast<BatchHeader*>(w);
  const bool f64 = current_arith() == QL_ARITH_F64;  // then every problem runs TSQR (the plan chose so)
  ql_status s = QL_OK;
  auto gram_pass = [&](int pass) {
    for (size_t g = 0; g < P.groups.size() && s == QL_OK; ++g) {
      const GramGroupPlan& G = P.groups[g];
      s = gram_group_launch(G.nc, G.dtype, pass, &hdr->gram_counter[2 * g + pass - 1],
                            reinterpret_cast<const GramGroupItem*>(w + G.off_items), (int)G.items.size(), G.total, st);
    }
  };
  gram_pass(1);
  if (s == QL_OK) s = f64 ? launch_batch<ArithF64>(w, P, count, st, 0) : launch_batch<ArithDF>(w, P, count, st, 0);
  if (s == QL_OK) gram_pass(2);
  if (s != QL_OK || f64) return s;
  return launch_batch<ArithF64>(w, P, count, st, 1);  // flagged problems, any method
}

ql_status ql_batch_methods(void* ws, int32_t* methods, int32_t count) {
  BatchPlan P;
  if (!ws || !methods || !g_plans.get(ws, P)) return QL_ERR_ARG;
  if (count != (int32_t)P.method.size()) return QL_ERR_ARG;
  std::memcpy(methods, P.method.data(), sizeof(int32_t) * count);
  return QL_OK;
}

ql_status ql_batch_qless(int32_t count, const ql_problem* probs, void* ws, size_t ws_bytes, void* stream) {
  ql_status s = ql_batch_prepare(count, probs, ws, ws_bytes, stream);
  if (s != QL_OK) return s;
  return ql_batch_launch(ws, stream);
}

}  // extern "C"
