// TSQR kernel entry and its launch templates; instantiated per (storage, arithmetic) in
// the tsqr_inst_*.cu translation units so that the build compiles them in parallel.
#pragma once

#include <mutex>

#include "epilogue.cuh"
#include "internal.h"
#include "tsqr.cuh"

namespace ql {

// Most CTAs per SM any TSQR configuration runs with (sizes the R-tree workspace).
constexpr int kMaxCtasPerSm = 4;

template <typename S>
struct TsqrArgs {
  TsqrProblem<S> p;
  TreeView tv;
  int64_t tiles;
  int gated;  // FP64 fallback launch: run only if the range flag is set
  int arity;  // R-tree arity (2 .. the column class's default)
  int epilogue;
  double* R;
  int64_t ldr;
  double* x;
  double* resnorm;
  double* Rext;
  int32_t* info;
};

template <int NC, int TC, int RPT, int T, typename S, typename Ar>
__global__ void __launch_bounds__(T, 1) tsqr_kernel(TsqrArgs<S> a) {
  extern __shared__ __align__(16) unsigned char smem[];
  using Cta = TsqrCta<NC, TC, RPT, T, S, Ar>;
  if (a.gated) {
    if (*(volatile int*)&a.tv.flags[0] == 0) return;
  }
  Cta cta;
  cta.init(smem);
  cta.reset_r();
  if (threadIdx.x == 0) cta.misc[0] = 0;
  __syncthreads();

  const int k = gridDim.x, bid = blockIdx.x;
  int64_t t0 = a.tiles * bid / k, t1 = a.tiles * (bid + 1) / k;
  cta.run(a.p, 0, t0, t1);

  const int n = a.p.n;
  if (threadIdx.x == 0 && cta.out_of_range(n, a.p.m)) atomicOr(&a.tv.flags[0], 1);
  // leaf triangle -> slot(0, bid), FP64 (hi + lo of a double-float is exact in a double)
  double* slot = a.tv.slots + (size_t)bid * n * n;
  for (int i = threadIdx.x; i < n * n; i += T) {
    int c = i / n, r = i % n;
    __stcg(slot + i, r <= c ? Ar::r_to_double(cta.R[r * NC + c]) : 0.0);
  }
  double* Ra = cta.arena;
  if (!climb_tree<NC, T>(a.tv, bid, n, cta.arena, cta.sd, &cta.misc[1], a.arity)) return;

  // root: every CTA has passed its range check and its tree arrival by now
  __threadfence();
  if (Ar::kRangeChecked && *(volatile int*)&a.tv.flags[0] != 0) return;  // FP64 launch redoes it
  if (a.epilogue == kEpiR)
    epilogue_r<T>(Ra, NC, n, a.R, a.ldr, a.info, &cta.misc[2]);
  else
    epilogue_lstsq<T>(Ra, NC, n, a.x, a.resnorm, a.Rext, a.info, cta.sd, &cta.misc[2]);
}

template <int NC, int TC, int RPT, int T, typename S, typename Ar>
ql_status launch_one(const TsqrCall& c, const TreeView& tv_in, int gated) {
  using Sm = TsqrSmem<NC, TC, RPT, T, S, Ar>;
  using Sh = TsqrShape<NC, TC, RPT, T>;
  auto kern = tsqr_kernel<NC, TC, RPT, T, S, Ar>;
  static int occ = 0;  // CTAs per SM at this configuration's registers and shared memory
  static std::mutex mu;
  {
    std::lock_guard<std::mutex> lk(mu);
    if (occ == 0) {
      if (cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)Sm::kBytes) != cudaSuccess)
        return QL_ERR_CUDA;
      int o = 0;
      if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&o, kern, T, Sm::kBytes) != cudaSuccess) return QL_ERR_CUDA;
      occ = o < 1 ? 1 : (o > kMaxCtasPerSm ? kMaxCtasPerSm : o);
    }
  }
  const int64_t tiles = (c.m + Sh::B - 1) / Sh::B;
  int64_t g = (int64_t)device_sm_count() * (c.ctas_per_sm > 0 ? (c.ctas_per_sm < occ ? c.ctas_per_sm : occ) : occ);
  if (c.max_ctas > 0 && g > c.max_ctas) g = c.max_ctas;
  if (g > tiles) g = tiles;
  if (g < 1) g = 1;
  TsqrArgs<S> a;
  a.p.src.A = static_cast<const S*>(c.A);
  a.p.src.lda = c.lda;
  a.p.src.b = static_cast<const S*>(c.b);
  a.p.src.nA = c.nA;
  a.p.m = c.m;
  a.p.n = c.n;
  {
    auto al16 = [](const void* q) { return (reinterpret_cast<uintptr_t>(q) & 15u) == 0; };
    bool v = al16(c.A) && ((size_t)c.lda * sizeof(S)) % 16 == 0;
    if (c.nA < c.n) v = v && al16(c.b);
    a.p.vec16 = v ? 1 : 0;
  }
  a.tv = tv_in;
  a.tv.leaves = (int)g;
  a.tiles = tiles;
  a.gated = gated;
  a.arity = (c.arity >= 2 && c.arity < tree_arity<NC>()) ? c.arity : tree_arity<NC>();
  a.epilogue = c.epilogue;
  a.R = c.R;
  a.ldr = c.ldr;
  a.x = c.x;
  a.resnorm = c.resnorm;
  a.Rext = c.Rext;
  a.info = c.info;
  count_launch();
  kern<<<(int)g, T, Sm::kBytes, c.stream>>>(a);
  return cudaPeekAtLastError() == cudaSuccess ? QL_OK : QL_ERR_CUDA;
}

// Configuration table: NC (padded column count), TC column groups, RPT rows per thread,
// T threads.  A thread holds RPT x NC/TC elements of the tile: 64 for n <= 8 (32 at n = 1)
// and for n > 8, where 256-thread CTAs with 16 rows per thread measured fastest (m = 2^25:
// n = 64 139.6 ms against 146.1 with 8 rows per thread and 216.2 with 512-thread CTAs;
// n = 32 35.4 against 37.0; n = 16 9.46 against 9.75): a column reduction across the row
// threads then serves twice the rows.  512-thread CTAs with the same 16 rows per thread and
// half the columns measured slower again (n = 64 154.4 ms, n = 32 60.1 or 40.1, n = 16 15.5).
template <typename S, typename Ar>
ql_status dispatch(const TsqrCall& c, const TreeView& tv, int gated) {
  const int n = c.n;
  if constexpr (std::is_same<S, double>::value && std::is_same<Ar, ArithDF>::value) {
    const int v = c.variant >= 0 ? c.variant : tsqr_variant();  // alternative thread layouts (tuner)
    if (v > 0 && n > 8) {
      if (n <= 16) {
        if (v == 1) return launch_one<16, 4, 8, 256, S, Ar>(c, tv, gated);
        if (v == 2) return launch_one<16, 2, 8, 128, S, Ar>(c, tv, gated);
      } else if (n <= 32) {
        if (v == 1) return launch_one<32, 8, 8, 256, S, Ar>(c, tv, gated);
        if (v == 2) return launch_one<32, 4, 8, 128, S, Ar>(c, tv, gated);
      } else {
        if (v == 1) return launch_one<64, 16, 8, 256, S, Ar>(c, tv, gated);
        if (v == 2) return launch_one<64, 8, 8, 128, S, Ar>(c, tv, gated);
      }
    }
  }
  if (n <= 1) return launch_one<1, 1, 16, 128, S, Ar>(c, tv, gated);
  if (n <= 2) return launch_one<2, 1, 16, 128, S, Ar>(c, tv, gated);
  if (n <= 4) return launch_one<4, 1, 8, 128, S, Ar>(c, tv, gated);
  if (n <= 8) return launch_one<8, 1, 8, 128, S, Ar>(c, tv, gated);
  if (n <= 16) return launch_one<16, 4, 16, 256, S, Ar>(c, tv, gated);
  if (n <= 32) return launch_one<32, 8, 16, 256, S, Ar>(c, tv, gated);
  return launch_one<64, 16, 16, 256, S, Ar>(c, tv, gated);
}


extern template ql_status dispatch<double, ArithDF>(const TsqrCall&, const TreeView&, int);
extern template ql_status dispatch<double, ArithF64>(const TsqrCall&, const TreeView&, int);
extern template ql_status dispatch<float, ArithDF>(const TsqrCall&, const TreeView&, int);
extern template ql_status dispatch<float, ArithF64>(const TsqrCall&, const TreeView&, int);

}  // namespace ql
