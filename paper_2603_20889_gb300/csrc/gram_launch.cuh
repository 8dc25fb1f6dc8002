// Gram-pass kernel of CholQR2 / SVQB2 and its launch template (paper Sec. 3.1).
// Instantiated per (storage, arithmetic) in gram_inst_*.cu.
#pragma once

#include <mutex>

#include "epilogue.cuh"
#include "gram.cuh"
#include "internal.h"
#include "small_dense.cuh"

namespace ql {

constexpr int kGramMaxCtasPerSm = 4;

struct GramWs {
  int* flags;        // [0] range, [1] first-pass breakdown, [2] arrival counter pass 1, [3] pass 2
  double* keep;      // 3 n x n blocks carried from pass 1 to pass 2 (row-major, ld n)
  double* partials;  // one NC x NC partial Gram per CTA
};

template <typename S>
struct GramArgs {
  ColSource<S> src;
  int64_t m;
  int n;
  int64_t tiles;
  int pass;    // 1 or 2
  int method;  // QL_CHOLQR2 or QL_SVQB2
  int gated;
  int epilogue;
  GramWs w;
  double* R;
  int64_t ldr;
  double* Z;
  double rank_tol;
  double* x;
  double* resnorm;
  double* Rext;
  int32_t* info;
};

QL_DEV double qnan() { return __longlong_as_double(0x7ff8000000000000ll); }

// Fill the outputs of a failed factorisation with NaN (R, or x and resnorm).
template <typename S>
QL_DEV void write_nan_outputs(const GramArgs<S>& a, int T) {
  if (a.epilogue == kEpiR) {
    for (int i = threadIdx.x; i < a.n * a.n; i += T) a.R[(int64_t)(i / a.n) * a.ldr + i % a.n] = qnan();
  } else {
    for (int i = threadIdx.x; i < a.n - 1; i += T) a.x[i] = qnan();
    if (threadIdx.x == 0) *a.resnorm = qnan();
  }
}

template <int NC, typename S, typename Ar, int XF>
__global__ void __launch_bounds__(GramShape<NC>::T, 1) gram_kernel(GramArgs<S> a) {
  using Sh = GramShape<NC>;
  using Sm = GramSmem<NC, S, Ar>;
  using V = typename Ar::T;
  using Acc = typename Ar::Acc;
  constexpr int T = Sh::T, B = Sh::B, BS = Sh::BS, NBT = Sh::NBT, SL = Sh::SL;
  extern __shared__ __align__(16) unsigned char smem[];
  const int tid = threadIdx.x, n = a.n;

  if (a.gated && *(volatile int*)&a.w.flags[0] == 0) return;
  if (Ar::kRangeChecked && a.pass == 2 && *(volatile int*)&a.w.flags[0] != 0) return;  // FP64 redoes it
  if (a.pass == 2 && *(volatile int*)&a.w.flags[1] != 0) {  // first pass broke down
    if (blockIdx.x == 0) write_nan_outputs(a, T);
    return;
  }

  S* stage = reinterpret_cast<S*>(smem);
  V* Y0 = reinterpret_cast<V*>(smem + Sm::kOffY);
  V* Y1 = Y0 + NC * B;
  V* Mv = reinterpret_cast<V*>(smem + Sm::kOffM);
  int* misc = reinterpret_cast<int*>(smem + Sm::kOffMisc);
  int* colmax = misc + 64;

  for (int i = tid; i < NC; i += T) colmax[i] = 0;
  if constexpr (XF != kXNone) {
    const double* M = a.w.keep + (size_t)n * n;  // pass-1 output: R1^{-1} or B1 (row-major, ld n)
    for (int i = tid; i < NC * NC; i += T) {
      int r = i / NC, c = i % NC;
      Mv[i] = (r < n && c < n) ? Ar::from_double(__ldcg(M + r * n + c)) : Ar::zero();
    }
  }

  // (bp, bq): this thread's block of the upper triangle of C, and its row slice
  const int blk = tid / SL, slice = tid % SL;
  const bool active = blk < NBT;
  int bp = 0, bq = 0;
  {
    int rem = active ? blk : 0;
    while (rem >= Sh::NB - bp) {
      rem -= Sh::NB - bp;
      ++bp;
    }
    bq = bp + rem;
  }
  const int p0 = bp * BS, q0 = bq * BS;
  const bool useful = active && p0 < n && q0 < n;

  Acc acc[BS][BS];
#pragma unroll
  for (int i = 0; i < BS; ++i)
#pragma unroll
    for (int j = 0; j < BS; ++j) acc[i][j] = Ar::acc_zero();

  const int k = gridDim.x, bid = blockIdx.x;
  const int64_t t0 = a.tiles * bid / k, t1 = a.tiles * (bid + 1) / k;

  auto issue = [&](int64_t t) {
    const int64_t row0 = t * B;
#pragma unroll 1
    for (int c = 0; c < NC; ++c) {
      const S* col = a.src.col(c < n ? c : 0);
      for (int r = tid; r < B; r += T) {
        int64_t row = row0 + r;
        bool v = c < n && row < a.m;
        cp_async_elem<S>(stage + c * B + r, v ? col + row : col, v);
      }
    }
    cp_async_commit();
  };

  if (t0 < t1) issue(t0);
  __syncthreads();
  for (int64_t t = t0; t < t1; ++t) {
    cp_async_wait_all();
    __syncthreads();
    // convert the staged tile once (and record column exponent maxima); a warp covers 32
    // consecutive rows of one column per chunk (B is a multiple of 32)
    for (int chunk = tid >> 5; chunk < NC * B / 32; chunk += T / 32) {
      const int i = chunk * 32 + (tid & 31);
      int E;
      Y0[i] = Ar::load(stage[i], E);
      if constexpr (Ar::kRangeChecked) {
        unsigned em = __reduce_max_sync(0xffffffffu, (unsigned)E);
        if ((tid & 31) == 0 && em > 0) atomicMax(&colmax[i / B], (int)em);
      }
    }
    __syncthreads();
    if (t + 1 < t1) issue(t + 1);
    const V* Y = Y0;
    if constexpr (XF != kXNone) {
      for (int i = tid; i < NC * B; i += T) {
        int c = i / B, r = i % B;
        Acc s = Ar::acc_zero();
        if (c < n) {
          const int kend = XF == kXUpper ? c + 1 : n;
          for (int kk = 0; kk < kend; ++kk) Ar::acc_fma(s, Y0[kk * B + r], Mv[kk * NC + c]);
        }
        Y1[i] = Ar::acc_get(s);
      }
      __syncthreads();
      Y = Y1;
    }
    if (useful) {
#pragma unroll 2
      for (int r = slice; r < B; r += SL) {
        V yp[BS], yq[BS];
#pragma unroll
        for (int i = 0; i < BS; ++i) {
          yp[i] = Y[(p0 + i) * B + r];
          yq[i] = Y[(q0 + i) * B + r];
        }
#pragma unroll
        for (int i = 0; i < BS; ++i)
#pragma unroll
          for (int j = 0; j < BS; ++j) Ar::acc_fma(acc[i][j], yp[i], yq[j]);
      }
    }
  }
  __syncthreads();

  // reduce the row slices: red[(slice * NBT + blk) * BS * BS + i * BS + j]
  V* red = Y0;
  if (active) {
#pragma unroll
    for (int i = 0; i < BS; ++i)
#pragma unroll
      for (int j = 0; j < BS; ++j) red[(slice * NBT + blk) * BS * BS + i * BS + j] = Ar::acc_get(acc[i][j]);
  }
  __syncthreads();
  double* part = a.w.partials + (size_t)bid * NC * NC;
  for (int e = tid; e < NBT * BS * BS; e += T) {
    int b = e / (BS * BS), ij = e % (BS * BS);
    V s = red[b * BS * BS + ij];
    for (int sl = 1; sl < SL; ++sl) s = Ar::add(s, red[(sl * NBT + b) * BS * BS + ij]);
    int rem = b, pp = 0;
    while (rem >= Sh::NB - pp) {
      rem -= Sh::NB - pp;
      ++pp;
    }
    int qq = pp + rem;
    int p = pp * BS + ij / BS, q = qq * BS + ij % BS;
    __stcg(part + p * NC + q, Ar::to_double(s));
  }
  if (tid == 0) {
    bool bad = false;
    if constexpr (Ar::kRangeChecked) {
      for (int c = 0; c < n; ++c) {
        int e = colmax[c];
        if (e != 0 && (e < kDfEminLimit || e > kDfEmaxLimit)) bad = true;
      }
    }
    if (bad) atomicOr(&a.w.flags[0], 1);
  }
  // last CTA done
  __threadfence();
  __syncthreads();
  int* counter = &a.w.flags[a.pass == 1 ? 2 : 3];
  if (tid == 0) {
    int old = atomicAdd(counter, 1);
    misc[0] = (old == k - 1);
    if (old == k - 1) *counter = 0;
  }
  __syncthreads();
  if (!misc[0]) return;
  __threadfence();
  if (Ar::kRangeChecked && *(volatile int*)&a.w.flags[0] != 0) return;  // the FP64 launches redo it

  // ---------------- epilogue: one CTA, FP64, shared memory reused from here on
  double* Cs = reinterpret_cast<double*>(smem);  // n x n, ld NC
  double* Us = Cs + NC * NC;
  double* Ps = Us + NC * NC;
  double* Qs = Ps + NC * NC;
  double* vec = Qs + NC * NC;  // 8 NC
  int* sflag = reinterpret_cast<int*>(vec + 8 * NC);
  __syncthreads();
  for (int e = tid; e < n * n; e += T) {
    int p = e / n, q = e % n;
    if (p > q) continue;
    V s = Ar::zero();
    for (int b = 0; b < k; ++b) {
      int E;
      s = Ar::add(s, Ar::load(__ldcg(a.w.partials + (size_t)b * NC * NC + p * NC + q), E));
    }
    double v = Ar::to_double(s);
    Cs[p * NC + q] = v;
    Cs[q * NC + p] = v;
  }
  __syncthreads();
  double* keep = a.w.keep;  // [0]: R1 or S1, [1]: M (R1^{-1} or B1)
  const int nn = n * n;
  if (a.method == QL_CHOLQR2) {
    int fail = chol_upper_inplace<T>(Cs, NC, n, sflag);
    if (fail) {
      if (a.pass == 1) a.w.flags[1] = 1;
      write_nan_outputs(a, T);
      write_info(a.info, QL_ERR_NOT_SPD, fail + (a.pass == 2 ? 1000 : 0));
      return;
    }
    if (a.pass == 1) {
      tri_upper_inverse<T>(Cs, NC, Us, NC, n);
      for (int e = tid; e < nn; e += T) {
        keep[e] = Cs[(e / n) * NC + e % n];
        keep[nn + e] = Us[(e / n) * NC + e % n];
      }
      return;
    }
    // pass 2: R = R2 R1
    for (int e = tid; e < nn; e += T) Us[(e / n) * NC + e % n] = __ldcg(keep + e);
    __syncthreads();
    upper_times_upper<T>(Cs, NC, Us, NC, Ps, NC, n);
  } else {
    jacobi_eig<T>(Cs, NC, Us, NC, n, vec, sflag);
    // lambda_max and the truncation threshold
    double lmax = 0.0;
    for (int i = 0; i < n; ++i) lmax = fmax(lmax, Cs[i * NC + i]);
    double tol = a.rank_tol > 0.0 ? a.rank_tol : (double)n * 2.220446049250313e-16;
    double cut = tol * lmax;
    if (a.pass == 1) {
      for (int e = tid; e < nn; e += T) {
        int r = e / n, i = e % n;  // B1(r, i) = U(r, i) lambda_i^{-1/2};  S1(i, r) = lambda_i^{1/2} U(r, i)
        double li = Cs[i * NC + i];
        bool keepit = li > cut && li > 0.0;
        double sq = keepit ? sqrt(li) : 0.0;
        keep[nn + r * n + i] = keepit ? Us[r * NC + i] / sq : 0.0;
        keep[i * n + r] = sq * Us[r * NC + i];
      }
      return;
    }
    // pass 2: Z = S2 S1 with S2(i, r) = lambda2_i^{1/2} U2(r, i);  R = qr_r(Z)
    for (int e = tid; e < nn; e += T) {
      int i = e / n, r = e % n;
      double li = Cs[i * NC + i];
      bool keepit = li > cut && li > 0.0;
      Qs[i * NC + r] = (keepit ? sqrt(li) : 0.0) * Us[r * NC + i];
    }
    __syncthreads();
    for (int e = tid; e < nn; e += T) Us[(e / n) * NC + e % n] = __ldcg(keep + e);  // S1
    __syncthreads();
    full_times_full<T>(Qs, NC, Us, NC, Ps, NC, n);
    if (a.Z && a.epilogue == kEpiR)
      for (int e = tid; e < nn; e += T) a.Z[(e / n) * n + e % n] = Ps[(e % n) * NC + e / n];  // column-major
    __syncthreads();
    householder_square<T>(Ps, NC, n, vec);
  }
  if (a.epilogue == kEpiR)
    epilogue_r<T>(Ps, NC, n, a.R, a.ldr, a.info, sflag);
  else
    epilogue_lstsq<T>(Ps, NC, n, a.x, a.resnorm, a.Rext, a.info, vec, sflag);
}

template <int NC, typename S, typename Ar, int XF>
ql_status gram_launch_one(const GramCall& c, const GramWs& w, int pass, int gated) {
  using Sh = GramShape<NC>;
  using Sm = GramSmem<NC, S, Ar>;
  auto kern = gram_kernel<NC, S, Ar, XF>;
  static int occ = 0;
  static std::mutex mu;
  {
    std::lock_guard<std::mutex> lk(mu);
    if (occ == 0) {
      if (cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)Sm::kBytes) != cudaSuccess)
        return QL_ERR_CUDA;
      int o = 0;
      if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&o, kern, Sh::T, Sm::kBytes) != cudaSuccess)
        return QL_ERR_CUDA;
      occ = o < 1 ? 1 : (o > kGramMaxCtasPerSm ? kGramMaxCtasPerSm : o);
    }
  }
  const int64_t tiles = (c.m + Sh::B - 1) / Sh::B;
  int64_t g = (int64_t)device_sm_count() * occ;
  if (g > tiles) g = tiles;
  if (g < 1) g = 1;
  GramArgs<S> a;
  a.src.A = static_cast<const S*>(c.A);
  a.src.lda = c.lda;
  a.src.b = static_cast<const S*>(c.b);
  a.src.nA = c.nA;
  a.m = c.m;
  a.n = c.n;
  a.tiles = tiles;
  a.pass = pass;
  a.method = c.method;
  a.gated = gated;
  a.epilogue = c.epilogue;
  a.w = w;
  a.R = c.R;
  a.ldr = c.ldr;
  a.Z = c.Z;
  a.rank_tol = c.rank_tol;
  a.x = c.x;
  a.resnorm = c.resnorm;
  a.Rext = c.Rext;
  a.info = c.info;
  count_launch();
  kern<<<(int)g, Sh::T, Sm::kBytes, c.stream>>>(a);
  return cudaPeekAtLastError() == cudaSuccess ? QL_OK : QL_ERR_CUDA;
}

// Both passes of one method for one (storage, arithmetic) pair.
template <typename S, typename Ar>
ql_status gram_dispatch(const GramCall& c, const GramWs& w, int gated) {
  auto two = [&](auto nc_tag) -> ql_status {
    constexpr int NC = decltype(nc_tag)::value;
    ql_status st = gram_launch_one<NC, S, Ar, kXNone>(c, w, 1, gated);
    if (st) return st;
    if (c.method == QL_CHOLQR2) return gram_launch_one<NC, S, Ar, kXUpper>(c, w, 2, gated);
    return gram_launch_one<NC, S, Ar, kXFull>(c, w, 2, gated);
  };
  const int n = c.n;
  if (n <= 1) return two(std::integral_constant<int, 1>{});
  if (n <= 2) return two(std::integral_constant<int, 2>{});
  if (n <= 4) return two(std::integral_constant<int, 4>{});
  if (n <= 8) return two(std::integral_constant<int, 8>{});
  if (n <= 16) return two(std::integral_constant<int, 16>{});
  if (n <= 32) return two(std::integral_constant<int, 32>{});
  return two(std::integral_constant<int, 64>{});
}

extern template ql_status gram_dispatch<double, ArithDF>(const GramCall&, const GramWs&, int);
extern template ql_status gram_dispatch<double, ArithF64>(const GramCall&, const GramWs&, int);
extern template ql_status gram_dispatch<float, ArithDF>(const GramCall&, const GramWs&, int);
extern template ql_status gram_dispatch<float, ArithF64>(const GramCall&, const GramWs&, int);

}  // namespace ql
