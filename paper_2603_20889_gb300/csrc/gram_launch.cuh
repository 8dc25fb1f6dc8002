// Gram-pass kernel of CholQR2 / SVQB2 and its launch template (paper Sec. 3.1).
// Instantiated per (storage, arithmetic) in gram_inst_*.cu.
#pragma once

#include <mutex>

#include "epilogue.cuh"
#include "gram.cuh"
#include "internal.h"
#include "small_dense.cuh"
#include "gram_tc.cuh"
#include "gram_umma.cuh"
#include "gram_pipe.cuh"

namespace ql {

constexpr int kGramMaxCtasPerSm = 4;
// The double-float Gram accumulators are moved into FP64 every kGramFlushTiles tiles (and
// at the end), so that no double-float sum runs over more than a few thousand rows: the
// rounding of the long running sums (which grows like the square root of their length)
// happens in FP64, and the short double-float sums' errors are independent from one flush
// to the next.
constexpr int kGramFlushTiles = 16;

struct GramWs {
  int* flags;        // [0] range, [1] first-pass breakdown, [2] arrival counter pass 1, [3] pass 2,
                    // [64 + c]: largest biased exponent of column c over all rows (tensor-core pass 1)
  double* keep;      // 3 n x n blocks carried from pass 1 to pass 2 (row-major, ld n)
  double* partials;  // one NC x NC partial Gram per CTA
  double* fbuf;      // tcgen05 kernel: FP64 accumulators per CTA, [NC columns][128 TMEM lanes]
};

template <typename S>
struct GramArgs {
  ColSource<S> src;
  int64_t m;
  int n;
  int64_t tiles;
  int pass;    // 1 or 2
  int method;  // QL_CHOLQR2, QL_SVQB2 or QL_SCHOLQR3
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
  int bulk;  // every column starts 16-byte aligned: full tiles load with bulk copies
  // How the next pass's kernel reads the carried M (so that the epilogue can carry the exact
  // inverse of what it applies): 0 FP64 as is, 1 double-float per entry, 2 the tensor-core
  // slicing (48-bit fixed point per column of M' = diag(2^e_k) M).
  int mround;
  // Batched form only (null otherwise): the problem's flag in the batch's gated FP64 TSQR
  // launch, and that launch's any-flag.  A problem that leaves the double-float range (or,
  // with redo_on_breakdown, whose Cholesky breaks down) is handed to that launch instead of
  // the FP64 Gram launches of a single call.
  int* redo;
  int* redo_any;
  int redo_on_breakdown;
};

// Ask the batched FP64 TSQR launch to redo this problem.  Bits 8.. of the flag carry where a
// bounded wait gave up (0: none), which that launch reports as {QL_ERR_TIMEOUT, where}.
QL_DEV void gram_request_redo(int* redo, int* redo_any, int timeout_where = 0) {
  atomicOr(redo, 1 | (timeout_where << 8));
  atomicOr(redo_any, 1);
}

// Round the upper triangular M (n x n, row-major ld LE in shared memory) the way the next
// pass's kernel reads it (GramArgs::mround), in place.  colexp[k] is the largest biased
// exponent of column k of X (the tensor-core kernels scale row k of M by 2^(colexp[k] - 1022)).
template <int T>
QL_DEV void round_m_like_consumer(double* Ms, int ldm, int n, int mround, const int* colexp) {
  if (mround == 1) {
    for (int e = threadIdx.x; e < n * n; e += T) {
      double& v = Ms[(e / n) * ldm + e % n];
      const float hi = __double2float_rn(v);
      const float lo = __double2float_rn(v - (double)hi);
      v = (double)hi + (double)lo;
    }
  } else if (mround == 2) {
    for (int j = threadIdx.x; j < n; j += T) {  // one column per thread
      for (int it = 0; it < 4; ++it) {           // a value that rounds up to the next binade moves F
        int F = 0;
        for (int k = 0; k <= j; ++k) {
          const int ek = colexp[k];
          const double v = ek > 0 ? Ms[k * ldm + j] * __longlong_as_double((long long)(ek + 1) << 52) : 0.0;
          F = max(F, (int)((__double_as_longlong(v) >> 52) & 0x7ff));
        }
        if (F == 0) break;
        bool moved = false;
        for (int k = 0; k <= j; ++k) {
          const int ek = colexp[k];
          if (ek <= 0) {
            Ms[k * ldm + j] = 0.0;
            continue;
          }
          const double sc = __longlong_as_double((long long)(ek + 1) << 52);  // 2^(ek - 1022)
          const double v = Ms[k * ldm + j] * sc;
          // the value the kernel's digits represent: N 2^(F - 1022 - 48)
          const double r = (double)fixed48_of_double(v, F) * __longlong_as_double((long long)(F - 48 + 1) << 52);
          if (((__double_as_longlong(r) >> 52) & 0x7ff) > F) moved = true;
          Ms[k * ldm + j] = r / sc;
        }
        if (!moved) break;
      }
    }
  }
  __syncthreads();
}

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

// k: the number of CTA partials of this pass (the grid, or the chunks of one problem in a
// grouped launch).
template <int NC, int T, typename S, typename Ar>
QL_DEV void gram_finish(const GramArgs<S>& a, unsigned char* smem, const int* colmax, int* misc, int k);

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
  if (Ar::kRangeChecked && a.pass >= 2 && *(volatile int*)&a.w.flags[0] != 0) return;  // FP64 redoes it
  if (a.pass >= 2 && *(volatile int*)&a.w.flags[1] != 0) {  // first pass broke down
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
  double acc64[BS][BS];  // FP64 level of the double-float sums (stays zero in FP64 arithmetic)
#pragma unroll
  for (int i = 0; i < BS; ++i)
#pragma unroll
    for (int j = 0; j < BS; ++j) {
      acc[i][j] = Ar::acc_zero();
      acc64[i][j] = 0.0;
    }

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
    if constexpr (!std::is_same<Acc, double>::value) {
      if ((t - t0) % kGramFlushTiles == kGramFlushTiles - 1) {
#pragma unroll
        for (int i = 0; i < BS; ++i)
#pragma unroll
          for (int j = 0; j < BS; ++j) {
            acc64[i][j] += Ar::to_double(Ar::acc_get(acc[i][j]));
            acc[i][j] = Ar::acc_zero();
          }
      }
    }
  }
  __syncthreads();

  // reduce the row slices in FP64: red[(slice * NBT + blk) * BS * BS + i * BS + j]
  double* red = reinterpret_cast<double*>(Y0);
  if (active) {
#pragma unroll
    for (int i = 0; i < BS; ++i)
#pragma unroll
      for (int j = 0; j < BS; ++j)
        red[(slice * NBT + blk) * BS * BS + i * BS + j] = acc64[i][j] + Ar::to_double(Ar::acc_get(acc[i][j]));
  }
  __syncthreads();
  double* part = a.w.partials + (size_t)bid * NC * NC;
  for (int e = tid; e < NBT * BS * BS; e += T) {
    int b = e / (BS * BS), ij = e % (BS * BS);
    double s = red[b * BS * BS + ij];
    for (int sl = 1; sl < SL; ++sl) s += red[(sl * NBT + b) * BS * BS + ij];
    int rem = b, pp = 0;
    while (rem >= Sh::NB - pp) {
      rem -= Sh::NB - pp;
      ++pp;
    }
    int qq = pp + rem;
    int p = pp * BS + ij / BS, q = qq * BS + ij % BS;
    __stcg(part + p * NC + q, s);
  }
  gram_finish<NC, T, S, Ar>(a, smem, colmax, misc, gridDim.x);
}

// Range verdict, "last CTA done" election and, in the last CTA, the fixed-order reduction
// of all CTA partials followed by the n x n FP64 epilogue of the pass.  Shared by the SIMT
// and the tensor-core Gram kernels (the caller has written this CTA's partial already).
template <int NC, int T, typename S, typename Ar>
QL_DEV void gram_finish(const GramArgs<S>& a, unsigned char* smem, const int* colmax, int* misc, int k) {
  using V = typename Ar::T;
  const int tid = threadIdx.x, n = a.n;
  if (tid == 0) {
    bool bad = false;
    if constexpr (Ar::kRangeChecked) {
      const int emax = df_emax_limit(a.m);  // Gram entries reach m max|x|^2
      for (int c = 0; c < n; ++c) {
        int e = colmax[c];
        if (e != 0 && (e < kDfEminLimit || e > emax)) bad = true;
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
  if (Ar::kRangeChecked && *(volatile int*)&a.w.flags[0] != 0) {  // the FP64 launches redo it
    if (a.redo && tid == 0) gram_request_redo(a.redo, a.redo_any, *(volatile int*)&a.w.flags[4]);
    return;
  }

  // ---------------- epilogue: one CTA, FP64, shared memory reused from here on; the odd
  // leading dimension keeps column walks (Jacobi rotations) free of bank conflicts
  constexpr int LE = NC + 1;
  double* Cs = reinterpret_cast<double*>(smem);  // n x n, ld LE
  double* Us = Cs + NC * LE;
  double* Ps = Us + NC * LE;
  double* Qs = Ps + NC * LE;
  double* vec = Qs + NC * LE;  // 8 LE doubles
  int* sflag = reinterpret_cast<int*>(vec + 8 * LE);
  __syncthreads();
  // fixed-order FP64 sum of the CTA partials (bitwise reproducible).  P lanes share an
  // entry (as many as the thread count allows, up to a warp): each sums a strided subset of
  // the k partials, so the L2 loads overlap instead of forming one dependent chain of k, and
  // shuffles combine the P sums.
  {
    const int ne = n * n;
    int P = 32;
    while (P > 1 && ne * P > T) P >>= 1;
    const int per = T / P, iters = (ne + per - 1) / per;
    const int li = tid % P;
    for (int it = 0; it < iters; ++it) {
      const int e = tid / P + it * per;
      const int p = e / n, q = e % n;
      const bool use = e < ne && p <= q;
      double v = 0.0;
      if (use)
        for (int b = li; b < k; b += P) v += __ldcg(a.w.partials + (size_t)b * NC * NC + p * NC + q);
      for (int o = P >> 1; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
      if (use && li == 0) {
        Cs[p * LE + q] = v;
        Cs[q * LE + p] = v;
      }
    }
  }
  __syncthreads();
  double* keep = a.w.keep;  // [0]: R1 or S1, [1]: M (R1^{-1} or B1)
  const int nn = n * n;
  if (a.method == QL_TSQR) {
    // one column: the Householder reflector of x is determined by ||x||, so R = sqrt(x^T x)
    // (a zero column gives R = 0, not a breakdown)
    if (tid == 0) Ps[0] = sqrt(fmax(Cs[0], 0.0));
    __syncthreads();
  } else if (a.method == QL_CHOLQR2 || a.method == QL_SCHOLQR3) {
    const int last = a.method == QL_SCHOLQR3 ? 3 : 2;
    if (a.method == QL_SCHOLQR3 && a.pass == 1) {
      // shifted Cholesky: C1 + s I with s = 11 (m n + n (n + 1)) u ||X||_F^2, u = 2^-53
      if (tid == 0) {
        double tr = 0.0;
        for (int i = 0; i < n; ++i) tr += Cs[i * LE + i];
        const double sh = 11.0 * ((double)a.m * n + (double)n * (n + 1)) * 0x1p-53 * tr;
        for (int i = 0; i < n; ++i) Cs[i * LE + i] += sh;
      }
      __syncthreads();
    }
    int fail = chol_upper_inplace<T>(Cs, LE, n, sflag);
    if (fail) {
      if (a.pass < last) a.w.flags[1] = 1;
      if (a.redo && a.redo_on_breakdown) {  // batched, method chosen automatically: TSQR redoes it
        if (tid == 0) gram_request_redo(a.redo, a.redo_any);
        return;
      }
      write_nan_outputs(a, T);
      write_info(a.info, QL_ERR_NOT_SPD, fail + 1000 * (a.pass - 1));
      return;
    }
    if (a.pass < last) {
      // carry R (= R1, or R2 R1) and its inverse, the next pass's M, to the next pass
      if (a.pass > 1) {
        for (int e = tid; e < nn; e += T) Us[(e / n) * LE + e % n] = __ldcg(keep + e);
        __syncthreads();
        upper_times_upper<T>(Cs, LE, Us, LE, Ps, LE, n);
        for (int e = tid; e < nn; e += T) Cs[(e / n) * LE + e % n] = Ps[(e / n) * LE + e % n];
        __syncthreads();
      }
      tri_upper_inverse<T>(Cs, LE, Us, LE, n);
      if (a.mround) {
        // the next pass applies M rounded as its kernel reads it; carry that M and, as R,
        // its exact inverse, so that R_last ... R1 stays consistent with the Y it formed
        __syncthreads();
        round_m_like_consumer<T>(Us, LE, n, a.mround, a.w.flags + 64);
        tri_upper_inverse<T>(Us, LE, Cs, LE, n);
      }
      for (int e = tid; e < nn; e += T) {
        keep[e] = Cs[(e / n) * LE + e % n];
        keep[nn + e] = Us[(e / n) * LE + e % n];
      }
      return;
    }
    // last pass: R = R_last (R_prev ... R1)
    for (int e = tid; e < nn; e += T) Us[(e / n) * LE + e % n] = __ldcg(keep + e);
    __syncthreads();
    upper_times_upper<T>(Cs, LE, Us, LE, Ps, LE, n);
  } else {
    jacobi_eig<T>(Cs, LE, Us, LE, n, vec, sflag);
    // lambda_max and the truncation threshold
    double lmax = 0.0;
    for (int i = 0; i < n; ++i) lmax = fmax(lmax, Cs[i * LE + i]);
    double tol = a.rank_tol > 0.0 ? a.rank_tol : (double)n * 2.220446049250313e-16;
    double cut = tol * lmax;
    if (a.pass == 1) {
      for (int e = tid; e < nn; e += T) {
        int r = e / n, i = e % n;  // B1(r, i) = U(r, i) lambda_i^{-1/2};  S1(i, r) = lambda_i^{1/2} U(r, i)
        double li = Cs[i * LE + i];
        bool keepit = li > cut && li > 0.0;
        double sq = keepit ? sqrt(li) : 0.0;
        keep[nn + r * n + i] = keepit ? Us[r * LE + i] / sq : 0.0;
        keep[i * n + r] = sq * Us[r * LE + i];
      }
      return;
    }
    // pass 2: Z = S2 S1 with S2(i, r) = lambda2_i^{1/2} U2(r, i);  R = qr_r(Z)
    for (int e = tid; e < nn; e += T) {
      int i = e / n, r = e % n;
      double li = Cs[i * LE + i];
      bool keepit = li > cut && li > 0.0;
      Qs[i * LE + r] = (keepit ? sqrt(li) : 0.0) * Us[r * LE + i];
    }
    __syncthreads();
    for (int e = tid; e < nn; e += T) Us[(e / n) * LE + e % n] = __ldcg(keep + e);  // S1
    __syncthreads();
    full_times_full<T>(Qs, LE, Us, LE, Ps, LE, n);
    if (a.Z && a.epilogue == kEpiR)
      for (int e = tid; e < nn; e += T) a.Z[(e / n) * n + e % n] = Ps[(e % n) * LE + e / n];  // column-major
    __syncthreads();
    householder_square<T>(Ps, LE, n, vec);
  }
  // a bounded wait of the double-float launches that gave up (flags[4] = where) is reported
  // by the FP64 launches that completed the call
  const int tmo = *(volatile int*)&a.w.flags[4];
  if (a.epilogue == kEpiR)
    epilogue_r<T>(Ps, LE, n, a.R, a.ldr, a.info, sflag, tmo);
  else
    epilogue_lstsq<T>(Ps, LE, n, a.x, a.resnorm, a.Rext, a.info, vec, sflag, tmo);
}


// ---------------------------------------------------------------------------------------
// Streaming Gram pass for narrow X (n <= 4).  There is no shared-memory staging: every
// thread loads 16-byte vectors of its columns straight into registers (U of them per column
// in flight), converts them, applies M in the later passes (M in shared memory, read by
// broadcast) and adds the n (n + 1) / 2 products of each row into its own accumulators.
// A thread sums only m / (CTAs x 256) rows, so its double-float sums stay short; they are
// added across the warp by shuffles and across warps and CTAs in FP64, then the same
// last-CTA epilogue as the other Gram kernels runs.
// ---------------------------------------------------------------------------------------
template <int NC>
struct StreamShape {
  static constexpr int T = 256;
  static constexpr int U = NC <= 1 ? 8 : (NC <= 2 ? 4 : 2);  // 16-byte loads per column and batch
  static constexpr int kMaxCtasPerSm = 8;
  static constexpr int NE = NC * (NC + 1) / 2;                 // upper-triangle entries
};

template <int NC, typename S, typename Ar>
struct StreamSmem {
  using Sh = StreamShape<NC>;
  static constexpr size_t kM = sizeof(typename Ar::T) * NC * NC;
  static constexpr size_t kOffRed = (kM + 15) / 16 * 16;
  static constexpr size_t kOffMisc = kOffRed + sizeof(double) * (Sh::T / 32) * Sh::NE;
  static constexpr size_t kMain = kOffMisc + (64 + NC) * sizeof(int);
  static constexpr size_t kEpi = GramSmem<NC, S, Ar>::kEpi + 64 * sizeof(int) + 16;
  static constexpr size_t kBytes = kMain > kEpi ? kMain : kEpi;
};

template <typename S>
QL_DEV void load16(S (&v)[16 / sizeof(S)], const S* p);
template <>
QL_DEV void load16<double>(double (&v)[2], const double* p) {
  const double2 t = __ldg(reinterpret_cast<const double2*>(p));
  v[0] = t.x;
  v[1] = t.y;
}
template <>
QL_DEV void load16<float>(float (&v)[4], const float* p) {
  const float4 t = __ldg(reinterpret_cast<const float4*>(p));
  v[0] = t.x;
  v[1] = t.y;
  v[2] = t.z;
  v[3] = t.w;
}

template <int NC, typename S, typename Ar, int XF>
__global__ void __launch_bounds__(StreamShape<NC>::T) gram_stream_kernel(GramArgs<S> a) {
  using Sh = StreamShape<NC>;
  using Sm = StreamSmem<NC, S, Ar>;
  using V = typename Ar::T;
  using Acc = typename Ar::Acc;
  constexpr int T = Sh::T, U = Sh::U, NE = Sh::NE, EPV = 16 / (int)sizeof(S), NW = T / 32;
  extern __shared__ __align__(16) unsigned char smem[];
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5, n = a.n;

  if (a.gated && *(volatile int*)&a.w.flags[0] == 0) return;
  if (Ar::kRangeChecked && a.pass >= 2 && *(volatile int*)&a.w.flags[0] != 0) return;  // FP64 redoes it
  if (a.pass >= 2 && *(volatile int*)&a.w.flags[1] != 0) {  // first pass broke down
    if (blockIdx.x == 0) write_nan_outputs(a, T);
    return;
  }
  V* Mv = reinterpret_cast<V*>(smem);
  double* red = reinterpret_cast<double*>(smem + Sm::kOffRed);
  int* misc = reinterpret_cast<int*>(smem + Sm::kOffMisc);
  int* colmax = misc + 64;
  for (int i = tid; i < NC; i += T) colmax[i] = 0;
  if constexpr (XF != kXNone) {
    const double* M = a.w.keep + (size_t)n * n;  // the previous pass's M (row-major, ld n)
    for (int i = tid; i < NC * NC; i += T) {
      const int r = i / NC, c = i % NC;
      Mv[i] = (r < n && c < n) ? Ar::from_double(__ldcg(M + r * n + c)) : Ar::zero();
    }
  }
  __syncthreads();

  Acc acc[NE];
#pragma unroll
  for (int e = 0; e < NE; ++e) acc[e] = Ar::acc_zero();
  unsigned emax[NC];
#pragma unroll
  for (int c = 0; c < NC; ++c) emax[c] = 0;
  const S* col[NC];
#pragma unroll
  for (int c = 0; c < NC; ++c) col[c] = a.src.col(c < n ? c : 0);

  // this CTA's rows, in 16-byte units of EPV rows; batches of U units per thread, the next
  // batch's loads issued before the current batch is consumed (two register buffers)
  const int64_t units = (a.m + EPV - 1) / EPV;
  const int64_t u0 = units * blockIdx.x / gridDim.x, u1 = units * (blockIdx.x + 1) / gridDim.x;
  const int64_t step = (int64_t)T * U;
  auto load_batch = [&](S (&v)[U][NC][EPV], int64_t ub) {
#pragma unroll
    for (int u = 0; u < U; ++u) {
      const int64_t uu = ub + (int64_t)u * T + tid;
      const int64_t row = uu * EPV;
#pragma unroll
      for (int c = 0; c < NC; ++c) {
        if (c < n && uu < u1 && a.bulk && row + EPV <= a.m) {
          load16<S>(v[u][c], col[c] + row);
        } else {
#pragma unroll
          for (int e = 0; e < EPV; ++e)
            v[u][c][e] = (c < n && uu < u1 && row + e < a.m) ? __ldg(col[c] + row + e) : S(0);
        }
      }
    }
  };
  auto consume_batch = [&](const S (&v)[U][NC][EPV]) {
#pragma unroll
    for (int u = 0; u < U; ++u)
#pragma unroll
      for (int e = 0; e < EPV; ++e) {
        V y[NC];
#pragma unroll
        for (int c = 0; c < NC; ++c) {
          int E;
          y[c] = Ar::load(v[u][c][e], E);
          if constexpr (Ar::kRangeChecked) emax[c] = max(emax[c], (unsigned)E);
        }
        if constexpr (XF != kXNone) {  // y = x M, one row
          V x[NC];
#pragma unroll
          for (int c = 0; c < NC; ++c) x[c] = y[c];
#pragma unroll
          for (int j = 0; j < NC; ++j) {
            Acc s = Ar::acc_zero();
#pragma unroll
            for (int k = 0; k < NC; ++k)
              if (XF != kXUpper || k <= j) Ar::acc_fma(s, x[k], Mv[k * NC + j]);
            y[j] = Ar::acc_get(s);
          }
        }
        int ei = 0;
#pragma unroll
        for (int i = 0; i < NC; ++i)
#pragma unroll
          for (int j = i; j < NC; ++j) Ar::acc_fma(acc[ei++], y[i], y[j]);
      }
  };
  S bufA[U][NC][EPV], bufB[U][NC][EPV];
  if (u0 < u1) load_batch(bufA, u0);
  for (int64_t ub = u0; ub < u1; ub += 2 * step) {
    if (ub + step < u1) load_batch(bufB, ub + step);
    consume_batch(bufA);
    if (ub + 2 * step < u1) load_batch(bufA, ub + 2 * step);
    if (ub + step < u1) consume_batch(bufB);
  }

  if constexpr (Ar::kRangeChecked) {
#pragma unroll
    for (int c = 0; c < NC; ++c) {
      const unsigned em = __reduce_max_sync(0xffffffffu, emax[c]);
      if (lane == 0 && em > 0) atomicMax(&colmax[c], (int)em);
    }
  }
  // warp sums (shuffles), then warps and CTAs in FP64
#pragma unroll
  for (int e = 0; e < NE; ++e) {
    V v = Ar::acc_get(acc[e]);
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v = Ar::add(v, Ar::shfl(v, o));
    if (lane == 0) red[warp * NE + e] = Ar::to_double(v);
  }
  __syncthreads();
  double* part = a.w.partials + (size_t)blockIdx.x * NC * NC;
  for (int e = tid; e < NE; e += T) {
    double v = 0.0;
    for (int w = 0; w < NW; ++w) v += red[w * NE + e];
    int i = 0, rem = e;
    while (rem >= NC - i) {
      rem -= NC - i;
      ++i;
    }
    __stcg(part + i * NC + (i + rem), v);
  }
  gram_finish<NC, T, S, Ar>(a, smem, colmax, misc, gridDim.x);
}

template <int NC, typename S, typename Ar, int XF>
ql_status gram_stream_launch_one(const GramCall& c, const GramWs& w, int pass, int gated) {
  using Sh = StreamShape<NC>;
  using Sm = StreamSmem<NC, S, Ar>;
  auto kern = gram_stream_kernel<NC, S, Ar, XF>;
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
      occ = o < 1 ? 1 : (o > Sh::kMaxCtasPerSm ? Sh::kMaxCtasPerSm : o);
    }
  }
  constexpr int EPV = 16 / (int)sizeof(S);
  const int64_t units = (c.m + EPV - 1) / EPV;
  int64_t g = (int64_t)device_sm_count() * occ;
  const int64_t need = (units + (int64_t)Sh::T * Sh::U - 1) / ((int64_t)Sh::T * Sh::U);  // one sweep per CTA at least
  if (g > need) g = need;
  if (g < 1) g = 1;
  GramArgs<S> a{};
  a.src.A = static_cast<const S*>(c.A);
  a.src.lda = c.lda;
  a.src.b = static_cast<const S*>(c.b);
  a.src.nA = c.nA;
  a.m = c.m;
  a.n = c.n;
  a.tiles = 0;
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
  {
    auto aligned = [](const void* p) { return (reinterpret_cast<uintptr_t>(p) & 15u) == 0; };
    bool b = aligned(c.A) && ((size_t)c.lda * sizeof(S)) % 16 == 0;
    if (c.nA < c.n) b = b && aligned(c.b);
    a.bulk = b ? 1 : 0;  // 16-byte loads
  }
  a.mround = std::is_same<Ar, ArithDF>::value ? 1 : 0;
  count_launch();
  kern<<<(int)g, Sh::T, Sm::kBytes, c.stream>>>(a);
  return cudaPeekAtLastError() == cudaSuccess ? QL_OK : QL_ERR_CUDA;
}

// Tensor-core Gram pass (double-float policy only): see gram_tc.cuh.  The body handles the
// row tiles [tiles bid / k, tiles (bid + 1) / k) of one problem as partial `bid` of `k`; the
// single-call kernel runs it with bid = CTA, k = grid, the grouped kernel of the batched form
// once per (problem, chunk) work item.
template <int NC, typename S, int XF>
QL_DEV void gram_tc_body(const GramArgs<S>& a, int bid, int k) {
  using Ar = ArithDF;
  using Sh = TcShape<NC>;
  using Sm = TcSmem<NC, S>;
  constexpr int T = 256, KT = Sh::KT, LDR = Sh::LDR, G = Sh::G, KS = Sh::KS, KPART = Sh::KPART;
  constexpr int GPR = Sh::NCB / G;              // column-block groups per row block
  constexpr int PAIRS = NC * KT / 2 / T;        // row pairs per thread and tile
  constexpr int LDY = Sm::LDY;
  constexpr int KSTEPS = NC / 16;               // 16-wide k-steps of Y = X M'
  constexpr int WPC = 8 / Sh::NCB;              // warps per 8-column block of Y
  extern __shared__ __align__(16) unsigned char smem[];
  const int tid = threadIdx.x, n = a.n, lane = tid & 31, warp = tid >> 5;

  if (a.pass >= 2 && *(volatile int*)&a.w.flags[0] != 0) return;  // the FP64 launches redo it
  if (a.pass >= 2 && *(volatile int*)&a.w.flags[1] != 0) {         // first pass broke down
    if (bid == 0) write_nan_outputs(a, T);
    return;
  }
  S* stage = reinterpret_cast<S*>(smem);
  df* ydf = reinterpret_cast<df*>(smem);  // second pass: the Y tile, column c at c * LDY
  unsigned short* slices = reinterpret_cast<unsigned short*>(smem + Sm::kOffSlices);
  float* pow2c = reinterpret_cast<float*>(smem + Sm::kOffPow);
  int* expo = reinterpret_cast<int*>(smem + Sm::kOffExpo);
  int* colmax = reinterpret_cast<int*>(smem + Sm::kOffColmax);
  int* gexp = reinterpret_cast<int*>(smem + Sm::kOffGexp);
  unsigned* zero16 = reinterpret_cast<unsigned*>(smem + Sm::kOffZero);
  int* misc = reinterpret_cast<int*>(smem + Sm::kOffMisc);

  for (int i = tid; i < NC; i += T) {
    colmax[i] = 0;
    gexp[i] = (XF != kXNone && i < n) ? __ldcg(&a.w.flags[64 + i]) : 0;
  }
  if (tid < 4) zero16[tid] = 0u;
  __syncthreads();
  constexpr int U = Sh::U;
  const int g = lane >> 2, t4 = lane & 3;

  // ---- second pass: this warp's 8-column block of Y and the B fragments of M' = diag(2^e_k) M
  // Upper-triangular M' (Cholesky-QR2) needs k-steps 0..cbw/2 only; with NC = 64 the blocks
  // are paired so that the two warps on one scheduler share 5 k-steps.
  const int cbw = (NC == 64 && warp >= 4) ? 11 - warp : warp / WPC;
  const int rpart = (NC == 64) ? 0 : warp % WPC;
  const int ksw = XF == kXUpper ? (cbw >> 1) + 1 : KSTEPS;
  unsigned bq[XF != kXNone ? KSTEPS : 1][7][2];
  float ysc[2][7];  // 2^(f_j - 12 - 7d) for this thread's two Y columns and the 7 weights
  if constexpr (XF != kXNone) {
    const double* M = a.w.keep + (size_t)n * n;  // pass-1 output, row-major, ld n
    const int jb = cbw * 8 + g;
    double mv[KSTEPS][4];
    int F = 0;
#pragma unroll
    for (int ks = 0; ks < KSTEPS; ++ks)
#pragma unroll
      for (int h = 0; h < 4; ++h) {
        const int k = 16 * ks + 2 * t4 + (h & 1) + 8 * (h >> 1);
        double v = 0.0;
        if (k < n && jb < n && (XF != kXUpper || k <= jb)) {
          const int ek = gexp[k];
          if (ek > 0) v = __ldcg(M + (size_t)k * n + jb) * __longlong_as_double((long long)(ek + 1) << 52);
        }
        mv[ks][h] = v;
        F = max(F, (int)((__double_as_longlong(v) >> 52) & 0x7ff));
      }
    F = max(F, __shfl_xor_sync(0xffffffffu, F, 1));
    F = max(F, __shfl_xor_sync(0xffffffffu, F, 2));  // max over column jb of M'
#pragma unroll
    for (int ks = 0; ks < KSTEPS; ++ks) {
      long long Nb[4];
#pragma unroll
      for (int h = 0; h < 4; ++h) Nb[h] = fixed48_of_double(mv[ks][h], F) + kDigitBias;
#pragma unroll
      for (int q = 0; q < 7; ++q) {
        bq[ks][q][0] = bf16x2_of_ints(balanced_digit_rt(Nb[0], q), balanced_digit_rt(Nb[1], q));
        bq[ks][q][1] = bf16x2_of_ints(balanced_digit_rt(Nb[2], q), balanced_digit_rt(Nb[3], q));
      }
    }
    // the flush scale of this thread's Y columns cbw*8 + 2 t4 + h must stay a normal float
    bool bad = false;
#pragma unroll
    for (int h = 0; h < 2; ++h) {
      const int Fj = __shfl_sync(0xffffffffu, F, 4 * (2 * t4 + h));
      const int f = Fj - 1022;  // |M'(:, j)| < 2^f
      if (Fj > 0 && (f < -70 || f > 100)) bad = true;
#pragma unroll
      for (int d = 0; d < 7; ++d) {
        const int e = f - kDigitScaleLog2 - 7 * d;
        ysc[h][d] = (Fj > 0 && !bad) ? __int_as_float((e + 127) << 23) : 0.0f;
      }
    }
    if (__syncthreads_or(bad)) {  // out of the double-float range: the FP64 launches redo it
      if (tid == 0) atomicOr(&a.w.flags[0], 1);
      gram_finish<NC, T, S, ArithDF>(a, smem, colmax, misc, k);
      return;
    }
  }

  df acc[U][G][4];        // per-unit C accumulators over the last few tiles
  double acc64[U][G][4];  // and their FP64 level
#pragma unroll
  for (int ui = 0; ui < U; ++ui)
#pragma unroll
    for (int gi = 0; gi < G; ++gi)
#pragma unroll
      for (int e = 0; e < 4; ++e) {
        acc[ui][gi][e] = df{0.0f, 0.0f};
        acc64[ui][gi][e] = 0.0;
      }

  const int64_t t0 = a.tiles * bid / k, t1 = a.tiles * (bid + 1) / k;
  auto issue = [&](int64_t t) {
    const int64_t row0 = t * KT;
#pragma unroll 1
    for (int c = 0; c < NC; ++c) {
      const S* col = a.src.col(c < n ? c : 0);
      for (int r = tid; r < KT; r += T) {
        int64_t row = row0 + r;
        bool v = c < n && row < a.m;
        cp_async_elem<S>(stage + c * KT + r, v ? col + row : col, v);
      }
    }
    cp_async_commit();
  };
  // seven signed base-128 digits of the staged X per value, two rows per 32-bit store;
  // ex[c] is the biased double exponent that bounds column c
  auto slice_stage = [&](const int* ex) {
#pragma unroll 4
    for (int k2 = 0; k2 < PAIRS; ++k2) {
      const int pi = tid + T * k2, c = (2 * pi) / KT, r = (2 * pi) % KT;
      const int em = ex[c];
      long long Nb[2];
#pragma unroll
      for (int h = 0; h < 2; ++h) {
        if constexpr (sizeof(S) == 8) {
          Nb[h] = (em > 0 ? fixed48_of_double((double)stage[c * KT + r + h], em) : 0ll) + kDigitBias;
        } else {
          Nb[h] = (em > 0 ? fixed48_of_float((float)stage[c * KT + r + h], em - 896) : 0ll) + kDigitBias;
        }
      }
#pragma unroll
      for (int p = 0; p < Sh::ND; ++p)
        *reinterpret_cast<unsigned*>(slices + ((size_t)p * NC + c) * LDR + r) =
            bf16x2_of_ints(balanced_digit_rt(Nb[0], p), balanced_digit_rt(Nb[1], p));
    }
  };

  if (t0 < t1) issue(t0);
  __syncthreads();
  for (int64_t t = t0; t < t1; ++t) {
    cp_async_wait_all();
    __syncthreads();
    for (int i = tid; i < NC; i += T) expo[i] = 0;
    __syncthreads();
    if constexpr (XF == kXNone) {
      // column maxima of the biased double exponent (and the range record)
#pragma unroll 4
      for (int k2 = 0; k2 < PAIRS; ++k2) {
        const int pi = tid + T * k2, c = (2 * pi) / KT, r = (2 * pi) % KT;
        unsigned em;
        if constexpr (sizeof(S) == 8) {
          unsigned long long b0 = (unsigned long long)__double_as_longlong((double)stage[c * KT + r]);
          unsigned long long b1 = (unsigned long long)__double_as_longlong((double)stage[c * KT + r + 1]);
          em = max((unsigned)((b0 >> 52) & 0x7ff), (unsigned)((b1 >> 52) & 0x7ff));
        } else {
          unsigned e0 = (__float_as_uint((float)stage[c * KT + r]) >> 23) & 0xff;
          unsigned e1 = (__float_as_uint((float)stage[c * KT + r + 1]) >> 23) & 0xff;
          em = max(e0 ? e0 + 896 : 0u, e1 ? e1 + 896 : 0u);
        }
        em = __reduce_max_sync(0xffffffffu, em);
        if (lane == 0 && em > 0) {
          atomicMax(&expo[c], (int)em);
          atomicMax(&colmax[c], (int)em);
        }
      }
      __syncthreads();
      // per-column scale 2^e_c, |x| < 2^e_c for the whole tile column
      for (int c = tid; c < NC; c += T) {
        const int em = expo[c];
        pow2c[c] = __int_as_float((max(-126, min(127, em > 0 ? em - 1022 : 0)) + 127) << 23);
      }
      slice_stage(expo);
    } else {
      slice_stage(gexp);
      __syncthreads();
      // Y = X M' on the tensor cores: per 16 x 8 block the 28 digit pairs (p + q <= 6, weight
      // d = p + q + 2 <= 8) accumulate exactly in FP32 per weight, then fold into double-float
      float ymax[2] = {0.0f, 0.0f};
#pragma unroll 1
      for (int i = 0; i < 8; ++i) {
        const int rb = rpart + WPC * i;
        float ac[7][4];
#pragma unroll
        for (int d = 0; d < 7; ++d)
#pragma unroll
          for (int e = 0; e < 4; ++e) ac[d][e] = 0.0f;
#pragma unroll
        for (int ks = 0; ks < KSTEPS; ++ks) {
          if (ks < ksw) {
            unsigned af[7][4];
            const int krow = 16 * ks + 8 * (lane >> 4) + (lane & 7);
            const int rcol = 16 * rb + 8 * ((lane >> 3) & 1);
#pragma unroll
            for (int p = 0; p < 7; ++p)
              ldsm_x4_t(af[p][0], af[p][1], af[p][2], af[p][3], slices + ((size_t)p * NC + krow) * LDR + rcol);
#pragma unroll
            for (int p = 0; p < 7; ++p)
#pragma unroll
              for (int q = 0; q + p < 7; ++q)
                mma_bf16(ac[p + q], af[p][0], af[p][1], af[p][2], af[p][3], bq[ks][q][0], bq[ks][q][1]);
          }
        }
#pragma unroll
        for (int e = 0; e < 4; ++e) {
          const int h = e & 1;
          float hi = ac[6][e] * ysc[h][6], lo = 0.0f;  // smallest weight first
#pragma unroll
          for (int d = 5; d >= 0; --d) {
            float s, err;
            two_sum(hi, ac[d][e] * ysc[h][d], s, err);
            hi = s;
            lo = __fadd_rn(lo, err);
          }
          const df y = df_make(hi, lo);
          ymax[h] = fmaxf(ymax[h], fabsf(y.hi));
          ydf[(cbw * 8 + 2 * t4 + h) * LDY + 16 * rb + g + 8 * (e >> 1)] = y;
        }
      }
#pragma unroll
      for (int h = 0; h < 2; ++h) {
        float v = ymax[h];
        v = fmaxf(v, __shfl_xor_sync(0xffffffffu, v, 4));
        v = fmaxf(v, __shfl_xor_sync(0xffffffffu, v, 8));
        v = fmaxf(v, __shfl_xor_sync(0xffffffffu, v, 16));
        const int em = (__float_as_int(v) >> 23) & 0xff;
        if (g == 0 && em > 0) atomicMax(&expo[cbw * 8 + 2 * t4 + h], em);
      }
      __syncthreads();
      // per-column scale 2^e_c, |y| < 2^e_c for the whole tile column
      for (int c = tid; c < NC; c += T) {
        const int em = expo[c];
        pow2c[c] = __int_as_float((max(-126, min(127, em > 0 ? em - 126 : 0)) + 127) << 23);
      }
      // slicing of Y: seven signed base-128 digits per value, two rows per 32-bit store
#pragma unroll 4
      for (int k2 = 0; k2 < PAIRS; ++k2) {
        const int pi = tid + T * k2, c = (2 * pi) / KT, r = (2 * pi) % KT;
        const int em = expo[c];
        long long Nb[2];
#pragma unroll
        for (int h = 0; h < 2; ++h) {
          const df y = ydf[c * LDY + r + h];
          Nb[h] = fixed48_of_float(y.hi, em) + fixed48_of_float(y.lo, em) + kDigitBias;
        }
#pragma unroll
        for (int p = 0; p < Sh::ND; ++p)
          *reinterpret_cast<unsigned*>(slices + ((size_t)p * NC + c) * LDR + r) =
              bf16x2_of_ints(balanced_digit_rt(Nb[0], p), balanced_digit_rt(Nb[1], p));
      }
    }
    __syncthreads();
    if (t + 1 < t1) issue(t + 1);
    // tensor-core digit products: per k-step, the fragments of all 7 digits are loaded
    // once and the 28 digit pairs (p + q <= 8) accumulate into one FP32 accumulator per
    // weight d = p + q; each accumulator is flushed (scaled, exact) into double-float.
#pragma unroll
    for (int ui = 0; ui < U; ++ui) {
      const int u = warp * U + ui, grp = u / KS, kp = u % KS;
      const int rb = grp / GPR, cb0 = (grp % GPR) * G;
      const int kbase = kp * KPART;
      const int ri0 = rb * 16 + g, ri1 = ri0 + 8;
      const float fi0 = ri0 < NC ? pow2c[ri0] : 0.0f, fi1 = ri1 < NC ? pow2c[ri1] : 0.0f;
      const int arow = rb * 16 + (lane & 15);
      const bool azero = NC < 16 && arow >= NC;
      float accd[7][G][4];
#pragma unroll
      for (int dd = 0; dd < 7; ++dd)
#pragma unroll
        for (int gi = 0; gi < G; ++gi)
#pragma unroll
          for (int e = 0; e < 4; ++e) accd[dd][gi][e] = 0.0f;
#pragma unroll 1
      for (int ks = 0; ks < KPART / 16; ++ks) {
        const int kk = kbase + ks * 16;
        unsigned af[7][4];
#pragma unroll
        for (int p = 0; p < 7; ++p) {
          const void* ap = azero ? (const void*)zero16
                                 : (const void*)(slices + ((size_t)p * NC + arow) * LDR + kk + (lane >> 4) * 8);
          ldsm_x4(af[p][0], af[p][1], af[p][2], af[p][3], ap);
        }
#pragma unroll
        for (int gi = 0; gi < G; ++gi) {
          unsigned bf[7][2];
          const int brow = (cb0 + gi) * 8 + (lane & 7);
#pragma unroll
          for (int q = 0; q < 7; ++q)
            ldsm_x2(bf[q][0], bf[q][1], slices + ((size_t)q * NC + brow) * LDR + kk + ((lane >> 3) & 1) * 8);
#pragma unroll
          for (int p = 0; p < 7; ++p)
#pragma unroll
            for (int q = 0; q + p < 7; ++q)  // digits p+1, q+1: weight d = p + q + 2 <= 8
              mma_bf16(accd[p + q][gi], af[p][0], af[p][1], af[p][2], af[p][3], bf[q][0], bf[q][1]);
        }
      }
      // fold the seven weights of each entry (weights 6..3 in FP32, together below 2^-21 of
      // the leading one; 2..0 with exact two-sums), scale by 2^(e_i + e_j) and add once
#pragma unroll
      for (int gi = 0; gi < G; ++gi) {
        const float fj0 = pow2c[(cb0 + gi) * 8 + 2 * t4], fj1 = pow2c[(cb0 + gi) * 8 + 2 * t4 + 1];
        const float f4[4] = {fi0 * fj0, fi0 * fj1, fi1 * fj0, fi1 * fj1};
#pragma unroll
        for (int e = 0; e < 4; ++e) {
          float hi = accd[6][gi][e] * __int_as_float((127 - kDigitScaleLog2 - 42) << 23);
#pragma unroll
          for (int dd = 5; dd >= 3; --dd)
            hi = __fmaf_rn(accd[dd][gi][e], __int_as_float((127 - kDigitScaleLog2 - 7 * dd) << 23), hi);
          float lo = 0.0f;
#pragma unroll
          for (int dd = 2; dd >= 0; --dd) {
            float s2, e2;
            two_sum(hi, accd[dd][gi][e] * __int_as_float((127 - kDigitScaleLog2 - 7 * dd) << 23), s2, e2);
            hi = s2;
            lo = __fadd_rn(lo, e2);
          }
          acc[ui][gi][e] = df_add(acc[ui][gi][e], df{hi * f4[e], lo * f4[e]});
        }
      }
    }
    if ((t - t0) % kGramFlushTiles == kGramFlushTiles - 1) {  // double-float sums -> FP64
#pragma unroll
      for (int ui = 0; ui < U; ++ui)
#pragma unroll
        for (int gi = 0; gi < G; ++gi)
#pragma unroll
          for (int e = 0; e < 4; ++e) {
            acc64[ui][gi][e] += df_to_double(acc[ui][gi][e]);
            acc[ui][gi][e] = df{0.0f, 0.0f};
          }
    }
  }
  __syncthreads();
  if constexpr (XF == kXNone) {  // column exponents of the whole matrix, for the second pass
    for (int c = tid; c < n; c += T)
      if (colmax[c] > 0) atomicMax(&a.w.flags[64 + c], colmax[c]);
  }
  // combine the row parts of each C tile (FP64) and store this CTA's partial Gram matrix
  double* red = reinterpret_cast<double*>(smem + Sm::kOffSlices);  // [unit][G][4][32]
#pragma unroll
  for (int ui = 0; ui < U; ++ui)
#pragma unroll
    for (int gi = 0; gi < G; ++gi)
#pragma unroll
      for (int e = 0; e < 4; ++e)
        red[(((warp * U + ui) * G + gi) * 4 + e) * 32 + lane] = acc64[ui][gi][e] + df_to_double(acc[ui][gi][e]);
  __syncthreads();
  double* part = a.w.partials + (size_t)bid * NC * NC;
  for (int idx = tid; idx < Sh::GROUPS * G * 4 * 32; idx += T) {
    const int ln = idx % 32, e = (idx / 32) % 4, gi = (idx / 128) % G, gr = idx / (128 * G);
    double s = 0.0;
    for (int kq = 0; kq < KS; ++kq) s += red[(((gr * KS + kq) * G + gi) * 4 + e) * 32 + ln];
    const int rb2 = gr / GPR, cbb = (gr % GPR) * G + gi;
    const int i = rb2 * 16 + (ln >> 2) + (e >= 2 ? 8 : 0), j = cbb * 8 + 2 * (ln & 3) + (e & 1);
    if (i < NC && j < NC) __stcg(part + i * NC + j, s);
  }
  gram_finish<NC, T, S, ArithDF>(a, smem, colmax, misc, k);
}

template <int NC, typename S, int XF>
__global__ void __launch_bounds__(256, 1) gram_tc_kernel(GramArgs<S> a) {
  gram_tc_body<NC, S, XF>(a, blockIdx.x, gridDim.x);
}

template <int NC, typename S, int XF>
ql_status gram_tc_launch_one(const GramCall& c, const GramWs& w, int pass) {
  using Sh = TcShape<NC>;
  using Sm = TcSmem<NC, S>;
  auto kern = gram_tc_kernel<NC, S, XF>;
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
  const int64_t tiles = (c.m + Sh::KT - 1) / Sh::KT;
  int64_t g = (int64_t)device_sm_count() * occ;
  if (g > tiles) g = tiles;
  if (g < 1) g = 1;
  GramArgs<S> a{};
  a.src.A = static_cast<const S*>(c.A);
  a.src.lda = c.lda;
  a.src.b = static_cast<const S*>(c.b);
  a.src.nA = c.nA;
  a.m = c.m;
  a.n = c.n;
  a.tiles = tiles;
  a.pass = pass;
  a.method = c.method;
  a.gated = 0;
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
  a.mround = 2;
  count_launch();
  kern<<<(int)g, Sh::T, Sm::kBytes, c.stream>>>(a);
  return cudaPeekAtLastError() == cudaSuccess ? QL_OK : QL_ERR_CUDA;
}

// Tensor-core Gram pass on tcgen05 (double-float policy only): see gram_umma.cuh.  The
// second pass forms Y = X M' with mma.sync as in gram_tc_kernel (B fragments of M' in
// registers), reading X's digit planes in the core-matrix layout.
// Block size: 512 threads for the first pass (latency-bound slicing and TMEM read-out gain
// from 16 warps), 256 for the later passes (their M' fragments need the registers).
template <int XF>
__host__ __device__ constexpr int umma_threads() {
  return XF == kXNone ? 512 : 256;
}

// Phase parities of the two barriers of a tcgen05 Gram CTA, carried from one work item to
// the next; ok turns false (uniformly across the CTA) once a bounded wait gave up.
struct UmmaBars {
  uint32_t phase = 0;   // MMA-completion barrier
  uint32_t lphase = 0;  // tile (bulk copy) barrier
  bool ok = true;
};

// Per-CTA set-up of the tcgen05 Gram kernels: the tensor-memory columns (written to *tslot
// and returned) and the two barriers at UmmaSmem::kOffBar, each initialised once.
template <int NC, typename S>
QL_DEV uint32_t umma_cta_begin(unsigned char* smem, uint32_t* tslot) {
  using Sm = UmmaSmem<NC, S>;
  if ((threadIdx.x >> 5) == 0) tmem_alloc(tslot, UmmaShape<NC>::TCOLS);
  if (threadIdx.x == 0) {
    mbar_init(reinterpret_cast<uint64_t*>(smem + Sm::kOffBar), 1);
    mbar_init(reinterpret_cast<uint64_t*>(smem + Sm::kOffBar + 8), 1);
  }
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  return *tslot;
}

// The body handles partial `bid` of `k` of one problem (see gram_tc_body) with the 512
// tensor-memory columns at tbase and the barriers that its caller set up (umma_cta_begin).
template <int NC, typename S, int XF>
QL_DEV void gram_umma_body(const GramArgs<S>& a, int bid, int k, uint32_t tbase, UmmaBars& bars) {
  using Sh = UmmaShape<NC>;
  using Sm = UmmaSmem<NC, S>;
  constexpr int T = umma_threads<XF>(), NW = T / 32, KT = Sh::KT, LDS = Sm::LDS, LDY = Sm::LDY, SP = Sh::SP,
                PLANE = Sh::PLANE;
  constexpr int SBO = Sh::SBO, LBO = Sh::LBO;
  constexpr int PAIRS = NC * KT / 2 / T;        // row pairs (and core-matrix quarters) per thread and tile
  constexpr int KSTEPS = NC / 16;               // 16-wide k-steps of Y = X M'
  constexpr int WPC = 8 / (NC / 8);             // warps per 8-column block of Y
  constexpr int HALF = NC / (NW / 4);           // accumulator columns per thread (NW / 4 warps per lane quarter)
  constexpr int CPG = KT / 8;                   // core matrices per 8-column group
  constexpr uint32_t IDESC = umma_idesc_bf16(128, NC);
  extern __shared__ __align__(1024) unsigned char smem_umma[];
  unsigned char* smem = smem_umma;
  const int tid = threadIdx.x, n = a.n, lane = tid & 31, warp = tid >> 5;

  if (a.pass >= 2 && *(volatile int*)&a.w.flags[0] != 0) return;  // the FP64 launches redo it
  if (a.pass >= 2 && *(volatile int*)&a.w.flags[1] != 0) {         // first pass broke down
    if (bid == 0) write_nan_outputs(a, T);
    return;
  }
  unsigned char* digits = smem;  // 7 planes, core-matrix layout
  S* stage = reinterpret_cast<S*>(smem + Sm::kOffStage);
  df* ydf = reinterpret_cast<df*>(smem + Sm::kOffStage);  // second pass: Y, column c at c * LDY
  float* pow2c = reinterpret_cast<float*>(smem + Sm::kOffPow);
  int* expo = reinterpret_cast<int*>(smem + Sm::kOffExpo);
  int* colmax = reinterpret_cast<int*>(smem + Sm::kOffColmax);
  int* gexp = reinterpret_cast<int*>(smem + Sm::kOffGexp);
  int* misc = reinterpret_cast<int*>(smem + Sm::kOffMisc);
  uint64_t* mbar = reinterpret_cast<uint64_t*>(smem + Sm::kOffBar);
  uint64_t* lbar = reinterpret_cast<uint64_t*>(smem + Sm::kOffBar + 8);

  for (int i = tid; i < NC; i += T) {
    colmax[i] = 0;
    gexp[i] = (XF != kXNone && i < n) ? __ldcg(&a.w.flags[64 + i]) : 0;
  }
  __syncthreads();
  const int g = lane >> 2, t4 = lane & 3;

  // ---- second pass: this warp's 8-column block of Y and the B fragments of M' = diag(2^e_k) M
  const int cbw = (NC == 64 && warp >= 4) ? 11 - warp : warp / WPC;
  const int rpart = (NC == 64) ? 0 : warp % WPC;
  const int ksw = XF == kXUpper ? (cbw >> 1) + 1 : KSTEPS;
  unsigned bq[XF != kXNone ? KSTEPS : 1][7][2];
  float ysc[2][7];  // 2^(f_j - 12 - 7d) for this thread's two Y columns and the 7 weights
  if constexpr (XF != kXNone) {
    const double* M = a.w.keep + (size_t)n * n;  // pass-1 output, row-major, ld n
    const int jb = cbw * 8 + g;
    double mv[KSTEPS][4];
    int F = 0;
#pragma unroll
    for (int ks = 0; ks < KSTEPS; ++ks)
#pragma unroll
      for (int h = 0; h < 4; ++h) {
        const int k = 16 * ks + 2 * t4 + (h & 1) + 8 * (h >> 1);
        double v = 0.0;
        if (k < n && jb < n && (XF != kXUpper || k <= jb)) {
          const int ek = gexp[k];
          if (ek > 0) v = __ldcg(M + (size_t)k * n + jb) * __longlong_as_double((long long)(ek + 1) << 52);
        }
        mv[ks][h] = v;
        F = max(F, (int)((__double_as_longlong(v) >> 52) & 0x7ff));
      }
    F = max(F, __shfl_xor_sync(0xffffffffu, F, 1));
    F = max(F, __shfl_xor_sync(0xffffffffu, F, 2));  // max over column jb of M'
#pragma unroll
    for (int ks = 0; ks < KSTEPS; ++ks) {
      long long Nb[4];
#pragma unroll
      for (int h = 0; h < 4; ++h) Nb[h] = fixed48_of_double(mv[ks][h], F) + kDigitBias;
#pragma unroll
      for (int q = 0; q < 7; ++q) {
        bq[ks][q][0] = bf16x2_of_ints(balanced_digit_rt(Nb[0], q), balanced_digit_rt(Nb[1], q));
        bq[ks][q][1] = bf16x2_of_ints(balanced_digit_rt(Nb[2], q), balanced_digit_rt(Nb[3], q));
      }
    }
    bool bad = false;
#pragma unroll
    for (int h = 0; h < 2; ++h) {
      const int Fj = __shfl_sync(0xffffffffu, F, 4 * (2 * t4 + h));
      const int f = Fj - 1022;  // |M'(:, j)| < 2^f
      if (Fj > 0 && (f < -70 || f > 100)) bad = true;
#pragma unroll
      for (int d = 0; d < 7; ++d) {
        const int e = f - kDigitScaleLog2 - 7 * d;
        ysc[h][d] = (Fj > 0 && !bad) ? __int_as_float((e + 127) << 23) : 0.0f;
      }
    }
    if (__syncthreads_or(bad)) {  // out of the double-float range: the FP64 launches redo it
      if (tid == 0) atomicOr(&a.w.flags[0], 1);
      gram_finish<NC, T, S, ArithDF>(a, smem, colmax, misc, k);
      return;
    }
  }

  // ---- the MMA-completion and tile barriers (the 7 accumulator blocks live at tbase) were
  // initialised once by the kernel (umma_cta_begin): a persistent launch runs this body for
  // many work items, and a barrier that copies and MMA commits have completed phases on is
  // not initialised again; bars carries the parities.  The fence orders the previous item's
  // generic shared-memory writes (its reduction and epilogue) before this item's bulk copies.
  fence_proxy_async_smem();
  tc_fence_before();
  __syncthreads();
  tc_fence_after();

  const int qd = warp & 3, hh = warp >> 2;  // TMEM lane quarter and column part of this warp
  const int L = 32 * qd + lane, kq = L / NC, li = L % NC;
  df acc[HALF];
  // FP64 level of the accumulators: this CTA's [NC columns][128 lanes] block of the
  // workspace (L2-resident; each thread touches only its own entries)
  double* fb = a.w.fbuf + (size_t)bid * NC * 128;
#pragma unroll
  for (int j = 0; j < HALF; ++j) {
    acc[j] = df{0.0f, 0.0f};
    __stcg(fb + (size_t)(hh * HALF + j) * 128 + L, 0.0);
  }

  const int64_t t0 = a.tiles * bid / k, t1 = a.tiles * (bid + 1) / k;
  // a full tile of 16-byte aligned columns arrives by bulk copies (one per column, issued by
  // one thread, completion on lbar); otherwise element by element with zero fill
  auto tile_bulk = [&](int64_t t) { return a.bulk != 0 && (t + 1) * KT <= a.m; };
  auto issue = [&](int64_t t) {
    const int64_t row0 = t * KT;
    if (tile_bulk(t)) {
      if (tid == 32) {  // warp 1: warp 0 issues the MMAs meanwhile
        mbar_arrive_expect_tx(lbar, (uint32_t)(n * KT * sizeof(S)));
        for (int c = 0; c < n; ++c) bulk_g2s(stage + c * LDS, a.src.col(c) + row0, KT * sizeof(S), lbar);
      }
      return;
    }
#pragma unroll 1
    for (int c = 0; c < NC; ++c) {
      const S* col = a.src.col(c < n ? c : 0);
      for (int r = tid; r < KT; r += T) {
        int64_t row = row0 + r;
        bool v = c < n && row < a.m;
        cp_async_elem<S>(stage + c * LDS + r, v ? col + row : col, v);
      }
    }
    cp_async_commit();
  };
  uint32_t& lphase = bars.lphase;
  auto wait_tile = [&](int64_t t) -> bool {  // this thread's view: the staged tile t has landed
    if (!tile_bulk(t)) {
      cp_async_wait_all();
      return true;
    }
    const bool landed = mbar_wait_bounded(lbar, lphase);
    lphase ^= 1u;
    return landed;
  };
  // seven balanced base-128 digits per value into the core-matrix layout: a warp writes one
  // 8 x 8 core matrix (128 contiguous bytes) per step, a lane two rows of one column
  auto put_digits = [&](int c, int r, long long Nb0, long long Nb1) {
    unsigned char* base = digits + (c >> 3) * SBO + (r >> 3) * LBO + (c & 7) * 16 + (r & 7) * 2;
#pragma unroll
    for (int p = 0; p < Sh::ND; ++p)
      *reinterpret_cast<unsigned*>(base + p * PLANE) =
          bf16x2_of_ints(balanced_digit_rt(Nb0, p), balanced_digit_rt(Nb1, p));
  };
  // the staged X, ex[c] the biased double exponent that bounds column c
  auto slice_stage = [&](const int* ex) {
#pragma unroll 4
    for (int k2 = 0; k2 < PAIRS; ++k2) {
      const int cm = warp + NW * k2, c = 8 * (cm / CPG) + (lane >> 2), r = 8 * (cm % CPG) + 2 * (lane & 3);
      const int em = c < n ? ex[c] : 0;  // columns past n are zero (a bulk-loaded stage holds stale data there)
      long long Nb[2];
#pragma unroll
      for (int h = 0; h < 2; ++h) {
        if constexpr (sizeof(S) == 8) {
          Nb[h] = (em > 0 ? fixed48_of_double((double)stage[c * LDS + r + h], em) : 0ll) + kDigitBias;
        } else {
          Nb[h] = (em > 0 ? fixed48_of_float((float)stage[c * LDS + r + h], em - 896) : 0ll) + kDigitBias;
        }
      }
      put_digits(c, r, Nb[0], Nb[1]);
    }
  };

  bool ok = true;
  int fail_where = 0;  // 1: a tile copy never completed, 2: the MMAs never completed
  if (t0 < t1) issue(t0);
  __syncthreads();
  uint32_t& phase = bars.phase;
  for (int64_t t = t0; t < t1; ++t) {
    if (!__syncthreads_and(wait_tile(t))) {  // the copy engine did not deliver: FP64 redoes the call
      ok = false;
      fail_where = 1;
      break;
    }
    for (int i = tid; i < NC; i += T) expo[i] = 0;
    __syncthreads();
    if constexpr (XF == kXNone) {
      // column maxima of the biased double exponent (and the range record)
#pragma unroll 4
      for (int k2 = 0; k2 < PAIRS; ++k2) {
        const int pi = tid + T * k2, c = (2 * pi) / KT, r = (2 * pi) % KT;
        unsigned em = 0;
        if (c < n) {  // warp-uniform: a warp covers 64 rows of one column
          if constexpr (sizeof(S) == 8) {
            unsigned long long b0 = (unsigned long long)__double_as_longlong((double)stage[c * LDS + r]);
            unsigned long long b1 = (unsigned long long)__double_as_longlong((double)stage[c * LDS + r + 1]);
            em = max((unsigned)((b0 >> 52) & 0x7ff), (unsigned)((b1 >> 52) & 0x7ff));
          } else {
            unsigned e0 = (__float_as_uint((float)stage[c * LDS + r]) >> 23) & 0xff;
            unsigned e1 = (__float_as_uint((float)stage[c * LDS + r + 1]) >> 23) & 0xff;
            em = max(e0 ? e0 + 896 : 0u, e1 ? e1 + 896 : 0u);
          }
        }
        em = __reduce_max_sync(0xffffffffu, em);
        if (lane == 0 && em > 0) {
          atomicMax(&expo[c], (int)em);
          atomicMax(&colmax[c], (int)em);
        }
      }
      __syncthreads();
      for (int c = tid; c < NC; c += T) {
        const int em = expo[c];
        pow2c[c] = __int_as_float((max(-126, min(127, em > 0 ? em - 1022 : 0)) + 127) << 23);
      }
      slice_stage(expo);
    } else {
      slice_stage(gexp);
      __syncthreads();
      // Y = X M' (mma.sync): per 16 x 8 block the 28 digit pairs accumulate exactly in FP32
      // per weight, then fold into double-float
      float ymax[2] = {0.0f, 0.0f};
#pragma unroll 1
      for (int i = 0; i < 8; ++i) {
        const int rb = rpart + WPC * i;
        float ac[7][4];
#pragma unroll
        for (int d = 0; d < 7; ++d)
#pragma unroll
          for (int e = 0; e < 4; ++e) ac[d][e] = 0.0f;
#pragma unroll
        for (int ks = 0; ks < KSTEPS; ++ks) {
          if (ks < ksw) {
            unsigned af[7][4];
            // ldmatrix .trans of core matrix (column group 2 ks + K, row group 2 rb + R), row lane & 7
            const unsigned char* ap = digits + (2 * ks + (lane >> 4)) * SBO + (2 * rb + ((lane >> 3) & 1)) * LBO +
                                      (lane & 7) * 16;
#pragma unroll
            for (int p = 0; p < 7; ++p) ldsm_x4_t(af[p][0], af[p][1], af[p][2], af[p][3], ap + p * PLANE);
#pragma unroll
            for (int p = 0; p < 7; ++p)
#pragma unroll
              for (int q = 0; q + p < 7; ++q)
                mma_bf16(ac[p + q], af[p][0], af[p][1], af[p][2], af[p][3], bq[ks][q][0], bq[ks][q][1]);
          }
        }
#pragma unroll
        for (int e = 0; e < 4; ++e) {
          const int h = e & 1;
          float hi = ac[6][e] * ysc[h][6], lo = 0.0f;  // smallest weight first
#pragma unroll
          for (int d = 5; d >= 0; --d) {
            float s, err;
            two_sum(hi, ac[d][e] * ysc[h][d], s, err);
            hi = s;
            lo = __fadd_rn(lo, err);
          }
          const df y = df_make(hi, lo);
          ymax[h] = fmaxf(ymax[h], fabsf(y.hi));
          ydf[(cbw * 8 + 2 * t4 + h) * LDY + 16 * rb + g + 8 * (e >> 1)] = y;
        }
      }
#pragma unroll
      for (int h = 0; h < 2; ++h) {
        float v = ymax[h];
        v = fmaxf(v, __shfl_xor_sync(0xffffffffu, v, 4));
        v = fmaxf(v, __shfl_xor_sync(0xffffffffu, v, 8));
        v = fmaxf(v, __shfl_xor_sync(0xffffffffu, v, 16));
        const int em = (__float_as_int(v) >> 23) & 0xff;
        if (g == 0 && em > 0) atomicMax(&expo[cbw * 8 + 2 * t4 + h], em);
      }
      __syncthreads();
      for (int c = tid; c < NC; c += T) {
        const int em = expo[c];
        pow2c[c] = __int_as_float((max(-126, min(127, em > 0 ? em - 126 : 0)) + 127) << 23);
      }
      // slicing of Y at its per-tile column scale
#pragma unroll 4
      for (int k2 = 0; k2 < PAIRS; ++k2) {
        const int cm = warp + NW * k2, c = 8 * (cm / CPG) + (lane >> 2), r = 8 * (cm % CPG) + 2 * (lane & 3);
        const int em = expo[c];
        long long Nb[2];
#pragma unroll
        for (int h = 0; h < 2; ++h) {
          const df y = ydf[c * LDY + r + h];
          Nb[h] = fixed48_of_float(y.hi, em) + fixed48_of_float(y.lo, em) + kDigitBias;
        }
        put_digits(c, r, Nb[0], Nb[1]);
      }
    }
    fence_proxy_async_smem();  // the digit planes are read by the tensor core
    __syncthreads();
    if (t + 1 < t1) issue(t + 1);
    // 7 accumulator blocks: block tb = p0 + q collects planes p0.. (stacked) times plane q
    if (tid == 0) {
      tc_fence_after();
      // descriptor of plane 0, k-step 0; other planes and k-steps add (byte offset >> 4) to
      // the 14-bit address field, which stays below 2^14 (shared addresses < 256 KB)
      const uint64_t d0 = umma_sdesc(smem_addr(digits), LBO, SBO);
#pragma unroll 1
      for (int kk = 0; kk < KT / 16; ++kk) {
        const uint64_t dk = d0 + (uint64_t)((kk * 2 * LBO) >> 4);
#pragma unroll
        for (int p0 = 0; p0 < 7; p0 += SP)
#pragma unroll
          for (int q = 0; q + p0 < 7; ++q)
            umma_bf16(tbase + (uint32_t)((p0 + q) * NC), dk + (uint64_t)((p0 * PLANE) >> 4),
                      dk + (uint64_t)((q * PLANE) >> 4), IDESC, (kk > 0 || p0 > 0) ? 1u : 0u);
      }
      umma_commit(mbar);
    }
    const bool done = mbar_wait_bounded(mbar, phase);
    phase ^= 1u;
    if (!__syncthreads_and(done)) {  // the tensor core did not finish: let FP64 redo the call
      if (t + 1 < t1) wait_tile(t + 1);  // no copy may still be writing when the CTA moves on
      ok = false;
      fail_where = 2;
      break;
    }
    tc_fence_after();
    // fold the blocks into the double-float accumulators: lane L holds plane offset kq and
    // column li, so block tb carries weight w = tb + kq (0-based; weights above 6 are beyond
    // the truncation).  Per column the seven weights are summed first: blocks 3..6 in FP32
    // (together below 2^-21 of the leading weight), blocks 2, 1, 0 with exact two-sums; the
    // result enters the accumulator with one double-float add.
    {
      const float fi = pow2c[li];
      float sw[7];
      uint32_t vm[7];  // lanes beyond the truncation may hold non-finite products of "plane 7": masked, not scaled
#pragma unroll
      for (int tb = 0; tb < 7; ++tb) {
        sw[tb] = tb + kq <= 6 ? fi * __int_as_float((127 - kDigitScaleLog2 - 7 * (tb + kq)) << 23) : 0.0f;
        vm[tb] = tb + kq <= 6 ? 0xffffffffu : 0u;
      }
      const uint32_t lane_base = tbase + ((uint32_t)(32 * qd) << 16) + (uint32_t)(hh * HALF);
#pragma unroll
      for (int c0 = 0; c0 < HALF; c0 += 4) {
        uint32_t v[7][4];
#pragma unroll
        for (int tb = 0; tb < 7; ++tb) tmem_ld(lane_base + (uint32_t)(tb * NC + c0), v[tb]);
        tmem_ld_wait();
#pragma unroll
        for (int j = 0; j < 4; ++j) {
          float hi = __uint_as_float(v[6][j] & vm[6]) * sw[6];
          hi = __fmaf_rn(__uint_as_float(v[5][j] & vm[5]), sw[5], hi);
          hi = __fmaf_rn(__uint_as_float(v[4][j] & vm[4]), sw[4], hi);
          hi = __fmaf_rn(__uint_as_float(v[3][j] & vm[3]), sw[3], hi);
          float lo = 0.0f;
#pragma unroll
          for (int tb = 2; tb >= 0; --tb) {
            float s2, e2;
            two_sum(hi, __uint_as_float(v[tb][j] & vm[tb]) * sw[tb], s2, e2);
            hi = s2;
            lo = __fadd_rn(lo, e2);
          }
          const float fj = pow2c[hh * HALF + c0 + j];
          acc[c0 + j] = df_add(acc[c0 + j], df{hi * fj, lo * fj});
        }
      }
    }
    if ((t - t0) % kGramFlushTiles == kGramFlushTiles - 1) {  // double-float sums -> FP64 (L2)
#pragma unroll
      for (int j = 0; j < HALF; ++j) {
        double* f = fb + (size_t)(hh * HALF + j) * 128 + L;
        __stcg(f, __ldcg(f) + df_to_double(acc[j]));
        acc[j] = df{0.0f, 0.0f};
      }
    }
    tc_fence_before();
  }
  cp_async_wait_all();  // an early exit may leave a prefetch in flight
  tc_fence_before();
  __syncthreads();
  if (!ok) {  // the FP64 launches redo the call and report {QL_ERR_TIMEOUT, where}
    bars.ok = false;  // a late arrival may still complete a phase: the CTA takes no more work
    if (tid == 0) {
      atomicCAS(&a.w.flags[4], 0, fail_where);
      atomicOr(&a.w.flags[0], 2);
    }
  }
  if constexpr (XF == kXNone) {  // column exponents of the whole matrix, for the second pass
    for (int c = tid; c < n; c += T)
      if (colmax[c] > 0) atomicMax(&a.w.flags[64 + c], colmax[c]);
  }
  // combine the plane offsets of each entry (FP64) and store this CTA's partial Gram matrix
  double* red = reinterpret_cast<double*>(smem + Sm::kOffStage);  // [lane L][column]
#pragma unroll
  for (int j = 0; j < HALF; ++j)
    red[L * NC + hh * HALF + j] = __ldcg(fb + (size_t)(hh * HALF + j) * 128 + L) + df_to_double(acc[j]);
  __syncthreads();
  double* part = a.w.partials + (size_t)bid * NC * NC;
  for (int e = tid; e < NC * NC; e += T) {
    const int i = e / NC, j = e % NC;
    double s = 0.0;
#pragma unroll
    for (int kk = 0; kk < SP; ++kk) s += red[(kk * NC + i) * NC + j];
    __stcg(part + e, s);
  }
  gram_finish<NC, T, S, ArithDF>(a, smem, colmax, misc, k);
}

template <int NC, typename S, int XF>
__global__ void __launch_bounds__(umma_threads<XF>(), 1) gram_umma_kernel(GramArgs<S> a) {
  using Sh = UmmaShape<NC>;
  using Sm = UmmaSmem<NC, S>;
  extern __shared__ __align__(1024) unsigned char smem_umma[];
  unsigned char* smem = smem_umma;
  uint32_t* tslot = reinterpret_cast<uint32_t*>(smem + Sm::kOffBar + 16);
  const uint32_t tbase = umma_cta_begin<NC, S>(smem, tslot);
  UmmaBars bars;
  gram_umma_body<NC, S, XF>(a, blockIdx.x, gridDim.x, tbase, bars);
  tc_fence_before();
  __syncthreads();
  if ((threadIdx.x >> 5) == 0) tmem_dealloc(tbase, Sh::TCOLS);
}

template <int NC, typename S, int XF>
ql_status gram_umma_launch_one(const GramCall& c, const GramWs& w, int pass) {
  using Sh = UmmaShape<NC>;
  using Sm = UmmaSmem<NC, S>;
  auto kern = gram_umma_kernel<NC, S, XF>;
  static bool ready = false;
  static std::mutex mu;
  {
    std::lock_guard<std::mutex> lk(mu);
    if (!ready) {
      if (cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)Sm::kBytes) != cudaSuccess)
        return QL_ERR_CUDA;
      ready = true;
    }
  }
  // one CTA per SM: the shared memory allows no second one, and tensor memory is sized so
  const int64_t tiles = (c.m + Sh::KT - 1) / Sh::KT;
  int64_t g = (int64_t)device_sm_count();
  if (g > tiles) g = tiles;
  if (g < 1) g = 1;
  GramArgs<S> a{};
  a.src.A = static_cast<const S*>(c.A);
  a.src.lda = c.lda;
  a.src.b = static_cast<const S*>(c.b);
  a.src.nA = c.nA;
  a.m = c.m;
  a.n = c.n;
  a.tiles = tiles;
  a.pass = pass;
  a.method = c.method;
  a.gated = 0;
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
  {
    auto aligned = [](const void* p) { return (reinterpret_cast<uintptr_t>(p) & 15u) == 0; };
    bool b = aligned(c.A) && ((size_t)c.lda * sizeof(S)) % 16 == 0;
    if (c.nA < c.n) b = b && aligned(c.b);
    a.bulk = b ? 1 : 0;
  }
  a.mround = 2;
  count_launch();
  kern<<<(int)g, umma_threads<XF>(), Sm::kBytes, c.stream>>>(a);
  return cudaPeekAtLastError() == cudaSuccess ? QL_OK : QL_ERR_CUDA;
}

// ---------------------------------------------------------------------------------------
// Pipelined first Gram pass on tcgen05 (see gram_pipe.cuh).  The body handles the row tiles
// [tiles bid / k, tiles (bid + 1) / k) of one problem as partial `bid` of `k`, with the
// tensor memory at tbase and the barriers that pipe_cta_begin set up; bars carries their
// phase counts from one work item to the next.
// The seven planes of the 48-bit convention (operands of Y = X M'), 8 rows per 16-byte store.
template <int PLANE, int P = 0>
QL_DEV void put_planes7(unsigned char* base, const unsigned long long (&Nb)[8]) {
  uint4 w;
  w.x = digit_word7<P>(Nb[0], Nb[1]);
  w.y = digit_word7<P>(Nb[2], Nb[3]);
  w.z = digit_word7<P>(Nb[4], Nb[5]);
  w.w = digit_word7<P>(Nb[6], Nb[7]);
  *reinterpret_cast<uint4*>(base + P * PLANE) = w;
  if constexpr (P + 1 < 7) put_planes7<PLANE, P + 1>(base, Nb);
}

template <int NC, int PLANE, int P = 0>
QL_DEV void put_planes8(unsigned char* base, const unsigned long long (&Nb)[8]) {
  uint4 w;
  w.x = digit_word<P>(Nb[0], Nb[1]);
  w.y = digit_word<P>(Nb[2], Nb[3]);
  w.z = digit_word<P>(Nb[4], Nb[5]);
  w.w = digit_word<P>(Nb[6], Nb[7]);
  *reinterpret_cast<uint4*>(base + P * PLANE) = w;
  if constexpr (P + 1 < 8) put_planes8<NC, PLANE, P + 1>(base, Nb);
}

// Digits P.. of one element (biased fixed point Nb, see biased_fixed56) into their planes,
// one 2-byte store per plane.
template <int PLANE, int P = 0>
QL_DEV void put_digits8_one(unsigned char* p0, unsigned long long Nb) {
  *reinterpret_cast<unsigned short*>(p0 + P * PLANE) = (unsigned short)(digit_word<P>(Nb, Nb) & 0xffffu);
  if constexpr (P + 1 < 8) put_digits8_one<PLANE, P + 1>(p0, Nb);
}

// XF = kXNone: the first pass (C = X^T X).  XF = kXUpper / kXFull (n <= 32): a later pass of
// Cholesky-QR2 / shifted Cholesky-QR3 (M = R1^{-1}, upper triangular) or SVQB2 (M = B1):
// C = Y^T Y with Y = X M formed tile by tile and never stored.  The slicer warps then cut X
// into seven digits at the whole matrix's column scale (the first pass recorded it), form
// Y = X M' (M' = diag(2^e_k) M) on mma.sync from those digits and the M' digits (B
// fragments in shared memory), fold the seven weights of each element into a double-float
// and cut Y into the eight digits of the Gram, as the first pass cuts X; the control warp,
// the copies and the tensor-memory sums are the first pass's.
template <int NC, typename S, int XF = kXNone>
QL_DEV void gram_pipe_body(GramArgs<S> a, int bid, int k, uint32_t tbase, PipeBars& bars, const CUtensorMap* tmA,
                           const CUtensorMap* tmB) {
  using Sh = PipeShape<NC>;
  using Sm = PipeSmem<NC, S, XF>;
  static_assert(XF == kXNone || NC <= 32, "later passes: the M' fragments of n <= 32 columns");
  constexpr int T = Sh::T, TS = Sh::TS, UPT = Sh::UPT, KT = Sh::KT, SP = Sh::SP, PLANE = Sh::PLANE,
                SBO = Sh::SBO, LBO = Sh::LBO, HALF = Sh::HALF, G = Sh::G, RPB = Sm::RPB, NBOX = Sm::NBOX;
  constexpr uint32_t IDESC = umma_idesc_bf16(128, 128);
  extern __shared__ __align__(1024) unsigned char smem_umma[];
  unsigned char* smem = smem_umma;
  const int tid = threadIdx.x, n = a.n, lane = tid & 31, warp = tid >> 5;
  const bool control = warp == TS / 32;

  unsigned char* dig0 = smem + Sm::kOffDig;
  unsigned char* raw0 = smem + Sm::kOffRaw;  // 2 staged tiles of kRaw bytes
  float* pow2c = reinterpret_cast<float*>(smem + Sm::kOffPow);
  int* scale = reinterpret_cast<int*>(smem + Sm::kOffScale);  // running scale exponents (biased)
  int* colmax = reinterpret_cast<int*>(smem + Sm::kOffColmax);
  int* misc = reinterpret_cast<int*>(smem + Sm::kOffMisc);
  uint64_t* mbar = reinterpret_cast<uint64_t*>(smem + Sm::kOffBar);  // [2] MMAs done, per digit buffer
  uint64_t* lbar = mbar + 2;                                          // [2] tile landed, per raw stage
  uint64_t* dbar = mbar + 4;                                          // [2] digits ready, per digit buffer
  uint64_t* rbar = mbar + 6;                                          // [2] stage read, per raw stage
  int* ngrp = reinterpret_cast<int*>(smem + Sm::kOffSlot + 4);        // [2] tile opens a new group
  int* sfail = ngrp + 2;                                              // [2] where each role gave up

  a.tiles = (a.m + KT - 1) / KT;  // in this kernel's tile height
  for (int i = tid; i < NC; i += T) {
    colmax[i] = 0;
    scale[i] = 0;
    pow2c[i] = 0.0f;
  }
  if (tid < 2) sfail[tid] = 0;
  bool skip_tiles = false;
  if constexpr (XF != kXNone) {
    int* gexp = reinterpret_cast<int*>(smem + Sm::kOffGexp);  // X's column exponents (whole matrix)
    int* fexp = reinterpret_cast<int*>(smem + Sm::kOffFexp);  // M''s column exponents
    int* entry = reinterpret_cast<int*>(smem + Sm::kOffEntry);
    uint2* bqs = reinterpret_cast<uint2*>(smem + Sm::kOffBq);
    // the entry conditions of every later pass, decided once for the whole CTA
    if (tid == 0) {
      int e = 0;
      if (*(volatile int*)&a.w.flags[0] != 0) e = 1;       // the FP64 launches redo the call
      else if (*(volatile int*)&a.w.flags[1] != 0) e = 2;  // the first pass broke down
      entry[0] = e;
    }
    __syncthreads();
    const int e0 = entry[0];
    if (e0 == 2 && bid == 0) write_nan_outputs(a, T);
    if (e0 != 0) return;
    for (int i = tid; i < NC; i += T) gexp[i] = i < n ? __ldcg(&a.w.flags[64 + i]) : 0;
    __syncthreads();
    const double* M = a.w.keep + (size_t)n * n;  // the previous pass's M (row-major, ld n)
    auto mprime = [&](int kk, int j) -> double {  // M'(kk, j), zero outside the used part
      if (kk >= n || j >= n || (XF == kXUpper && kk > j)) return 0.0;
      const int ek = gexp[kk];
      return ek > 0 ? __ldcg(M + (size_t)kk * n + j) * __longlong_as_double((long long)(ek + 1) << 52) : 0.0;
    };
    for (int j = tid; j < NC; j += T) {
      int F = 0;
      for (int kk = 0; kk < NC; ++kk) F = max(F, (int)((__double_as_longlong(mprime(kk, j)) >> 52) & 0x7ff));
      fexp[j] = F;
    }
    __syncthreads();
    bool bad = false;  // the fold scales of Y must stay normal floats
    for (int j = tid; j < NC; j += T) {
      const int F = fexp[j], f = F - 1022;
      if (F > 0 && (f < -70 || f > 100)) bad = true;
    }
    if (__syncthreads_or(bad)) {  // out of the double-float range: the FP64 launches redo it
      if (tid == 0) atomicOr(&a.w.flags[0], 1);
      skip_tiles = true;
    }
    // B fragments of M' for mma m16n8k16: lane (g, t4) of 8-column block cb holds rows
    // k = 16 ks + 2 t4 + {0, 1} (first word) and k + 8 (second word) of column 8 cb + g,
    // seven balanced digits of the 48-bit fixed point relative to that column's exponent
    constexpr int NCB = Sm::NCB, KSTEPS = Sm::KSTEPS;
    for (int it = tid; it < NCB * KSTEPS * 32; it += T) {
      const int ln = it & 31, ks = (it >> 5) % KSTEPS, cb = (it >> 5) / KSTEPS;
      const int j = cb * 8 + (ln >> 2), t4 = ln & 3, F = fexp[j];
      long long Nb[4];
#pragma unroll
      for (int h = 0; h < 4; ++h) {
        const int kk = 16 * ks + 2 * t4 + (h & 1) + 8 * (h >> 1);
        Nb[h] = (F > 0 ? fixed48_of_double(mprime(kk, j), F) : 0ll) + kDigitBias;
      }
#pragma unroll
      for (int q = 0; q < 7; ++q)
        bqs[((cb * KSTEPS + ks) * 7 + q) * 32 + ln] =
            make_uint2(bf16x2_of_ints(balanced_digit_rt(Nb[0], q), balanced_digit_rt(Nb[1], q)),
                       bf16x2_of_ints(balanced_digit_rt(Nb[2], q), balanced_digit_rt(Nb[3], q)));
    }
  }
  // the previous work item's generic writes (its reduction and epilogue) come before this
  // item's bulk copies and MMA operand reads
  fence_proxy_async_smem();
  tc_fence_before();
  __syncthreads();
  tc_fence_after();

  const int64_t t0 = a.tiles * bid / k, t1 = skip_tiles ? t0 : a.tiles * (bid + 1) / k;
  // with 16-byte aligned columns every tile arrives by tensor copies (rows past m read as
  // zeros); otherwise the slicers read X from global memory themselves
  auto tile_bulk = [&](int64_t) { return a.bulk != 0; };

  // this slicer's units of a tile: unit u = tid + TS uu covers rows r0..r0+7 of column c
  // (8 consecutive threads hold 8 consecutive columns, so their digit stores fill whole
  // core-matrix rows)
  int c_[UPT], r0_[UPT];
  bool live_[UPT];
#pragma unroll
  for (int uu = 0; uu < UPT; ++uu) {
    const int u = (tid & (TS - 1)) + TS * uu, u8 = u >> 3, rg = u8 % (KT / 8), cg = u8 / (KT / 8);
    c_[uu] = 8 * cg + (u & 7);
    r0_[uu] = 8 * rg;
    live_[uu] = c_[uu] < n && !control;
  }
  // read-out role: TMEM lane quarter qd, column part hh; lane L is plane offset kq, column li
  const int qd = warp & 3, hh = (warp >> 2) % (TS / 128);
  const int L = 32 * qd + lane, kq = L / NC, li = L % NC;
  // accumulators of this CTA's [NC columns][128 lanes] entries, in an L2-resident workspace
  // block: the FP64 level, then the double-float sums (each slicer touches only its own)
  double* fb = a.w.fbuf + (size_t)bid * NC * 128 * 2;
  float2* fd = reinterpret_cast<float2*>(fb + (size_t)NC * 128);
  int erun[UPT];  // largest exponent each unit's column has shown this slicer (range record)
#pragma unroll
  for (int uu = 0; uu < UPT; ++uu) erun[uu] = 0;

  if (control) {
    // ---- control warp: copies two tiles ahead, then per tile: once the slicers have read
    // its stage, copy the tile two ahead into it; once its digits are ready, issue the MMAs
    // and commit them
    bool ok = true;
    uint32_t pend = 0u, ppar = 0u;  // bit b: a copy into stage b in flight, and its phase parity
    auto copy = [&](int64_t t, int b) {
      if (!tile_bulk(t)) return;
      unsigned char* stage = raw0 + (size_t)b * Sm::kRaw;
      const int row0 = (int)(t * KT);
      if (lane == 0) {
        mbar_arrive_expect_tx(&lbar[b], (uint32_t)(NBOX * n * 128));
#pragma unroll 1
        for (int kb = 0; kb < NBOX; ++kb) {
          tma_load_2d(stage + (size_t)kb * NC * 128, tmA, row0 + kb * RPB, 0, &lbar[b]);
          if (tmB) tma_load_2d(stage + (size_t)(kb * NC + a.src.nA) * 128, tmB, row0 + kb * RPB, 0, &lbar[b]);
        }
      }
      __syncwarp();
      pend |= 1u << b;
      ppar = (ppar & ~(1u << b)) | (bars.lpar & (1u << b));
      bars.lpar ^= 1u << b;
    };
    if (t0 < t1) copy(t0, 0);
    if (t0 + 1 < t1) copy(t0 + 1, 1);
    for (int64_t t = t0; t < t1; ++t) {
      const int b = (int)((t - t0) & 1);
      if (!__all_sync(0xffffffffu, mbar_wait_bounded(&rbar[b], (bars.mpar >> b) & 1u))) {
        ok = false;
        break;
      }
      pend &= ~(1u << b);  // the slicers have read stage b
      if (t + 2 < t1) copy(t + 2, b);
      if (!__all_sync(0xffffffffu, mbar_wait_bounded(&dbar[b], (bars.mpar >> b) & 1u))) {
        ok = false;
        break;
      }
      bars.mpar ^= 1u << b;
      tc_fence_after();
      if (lane == 0) {
        const uint32_t fresh = (uint32_t)ngrp[b];
        // descriptor of plane 0, k-step 0; other planes and k-steps add (byte offset >> 4)
        // to the 14-bit address field, which stays below 2^14 (shared addresses < 256 KB)
        const uint64_t d0 = umma_sdesc(smem_addr(dig0 + (size_t)b * Sh::DBUF), LBO, SBO);
#pragma unroll 1
        for (int kk = 0; kk < KT / 16; ++kk) {
          const uint64_t dk = d0 + (uint64_t)((kk * 2 * LBO) >> 4);
#pragma unroll
          for (int p0 = 0; p0 < 8; p0 += SP)
#pragma unroll
            for (int q0 = 0; q0 < 8; q0 += SP)
              if (p0 + q0 <= 7)
                umma_bf16(tbase + (uint32_t)((p0 + q0) * NC), dk + (uint64_t)((p0 * PLANE) >> 4),
                          dk + (uint64_t)((q0 * PLANE) >> 4), IDESC, (!fresh || kk > 0 || p0 > 0) ? 1u : 0u);
        }
        umma_commit(&mbar[b]);
      }
      __syncwarp();
    }
    // no copy may still be writing when the CTA moves on
    for (int b = 0; b < 2; ++b)
      if (pend & (1u << b)) mbar_wait_bounded(&lbar[b], (ppar >> b) & 1u);
    if (!ok && lane == 0) sfail[1] = 2;
  } else {
    // ---- slicer warps
    bool ok = true;
    int fail_where = 0;   // 1: a tile copy never completed, 2: the MMAs never completed
    int grp = 0;          // tiles summed in tensor memory since the last read-out
    int nread = 0;        // read-outs since the last move into FP64
    int last_b = 0;       // digit buffer of the latest tile handed to the MMAs
    uint32_t cpar = 0u;   // bit b: phase parity of the MMAs of the latest tile on buffer b
#pragma unroll
    for (int j = 0; j < HALF; ++j) {
      __stcg(fb + (size_t)(hh * HALF + j) * 128 + L, 0.0);
      __stcg(fd + (size_t)(hh * HALF + j) * 128 + L, make_float2(0.0f, 0.0f));
    }

    // fold the eight accumulator combinations into the double-float sums: combination tb of
    // this lane sits at column tb NC + j and weighs tb + kq (above 7: beyond the truncation,
    // masked).  Every block value is an exact integer and every product with its
    // power-of-two weight is exact; the weights are summed with exact two-sums.
    auto readout = [&]() {
      const float fi = pow2c[li];
      float sw[8];
      uint32_t vm[8];
#pragma unroll
      for (int tb = 0; tb < 8; ++tb) {
        const int w = tb + kq;
        sw[tb] = w <= 7 ? fi * __int_as_float((127 - kDigitScaleLog2 - 7 * w) << 23) : 0.0f;
        vm[tb] = w <= 7 ? 0xffffffffu : 0u;
      }
      const uint32_t lane_base = tbase + ((uint32_t)(32 * qd) << 16) + (uint32_t)(hh * HALF);
#pragma unroll 1
      for (int c0 = 0; c0 < HALF; c0 += 4) {
        uint32_t v[8][4];
#pragma unroll
        for (int tb = 0; tb < 8; ++tb) tmem_ld(lane_base + (uint32_t)(tb * NC + c0), v[tb]);
        float2 old[4];
#pragma unroll
        for (int j = 0; j < 4; ++j) old[j] = __ldcg(fd + (size_t)(hh * HALF + c0 + j) * 128 + L);
        tmem_ld_wait();
#pragma unroll
        for (int j = 0; j < 4; ++j) {
          float hi = __uint_as_float(v[7][j] & vm[7]) * sw[7], lo = 0.0f;
#pragma unroll
          for (int tb = 6; tb >= 0; --tb) {
            float s2, e2;
            two_sum(hi, __uint_as_float(v[tb][j] & vm[tb]) * sw[tb], s2, e2);
            hi = s2;
            lo = __fadd_rn(lo, e2);
          }
          const float fj = pow2c[hh * HALF + c0 + j];
          const df sum = df_add(df{old[j].x, old[j].y}, df{hi * fj, lo * fj});
          __stcg(fd + (size_t)(hh * HALF + c0 + j) * 128 + L, make_float2(sum.hi, sum.lo));
        }
      }
    };

    for (int64_t t = t0; t < t1; ++t) {
      const int i = (int)(t - t0), b = i & 1;
      unsigned char* dig = dig0 + (size_t)b * Sh::DBUF;
      const bool bulk = tile_bulk(t);
      bool landed = true;
      if (bulk) {
        landed = mbar_wait_bounded(&lbar[b], (bars.lpar >> b) & 1u);
        bars.lpar ^= 1u << b;
      }
      if (!slicer_and<TS>(landed)) {  // the copy engine did not deliver: FP64 redoes the call
        ok = false;
        fail_where = 1;
        break;
      }
      if constexpr (XF == kXNone) {
        S v[UPT][8];
        int e[UPT];
        bool over = false;
  #pragma unroll
        for (int uu = 0; uu < UPT; ++uu) {
          e[uu] = 0;
          if (live_[uu]) {
            if (bulk) {
              load8_swz<NC, S>(v[uu], raw0 + (size_t)b * Sm::kRaw, c_[uu], r0_[uu],
                               c_[uu] == a.src.nA ? 0 : (c_[uu] & 7));
            } else {
              const S* col = a.src.col(c_[uu]);
              const int64_t row0 = t * KT + r0_[uu];
  #pragma unroll
              for (int j = 0; j < 8; ++j) v[uu][j] = row0 + j < a.m ? __ldg(col + row0 + j) : S(0);
            }
  #pragma unroll
            for (int j = 0; j < 8; ++j) e[uu] = max(e[uu], elem_exponent(v[uu][j]));
            erun[uu] = max(erun[uu], e[uu]);
            over = over || e[uu] > scale[c_[uu]];
          } else {
  #pragma unroll
            for (int j = 0; j < 8; ++j) v[uu][j] = S(0);
          }
        }
        // stage b is read: the control warp may copy the tile two ahead into it
        fence_proxy_async_smem();
        __syncwarp();
        if (lane == 0) mbar_arrive(&rbar[b]);
        // digit buffer b is free once the MMAs of tile t - 2 are done; a column whose tile
        // maximum exceeds its scale, or a full group, needs a read-out first (rare)
        const bool okw = i >= 2 ? mbar_wait_bounded(&mbar[b], (cpar >> b) & 1u) : true;
        const bool full = grp >= G;
        if (slicer_or<TS>(over || !okw) || full) {
          if (!slicer_and<TS>(okw)) {  // the tensor core did not finish: FP64 redoes the call
            ok = false;
            fail_where = 2;
            break;
          }
          const bool anyover = slicer_or<TS>(over);
          if ((anyover || full) && grp > 0) {  // read the sums out before their scale changes or they could round
            if (!slicer_and<TS>(mbar_wait_bounded(&mbar[last_b], (cpar >> last_b) & 1u))) {
              ok = false;
              fail_where = 2;
              break;
            }
            tc_fence_after();
            readout();
            grp = 0;
            if (++nread == Sh::DF_FLUSH) {  // double-float sums -> FP64
  #pragma unroll 4
              for (int j = 0; j < HALF; ++j) {
                double* f = fb + (size_t)(hh * HALF + j) * 128 + L;
                float2* g = fd + (size_t)(hh * HALF + j) * 128 + L;
                const float2 d2 = __ldcg(g);
                __stcg(f, __ldcg(f) + df_to_double(df{d2.x, d2.y}));
                __stcg(g, make_float2(0.0f, 0.0f));
              }
              nread = 0;
            }
            slicer_sync<TS>();  // every read of the blocks and of the old scales is done
          }
  #pragma unroll
          for (int uu = 0; uu < UPT; ++uu)
            if (live_[uu] && e[uu] > scale[c_[uu]]) atomicMax(&scale[c_[uu]], e[uu] + Sh::SLACK);
          slicer_sync<TS>();
          for (int cc = tid; cc < NC; cc += TS) {
            const int s = scale[cc];
            pow2c[cc] = s > 0 ? __int_as_float(max(1, min(254, s - 895)) << 23) : 0.0f;  // 2^(s - 1022)
          }
        }
        // eight digits of every element into the core-matrix layout of buffer b
  #pragma unroll
        for (int uu = 0; uu < UPT; ++uu) {
          const int cu = c_[uu], Es = live_[uu] ? scale[cu] : 0;
          unsigned long long Nb[8];
  #pragma unroll
          for (int j = 0; j < 8; ++j) Nb[j] = biased_fixed56<S>(v[uu][j], Es);  // dead columns hold zeros
          put_planes8<NC, PLANE>(dig + (cu >> 3) * SBO + (r0_[uu] >> 3) * LBO + (cu & 7) * 16, Nb);
        }
        if (tid == 0) ngrp[b] = grp == 0 ? 1 : 0;
        fence_proxy_async_smem();  // the digit planes are read by the tensor core
        tc_fence_before();         // the read-out's TMEM loads come before the next MMAs
        __syncwarp();
        if (lane == 0) mbar_arrive(&dbar[b]);
        cpar = (cpar & ~(1u << b)) | (bars.mpar & (1u << b));
        bars.mpar ^= 1u << b;
        last_b = b;
        ++grp;
      } else {
        // ---- later pass: Y = X M' for this tile, then Y's digits
        const int* gexp = reinterpret_cast<const int*>(smem + Sm::kOffGexp);
        const int* fexp = reinterpret_cast<const int*>(smem + Sm::kOffFexp);
        const uint2* bqs = reinterpret_cast<const uint2*>(smem + Sm::kOffBq);
        constexpr int NCB = Sm::NCB, KSTEPS = Sm::KSTEPS;
        static_assert(NCB * (KT / 16) == 2 * (TS / 32), "two 16 x 8 blocks of Y per slicer warp");
        // buffer b takes X's digits first: the MMAs of tile t - 2 must be done with it
        const bool okw = i >= 2 ? mbar_wait_bounded(&mbar[b], (cpar >> b) & 1u) : true;
        if (!slicer_and<TS>(okw)) {  // the tensor core did not finish: FP64 redoes the call
          ok = false;
          fail_where = 2;
          break;
        }
        // seven balanced digits of X at the whole matrix's column scale, 8 rows of one
        // column per unit (the core-matrix layout of the Gram digits)
#pragma unroll
        for (int uu = 0; uu < UPT; ++uu) {
          const int cu = c_[uu], em = live_[uu] ? gexp[cu] : 0;
          S xv[8];
          if (live_[uu]) {
            if (bulk) {
              load8_swz<NC, S>(xv, raw0 + (size_t)b * Sm::kRaw, cu, r0_[uu], cu == a.src.nA ? 0 : (cu & 7));
            } else {
              const S* col = a.src.col(cu);
              const int64_t row0 = t * KT + r0_[uu];
#pragma unroll
              for (int j = 0; j < 8; ++j) xv[j] = row0 + j < a.m ? __ldg(col + row0 + j) : S(0);
            }
          } else {
#pragma unroll
            for (int j = 0; j < 8; ++j) xv[j] = S(0);
          }
          unsigned long long Nb[8];  // N + kDigitBias + kDigitTop7 >= 0 (see digit_word7)
#pragma unroll
          for (int j = 0; j < 8; ++j) {
            long long N;
            if constexpr (sizeof(S) == 8) {
              N = em > 0 ? fixed48_of_double((double)xv[j], em) : 0ll;
            } else {
              N = em > 0 ? fixed48_of_float((float)xv[j], em - 896) : 0ll;
            }
            Nb[j] = (unsigned long long)(N + kDigitBias) + kDigitTop7;
          }
          put_planes7<PLANE>(dig + (cu >> 3) * SBO + (r0_[uu] >> 3) * LBO + (cu & 7) * 16, Nb);
        }
        // stage b is read: the control warp may copy the tile two ahead into it
        fence_proxy_async_smem();
        __syncwarp();
        if (lane == 0) mbar_arrive(&rbar[b]);
        slicer_sync<TS>();  // X's digits are in place
        // Y = X M' on mma.sync: this warp's 8-column block cb and two 16-row blocks; per
        // block the 28 digit pairs (p + q <= 6) accumulate exactly in FP32 per weight
        const int g = lane >> 2, t4 = lane & 3, cb = warp % NCB;
        const int ksw = XF == kXUpper ? (cb >> 1) + 1 : KSTEPS;  // M' upper triangular: k <= j
        df y[2][4];
#pragma unroll
        for (int bi = 0; bi < 2; ++bi) {
          const int rb = warp / NCB + bi * (16 / NCB);
          float ac[7][4];
#pragma unroll
          for (int d = 0; d < 7; ++d)
#pragma unroll
            for (int e = 0; e < 4; ++e) ac[d][e] = 0.0f;
#pragma unroll
          for (int ks = 0; ks < KSTEPS; ++ks) {
            if (ks < ksw) {
              uint2 bw[7];
#pragma unroll
              for (int q = 0; q < 7; ++q) bw[q] = bqs[((cb * KSTEPS + ks) * 7 + q) * 32 + lane];
              // ldmatrix .trans of core matrix (column group 2 ks + K, row group 2 rb + R)
              const unsigned char* ap =
                  dig + (2 * ks + (lane >> 4)) * SBO + (2 * rb + ((lane >> 3) & 1)) * LBO + (lane & 7) * 16;
#pragma unroll
              for (int p = 0; p < 7; ++p) {
                unsigned a0, a1, a2, a3;
                ldsm_x4_t(a0, a1, a2, a3, ap + p * PLANE);
#pragma unroll
                for (int q = 0; q + p < 7; ++q) mma_bf16(ac[p + q], a0, a1, a2, a3, bw[q].x, bw[q].y);
              }
            }
          }
          // fold the seven weights (smallest first) into one double-float per element;
          // weight d of column j weighs 2^(f_j - 12 - 7 d), f_j = fexp[j] - 1022
#pragma unroll
          for (int e = 0; e < 4; ++e) {
            const int F = fexp[cb * 8 + 2 * t4 + (e & 1)], f = F - 1022;
            float hi = ac[6][e] * __int_as_float((f - kDigitScaleLog2 - 42 + 127) << 23), lo = 0.0f;
#pragma unroll
            for (int d = 5; d >= 0; --d) {
              float s2, e2;
              two_sum(hi, ac[d][e] * __int_as_float((f - kDigitScaleLog2 - 7 * d + 127) << 23), s2, e2);
              hi = s2;
              lo = __fadd_rn(lo, e2);
            }
            y[bi][e] = F > 0 ? df_make(hi, lo) : df{0.0f, 0.0f};
          }
        }
        slicer_sync<TS>();  // every read of X's digits is done: buffer b takes Y's digits next
        // Y against the running column scales (this lane holds columns c0 and c0 + 1); the
        // exponent of the high part bounds the double-float's (no FP64 instruction here: the
        // FP64 pipe runs at 1/64 of the FP32 rate)
        const int c0 = cb * 8 + 2 * t4;
        int ey[2] = {0, 0};
#pragma unroll
        for (int bi = 0; bi < 2; ++bi)
#pragma unroll
          for (int e = 0; e < 4; ++e) ey[e & 1] = max(ey[e & 1], elem_exponent(y[bi][e].hi));
        const bool over = ey[0] > scale[c0] || ey[1] > scale[c0 + 1];
        const bool full = grp >= G;
        if (slicer_or<TS>(over) || full) {
          if (grp > 0) {  // read the sums out before their scale changes or they could round
            if (!slicer_and<TS>(mbar_wait_bounded(&mbar[last_b], (cpar >> last_b) & 1u))) {
              ok = false;
              fail_where = 2;
              break;
            }
            tc_fence_after();
            readout();
            grp = 0;
            if (++nread == Sh::DF_FLUSH) {  // double-float sums -> FP64
#pragma unroll 4
              for (int j = 0; j < HALF; ++j) {
                double* f = fb + (size_t)(hh * HALF + j) * 128 + L;
                float2* gd = fd + (size_t)(hh * HALF + j) * 128 + L;
                const float2 d2 = __ldcg(gd);
                __stcg(f, __ldcg(f) + df_to_double(df{d2.x, d2.y}));
                __stcg(gd, make_float2(0.0f, 0.0f));
              }
              nread = 0;
            }
            slicer_sync<TS>();  // every read of the blocks and of the old scales is done
          }
#pragma unroll
          for (int h = 0; h < 2; ++h)
            if (ey[h] > scale[c0 + h]) atomicMax(&scale[c0 + h], ey[h] + Sh::SLACK);
          slicer_sync<TS>();
          for (int cc = tid; cc < NC; cc += TS) {
            const int sc = scale[cc];
            pow2c[cc] = sc > 0 ? __int_as_float(max(1, min(254, sc - 895)) << 23) : 0.0f;  // 2^(s - 1022)
          }
        }
        // eight digits of every Y element into buffer b (rows g, g + 8 of each 16-row block)
#pragma unroll
        for (int bi = 0; bi < 2; ++bi) {
          const int rb = warp / NCB + bi * (16 / NCB);
#pragma unroll
          for (int e = 0; e < 4; ++e) {
            const int c = c0 + (e & 1), r = 16 * rb + g + 8 * (e >> 1);
            // fixed point of hi + lo: the two parts rounded separately (hi is exact unless the
            // element lies 2^32 below its column's scale), one bias removed
            const unsigned long long Nb = biased_fixed56<float>(y[bi][e].hi, scale[c]) +
                                          biased_fixed56<float>(y[bi][e].lo, scale[c]) - kDigitBias8;
            put_digits8_one<PLANE>(dig + (c >> 3) * SBO + (r >> 3) * LBO + (c & 7) * 16 + (r & 7) * 2, Nb);
          }
        }
        if (tid == 0) ngrp[b] = grp == 0 ? 1 : 0;
        fence_proxy_async_smem();  // the digit planes are read by the tensor core
        tc_fence_before();         // the read-out's TMEM loads come before the next MMAs
        __syncwarp();
        if (lane == 0) mbar_arrive(&dbar[b]);
        cpar = (cpar & ~(1u << b)) | (bars.mpar & (1u << b));
        bars.mpar ^= 1u << b;
        last_b = b;
        ++grp;
      }
    }
    if (ok && grp > 0) {  // the last group
      if (!slicer_and<TS>(mbar_wait_bounded(&mbar[last_b], (cpar >> last_b) & 1u))) {
        ok = false;
        fail_where = 2;
      } else {
        tc_fence_after();
        readout();
      }
    }
    if (!ok && tid == 0) sfail[0] = fail_where;
#pragma unroll
    for (int uu = 0; uu < UPT; ++uu)
      if (live_[uu] && erun[uu] > 0) atomicMax(&colmax[c_[uu]], erun[uu]);
  }
  tc_fence_before();
  __syncthreads();
  const int fw = sfail[0] ? sfail[0] : sfail[1];
  if (fw) {
    bars.ok = false;  // a late arrival may still complete a phase: the CTA takes no more work
    if (tid == 0) {   // the FP64 launches redo the call and report {QL_ERR_TIMEOUT, where}
      atomicCAS(&a.w.flags[4], 0, fw);
      atomicOr(&a.w.flags[0], 2);
    }
  }
  for (int cc = tid; cc < n; cc += T)  // column exponents of the whole matrix, for the second pass
    if (colmax[cc] > 0) atomicMax(&a.w.flags[64 + cc], colmax[cc]);
  // combine the plane offsets of each entry (FP64) and store this CTA's partial Gram matrix
  double* red = reinterpret_cast<double*>(smem + Sm::kOffDig);  // [lane L][column]
  if (!control) {
#pragma unroll 4
    for (int j = 0; j < HALF; ++j) {
      const float2 d2 = __ldcg(fd + (size_t)(hh * HALF + j) * 128 + L);
      red[L * NC + hh * HALF + j] = __ldcg(fb + (size_t)(hh * HALF + j) * 128 + L) + df_to_double(df{d2.x, d2.y});
    }
  }
  __syncthreads();
  double* part = a.w.partials + (size_t)bid * NC * NC;
  for (int e2 = tid; e2 < NC * NC; e2 += T) {
    const int i = e2 / NC, j = e2 % NC;
    double s = 0.0;
#pragma unroll
    for (int kk = 0; kk < SP; ++kk) s += red[(kk * NC + i) * NC + j];
    __stcg(part + e2, s);
  }
  gram_finish<NC, T, S, ArithDF>(a, smem, colmax, misc, k);
}

template <int NC, typename S, int XF = kXNone>
__global__ void __launch_bounds__(PipeShape<NC>::T, 1)
    gram_pipe_kernel(const __grid_constant__ GramArgs<S> a, const __grid_constant__ CUtensorMap tmA,
                     const __grid_constant__ CUtensorMap tmB, int has_b) {
  extern __shared__ __align__(1024) unsigned char smem_umma[];
  const uint32_t tbase = pipe_cta_begin<NC, S>(smem_umma);
  PipeBars bars;
  gram_pipe_body<NC, S, XF>(a, blockIdx.x, gridDim.x, tbase, bars, &tmA, has_b ? &tmB : nullptr);
  tc_fence_before();
  __syncthreads();
  if ((threadIdx.x >> 5) == 0) tmem_dealloc(tbase, PipeShape<NC>::TCOLS);
}

// pass 1 (XF = kXNone) or a later pass (XF = kXUpper / kXFull, pass 2 or 3)
template <int NC, typename S, int XF = kXNone>
ql_status gram_pipe_launch_one(const GramCall& c, const GramWs& w, int pass = 1) {
  using Sh = PipeShape<NC>;
  using Sm = PipeSmem<NC, S, XF>;
  auto kern = gram_pipe_kernel<NC, S, XF>;
  static bool ready = false;
  static std::mutex mu;
  {
    std::lock_guard<std::mutex> lk(mu);
    if (!ready) {
      if (cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)Sm::kBytes) != cudaSuccess)
        return QL_ERR_CUDA;
      ready = true;
    }
  }
  // one CTA per SM: the shared memory allows no second one
  const int64_t tiles = (c.m + Sh::KT - 1) / Sh::KT;
  int64_t g = (int64_t)device_sm_count();
  if (g > tiles) g = tiles;
  if (g < 1) g = 1;
  GramArgs<S> a{};
  a.src.A = static_cast<const S*>(c.A);
  a.src.lda = c.lda;
  a.src.b = static_cast<const S*>(c.b);
  a.src.nA = c.nA;
  a.m = c.m;
  a.n = c.n;
  a.tiles = tiles;
  a.pass = pass;
  a.method = c.method;
  a.gated = 0;
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
  CUtensorMap tmA{}, tmB{};
  const bool has_b = c.nA < c.n;
  a.bulk = pipe_tensor_maps(&tmA, has_b ? &tmB : nullptr, c.A, c.b, std::is_same<S, double>::value ? QL_F64 : QL_F32,
                            c.m, c.nA, c.lda)
               ? 1
               : 0;
  a.mround = 2;
  count_launch();
  kern<<<(int)g, Sh::T, Sm::kBytes, c.stream>>>(a, tmA, tmB, has_b ? 1 : 0);
  return cudaPeekAtLastError() == cudaSuccess ? QL_OK : QL_ERR_CUDA;
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
  GramArgs<S> a{};
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
  a.mround = std::is_same<Ar, ArithDF>::value ? 1 : 0;
  count_launch();
  kern<<<(int)g, Sh::T, Sm::kBytes, c.stream>>>(a);
  return cudaPeekAtLastError() == cudaSuccess ? QL_OK : QL_ERR_CUDA;
}

// All passes of one method (two, three for shifted Cholesky-QR3) for one (storage, arithmetic) pair.
template <typename S, typename Ar>
ql_status gram_dispatch(const GramCall& c, const GramWs& w, int gated) {
  if (c.method == QL_TSQR) return gram_stream_launch_one<1, S, Ar, kXNone>(c, w, 1, gated);  // n = 1: ||x||
  auto two = [&](auto nc_tag) -> ql_status {
    constexpr int NC = decltype(nc_tag)::value;
    if constexpr (NC >= 16 && std::is_same<Ar, ArithDF>::value) {
      if (tc_gram_enabled()) {
        // first pass: the pipelined tcgen05 kernel (its read-outs are rare, so stacking
        // 128 / NC planes costs little).  Later passes: tcgen05 per tile for 64 columns;
        // below that mma.sync, whose per-tile read-out is cheaper than TMEM's
        if constexpr (NC == 64) {
          ql_status st =
              pipe_gram_enabled() ? gram_pipe_launch_one<NC, S>(c, w) : gram_umma_launch_one<NC, S, kXNone>(c, w, 1);
          if (st) return st;
          if (c.method == QL_SVQB2) return gram_umma_launch_one<NC, S, kXFull>(c, w, 2);
          st = gram_umma_launch_one<NC, S, kXUpper>(c, w, 2);
          if (st || c.method != QL_SCHOLQR3) return st;
          return gram_umma_launch_one<NC, S, kXUpper>(c, w, 3);
        } else {
          ql_status st =
              pipe_gram_enabled() ? gram_pipe_launch_one<NC, S>(c, w) : gram_tc_launch_one<NC, S, kXNone>(c, w, 1);
          if (st) return st;
          // later passes: the pipelined kernel forms Y = X M' in its slicer warps
          const bool pipe2 = pipe_gram_enabled() && pipe_gram2_enabled();
          if (c.method == QL_SVQB2)
            return pipe2 ? gram_pipe_launch_one<NC, S, kXFull>(c, w, 2) : gram_tc_launch_one<NC, S, kXFull>(c, w, 2);
          st = pipe2 ? gram_pipe_launch_one<NC, S, kXUpper>(c, w, 2) : gram_tc_launch_one<NC, S, kXUpper>(c, w, 2);
          if (st || c.method != QL_SCHOLQR3) return st;
          return pipe2 ? gram_pipe_launch_one<NC, S, kXUpper>(c, w, 3) : gram_tc_launch_one<NC, S, kXUpper>(c, w, 3);
        }
      }
    }
    if constexpr (NC <= 4) {  // narrow X: the streaming kernel (n = 8 would spill its 36 accumulators)
      ql_status st = gram_stream_launch_one<NC, S, Ar, kXNone>(c, w, 1, gated);
      if (st) return st;
      if (c.method == QL_SVQB2) return gram_stream_launch_one<NC, S, Ar, kXFull>(c, w, 2, gated);
      st = gram_stream_launch_one<NC, S, Ar, kXUpper>(c, w, 2, gated);
      if (st || c.method != QL_SCHOLQR3) return st;
      return gram_stream_launch_one<NC, S, Ar, kXUpper>(c, w, 3, gated);
    }
    ql_status st = gram_launch_one<NC, S, Ar, kXNone>(c, w, 1, gated);
    if (st) return st;
    if (c.method == QL_SVQB2) return gram_launch_one<NC, S, Ar, kXFull>(c, w, 2, gated);
    st = gram_launch_one<NC, S, Ar, kXUpper>(c, w, 2, gated);
    if (st || c.method != QL_SCHOLQR3) return st;
    return gram_launch_one<NC, S, Ar, kXUpper>(c, w, 3, gated);
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
