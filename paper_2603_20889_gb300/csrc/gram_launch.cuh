// Gram-pass kernel of CholQR2 / SVQB2 and its launch template (paper Sec. 3.1).
// Instantiated per (storage, arithmetic) in gram_inst_*.cu.
#pragma once

#include <mutex>

#include "epilogue.cuh"
#include "gram.cuh"
#include "internal.h"
#include "small_dense.cuh"
#include "gram_tc.cuh"

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

template <int NC, int T, typename S, typename Ar>
QL_DEV void gram_finish(const GramArgs<S>& a, unsigned char* smem, const int* colmax, int* misc);

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
  gram_finish<NC, T, S, Ar>(a, smem, colmax, misc);
}

// Range verdict, "last CTA done" election and, in the last CTA, the fixed-order reduction
// of all CTA partials followed by the n x n FP64 epilogue of the pass.  Shared by the SIMT
// and the tensor-core Gram kernels (the caller has written this CTA's partial already).
template <int NC, int T, typename S, typename Ar>
QL_DEV void gram_finish(const GramArgs<S>& a, unsigned char* smem, const int* colmax, int* misc) {
  using V = typename Ar::T;
  const int tid = threadIdx.x, n = a.n, k = gridDim.x;
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


// Tensor-core Gram pass (double-float policy only): see gram_tc.cuh.
template <int NC, typename S, int XF>
__global__ void __launch_bounds__(256, 1) gram_tc_kernel(GramArgs<S> a) {
  using Ar = ArithDF;
  using Sh = TcShape<NC>;
  using Sm = TcSmem<NC, S>;
  constexpr int T = 256, KT = Sh::KT, LDR = Sh::LDR, G = Sh::G, KS = Sh::KS, KPART = Sh::KPART;
  constexpr int GPR = Sh::NCB / G;              // column-block groups per row block
  constexpr int PAIRS = NC * KT / 2 / T;        // row pairs per thread and tile
  extern __shared__ __align__(16) unsigned char smem[];
  const int tid = threadIdx.x, n = a.n, lane = tid & 31, warp = tid >> 5;

  if (a.pass == 2 && *(volatile int*)&a.w.flags[0] != 0) return;  // the FP64 launches redo it
  if (a.pass == 2 && *(volatile int*)&a.w.flags[1] != 0) {         // first pass broke down
    if (blockIdx.x == 0) write_nan_outputs(a, T);
    return;
  }
  S* stage = reinterpret_cast<S*>(smem);
  df* stage_df = reinterpret_cast<df*>(smem);
  unsigned short* slices = reinterpret_cast<unsigned short*>(smem + Sm::kOffSlices);
  df* Mv = reinterpret_cast<df*>(smem + Sm::kOffM);
  float* pow2c = reinterpret_cast<float*>(smem + Sm::kOffPow);
  int* expo = reinterpret_cast<int*>(smem + Sm::kOffExpo);
  int* colmax = reinterpret_cast<int*>(smem + Sm::kOffColmax);
  unsigned* zero16 = reinterpret_cast<unsigned*>(smem + Sm::kOffZero);
  int* misc = reinterpret_cast<int*>(smem + Sm::kOffMisc);

  for (int i = tid; i < NC; i += T) colmax[i] = 0;
  if (tid < 4) zero16[tid] = 0u;
  if constexpr (XF != kXNone) {
    const double* M = a.w.keep + (size_t)n * n;
    for (int i = tid; i < NC * NC; i += T) {
      int r = i / NC, c = i % NC;
      Mv[i] = (r < n && c < n) ? df_from_double_rn(__ldcg(M + r * n + c)) : df{0.0f, 0.0f};
    }
  }
  constexpr int U = Sh::U;
  const int g = lane >> 2, t4 = lane & 3;
  df acc[U][G][4];  // persistent per-unit C accumulators
#pragma unroll
  for (int ui = 0; ui < U; ++ui)
#pragma unroll
    for (int gi = 0; gi < G; ++gi)
#pragma unroll
      for (int e = 0; e < 4; ++e) acc[ui][gi][e] = df{0.0f, 0.0f};

  const int k = gridDim.x, bid = blockIdx.x;
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

  if (t0 < t1) issue(t0);
  __syncthreads();
  for (int64_t t = t0; t < t1; ++t) {
    cp_async_wait_all();
    __syncthreads();
    for (int i = tid; i < NC; i += T) expo[i] = 0;
    __syncthreads();
    df yv[XF != kXNone ? 2 * PAIRS : 1];
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
    } else {
      if constexpr (sizeof(S) == 8) {
        // convert the stage in place to double-float, once per element (+ range record)
#pragma unroll 4
        for (int k2 = 0; k2 < PAIRS; ++k2) {
          const int pi = tid + T * k2, c = (2 * pi) / KT, r = (2 * pi) % KT;
          int E0, E1;
          df d0 = Ar::load((double)stage[c * KT + r], E0);
          df d1 = Ar::load((double)stage[c * KT + r + 1], E1);
          stage_df[c * KT + r] = d0;
          stage_df[c * KT + r + 1] = d1;
          unsigned em = __reduce_max_sync(0xffffffffu, (unsigned)max(E0, E1));
          if (lane == 0 && em > 0) atomicMax(&colmax[c], (int)em);
        }
      } else {
#pragma unroll 4
        for (int k2 = 0; k2 < PAIRS; ++k2) {
          const int pi = tid + T * k2, c = (2 * pi) / KT, r = (2 * pi) % KT;
          unsigned e0 = (__float_as_uint((float)stage[c * KT + r]) >> 23) & 0xff;
          unsigned e1 = (__float_as_uint((float)stage[c * KT + r + 1]) >> 23) & 0xff;
          unsigned em = __reduce_max_sync(0xffffffffu, max(e0 ? e0 + 896 : 0u, e1 ? e1 + 896 : 0u));
          if (lane == 0 && em > 0) atomicMax(&colmax[c], (int)em);
        }
      }
      __syncthreads();
      // Y = W M, one pair of rows of one column per step (unrolled: yv stays in registers)
#pragma unroll
      for (int k2 = 0; k2 < PAIRS; ++k2) {
        const int pi = tid + T * k2, c = (2 * pi) / KT, r = (2 * pi) % KT;
        Ar::Acc s0 = Ar::acc_zero(), s1 = Ar::acc_zero();
        if (c < n) {
          const int kend = XF == kXUpper ? c + 1 : n;
          for (int kk = 0; kk < kend; ++kk) {
            df w0, w1;
            if constexpr (sizeof(S) == 8) {
              w0 = stage_df[kk * KT + r];
              w1 = stage_df[kk * KT + r + 1];
            } else {
              w0 = df{(float)stage[kk * KT + r], 0.0f};
              w1 = df{(float)stage[kk * KT + r + 1], 0.0f};
            }
            const df mk = Mv[kk * NC + c];
            Ar::acc_fma(s0, w0, mk);
            Ar::acc_fma(s1, w1, mk);
          }
        }
        yv[2 * k2] = Ar::acc_get(s0);
        yv[2 * k2 + 1] = Ar::acc_get(s1);
        unsigned e0 = (__float_as_uint(yv[2 * k2].hi) >> 23) & 0xff;
        unsigned e1 = (__float_as_uint(yv[2 * k2 + 1].hi) >> 23) & 0xff;
        unsigned em = __reduce_max_sync(0xffffffffu, max(e0, e1));
        if (lane == 0 && em > 0) atomicMax(&expo[c], (int)em);
      }
    }
    __syncthreads();
    // per-column scale 2^e_c, |y| < 2^e_c for the whole tile column
    for (int c = tid; c < NC; c += T) {
      const int em = expo[c];
      int e = 0;
      if (em > 0) e = (XF == kXNone) ? em - 1022 : em - 126;
      e = max(-126, min(127, e));
      pow2c[c] = __int_as_float((e + 127) << 23);
    }
    // slicing: seven signed base-128 digits per value, two rows per 32-bit store
#pragma unroll
    for (int k2 = 0; k2 < PAIRS; ++k2) {
      const int pi = tid + T * k2, c = (2 * pi) / KT, r = (2 * pi) % KT;
      const int em = expo[c];
      unsigned long long N[2];
      unsigned sg[2];
#pragma unroll
      for (int h = 0; h < 2; ++h) {
        if constexpr (XF == kXNone) {
          if constexpr (sizeof(S) == 8) {
            N[h] = fixed_of_double((double)stage[c * KT + r + h], em, sg[h]);
          } else {
            float x = (float)stage[c * KT + r + h];
            sg[h] = __float_as_uint(x) & 0x80000000u;
            N[h] = fixed_of_float(x, em - 896);
          }
        } else {
          const df y = yv[2 * k2 + h];
          sg[h] = __float_as_uint(y.hi) & 0x80000000u;
          unsigned long long nh = fixed_of_float(y.hi, em);
          unsigned long long nl = fixed_of_float(y.lo, em);
          bool same = ((__float_as_uint(y.lo) ^ __float_as_uint(y.hi)) & 0x80000000u) == 0u;
          N[h] = same ? nh + nl : (nh > nl ? nh - nl : 0ull);
        }
      }
#pragma unroll
      for (int p = 0; p < Sh::ND; ++p) {
        const int sh = 7 * (Sh::ND - 1 - p);
        unsigned lo16 = bf16_digit((unsigned)(N[0] >> sh) & 127u, sg[0]);
        unsigned hi16 = bf16_digit((unsigned)(N[1] >> sh) & 127u, sg[1]);
        *reinterpret_cast<unsigned*>(slices + ((size_t)p * NC + c) * LDR + r) = lo16 | (hi16 << 16);
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
#pragma unroll
      for (int gi = 0; gi < G; ++gi) {
        const float fj0 = pow2c[(cb0 + gi) * 8 + 2 * t4], fj1 = pow2c[(cb0 + gi) * 8 + 2 * t4 + 1];
#pragma unroll
        for (int dd = 0; dd < 7; ++dd) {
          const float sd = __int_as_float((127 - 7 * (dd + 2)) << 23);  // 2^(-7d)
          acc[ui][gi][0] = df_add(acc[ui][gi][0], df{accd[dd][gi][0] * (fi0 * fj0 * sd), 0.0f});
          acc[ui][gi][1] = df_add(acc[ui][gi][1], df{accd[dd][gi][1] * (fi0 * fj1 * sd), 0.0f});
          acc[ui][gi][2] = df_add(acc[ui][gi][2], df{accd[dd][gi][2] * (fi1 * fj0 * sd), 0.0f});
          acc[ui][gi][3] = df_add(acc[ui][gi][3], df{accd[dd][gi][3] * (fi1 * fj1 * sd), 0.0f});
        }
      }
    }
  }
  __syncthreads();
  // combine the row parts of each C tile and store this CTA's partial Gram matrix
  df* red = reinterpret_cast<df*>(smem + Sm::kOffSlices);  // [unit][G][4][32]
#pragma unroll
  for (int ui = 0; ui < U; ++ui)
#pragma unroll
    for (int gi = 0; gi < G; ++gi)
#pragma unroll
      for (int e = 0; e < 4; ++e) red[(((warp * U + ui) * G + gi) * 4 + e) * 32 + lane] = acc[ui][gi][e];
  __syncthreads();
  double* part = a.w.partials + (size_t)bid * NC * NC;
  for (int idx = tid; idx < Sh::GROUPS * G * 4 * 32; idx += T) {
    const int ln = idx % 32, e = (idx / 32) % 4, gi = (idx / 128) % G, gr = idx / (128 * G);
    df s = df{0.0f, 0.0f};
    for (int kq = 0; kq < KS; ++kq) s = df_add(s, red[(((gr * KS + kq) * G + gi) * 4 + e) * 32 + ln]);
    const int rb2 = gr / GPR, cbb = (gr % GPR) * G + gi;
    const int i = rb2 * 16 + (ln >> 2) + (e >= 2 ? 8 : 0), j = cbb * 8 + 2 * (ln & 3) + (e & 1);
    if (i < NC && j < NC) __stcg(part + i * NC + j, df_to_double(s));
  }
  gram_finish<NC, T, S, ArithDF>(a, smem, colmax, misc);
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
  count_launch();
  kern<<<(int)g, Sh::T, Sm::kBytes, c.stream>>>(a);
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
    if constexpr (NC >= 16 && std::is_same<Ar, ArithDF>::value) {
      if (tc_gram_enabled()) {
        ql_status st = gram_tc_launch_one<NC, S, kXNone>(c, w, 1);
        if (st) return st;
        if (c.method == QL_CHOLQR2) return gram_tc_launch_one<NC, S, kXUpper>(c, w, 2);
        return gram_tc_launch_one<NC, S, kXFull>(c, w, 2);
      }
    }
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
