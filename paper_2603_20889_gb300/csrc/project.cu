// Two-phase orthogonalisation (the "two-phase problem" QR = (I - Y Y^T) X with
// re-orthogonalisation that Sec. 2 discusses for the Gram methods): for Y (m x k) with
// orthonormal columns and X (m x n),
//   C1 = Y^T X,  W1 = X - Y C1,  C2 = Y^T W1,  W = W1 - Y C2,  C = C1 + C2,
// so that W = (I - Y Y^T) X to working precision even when X is nearly in range(Y).  The R
// of the orthogonalised block is then any of the Q-less calls on W.
//
// Four launches (cross product, update, cross product, update).  The cross product Y^T V is
// a reduction over the m rows: every CTA accumulates 4 x 4 blocks of the k x n product over
// its row tiles in double-float, writes one FP64 partial, and the last CTA to finish sums
// the partials in a fixed order (reproducible).  The update W = V - Y C streams the rows,
// one per thread.  Tiles outside the double-float exponent range run in FP64.
#include <mutex>

#include "internal.h"
#include "small_dense.cuh"

namespace ql {

constexpr int kProjT = 256;
constexpr int kProjB = 128;  // rows per tile of the cross product

struct ProjWs {
  int* flags;        // [0] arrival counter
  double* cprev;     // C of the first pass (k x n, ld n)
  double* cpass;     // C of the current pass, read by the update (k x n, ld n)
  double* partials;  // one KC x NC partial per CTA
};

template <typename S>
struct ProjArgs {
  int64_t m;
  int k, n;
  const S* Y;
  int64_t ldy;
  const S* V;  // X (pass 1) or W1 (pass 2)
  int64_t ldv;
  S* W;
  int64_t ldw;
  double* C;  // output coefficients (k x n, ld ldc)
  int64_t ldc;
  int pass;
  ProjWs w;
  int64_t tiles;
};

QL_DEV bool df_range_ok_dev(int E) { return E == 0 || (E >= kDfEminLimit && E <= kDfEmaxLimit); }

QL_DEV df load_df(double x, int& E) { return df_split_double(x, E); }
QL_DEV df load_df(float x, int& E) {
  const int e = (__float_as_int(x) >> 23) & 0xff;
  E = e == 0 ? 0 : e + 896;
  return df{x, 0.0f};
}

// ---- C = Y^T V over the rows (partials per CTA, fixed-order reduction in the last CTA)
template <int KC, int NC, typename S>
__global__ void __launch_bounds__(kProjT, 1) cross_kernel(ProjArgs<S> a) {
  constexpr int T = kProjT, B = kProjB;
  constexpr int NBLK = (KC / 4) * (NC / 4);  // 4 x 4 blocks of C
  constexpr int SL = T / NBLK >= 1 ? T / NBLK : 1;
  static_assert(NBLK <= T, "one block per thread at least");
  extern __shared__ __align__(16) unsigned char smem[];
  df* Ys = reinterpret_cast<df*>(smem);             // [KC][B]
  df* Vs = Ys + KC * B;                             // [NC][B]
  double* red = reinterpret_cast<double*>(Vs + NC * B);  // [SL][KC][NC] at the end
  int* misc = reinterpret_cast<int*>(red + (size_t)SL * KC * NC);
  const int tid = threadIdx.x, k = a.k, n = a.n;
  const int blk = tid / SL, slice = tid % SL;
  const bool active = blk < NBLK;
  const int bi = active ? (blk / (NC / 4)) * 4 : 0, bj = active ? (blk % (NC / 4)) * 4 : 0;

  ArithDF::Acc acc[4][4];
  double acc64[4][4];
#pragma unroll
  for (int i = 0; i < 4; ++i)
#pragma unroll
    for (int j = 0; j < 4; ++j) {
      acc[i][j] = ArithDF::acc_zero();
      acc64[i][j] = 0.0;
    }
  const int64_t nb = gridDim.x, bid = blockIdx.x;
  const int64_t t0 = a.tiles * bid / nb, t1 = a.tiles * (bid + 1) / nb;
  for (int64_t t = t0; t < t1; ++t) {
    const int64_t row0 = t * B;
    bool bad = false;
    for (int e = tid; e < (KC + NC) * B; e += T) {
      const int c = e / B, r = e % B;
      const int64_t row = row0 + r;
      df v = df{0.0f, 0.0f};
      int E = 0;
      if (c < KC) {
        if (c < k && row < a.m) v = load_df(a.Y[c * a.ldy + row], E);
        Ys[c * B + r] = v;
      } else {
        const int cv = c - KC;
        if (cv < n && row < a.m) v = load_df(a.V[cv * a.ldv + row], E);
        Vs[cv * B + r] = v;
      }
      if (!df_range_ok_dev(E)) bad = true;
    }
    const bool f64 = __syncthreads_or(bad);
    if (active) {
      if (!f64) {
        for (int r = slice; r < B; r += SL) {
          df y[4], v[4];
#pragma unroll
          for (int i = 0; i < 4; ++i) y[i] = Ys[(bi + i) * B + r];
#pragma unroll
          for (int j = 0; j < 4; ++j) v[j] = Vs[(bj + j) * B + r];
#pragma unroll
          for (int i = 0; i < 4; ++i)
#pragma unroll
            for (int j = 0; j < 4; ++j) ArithDF::acc_fma(acc[i][j], y[i], v[j]);
        }
      } else {  // FP64 for this tile, straight from global memory
        for (int r = slice; r < B; r += SL) {
          const int64_t row = row0 + r;
          if (row >= a.m) break;
          double y[4], v[4];
#pragma unroll
          for (int i = 0; i < 4; ++i) y[i] = bi + i < k ? (double)a.Y[(bi + i) * a.ldy + row] : 0.0;
#pragma unroll
          for (int j = 0; j < 4; ++j) v[j] = bj + j < n ? (double)a.V[(bj + j) * a.ldv + row] : 0.0;
#pragma unroll
          for (int i = 0; i < 4; ++i)
#pragma unroll
            for (int j = 0; j < 4; ++j) acc64[i][j] = fma(y[i], v[j], acc64[i][j]);
        }
      }
    }
    __syncthreads();
  }
  // combine the slices and store this CTA's partial (FP64)
  if (active) {
#pragma unroll
    for (int i = 0; i < 4; ++i)
#pragma unroll
      for (int j = 0; j < 4; ++j)
        red[((size_t)slice * KC + bi + i) * NC + bj + j] =
            df_to_double(ArithDF::acc_get(acc[i][j])) + acc64[i][j];
  }
  __syncthreads();
  double* part = a.w.partials + (size_t)bid * KC * NC;
  for (int e = tid; e < KC * NC; e += T) {
    double s = 0.0;
    for (int sl = 0; sl < SL; ++sl) s += red[(size_t)sl * KC * NC + e];
    __stcg(part + e, s);
  }
  __threadfence();
  __syncthreads();
  if (tid == 0) {
    const int old = atomicAdd(&a.w.flags[0], 1);
    misc[0] = old == (int)nb - 1;
    if (old == (int)nb - 1) a.w.flags[0] = 0;
  }
  __syncthreads();
  if (!misc[0]) return;
  __threadfence();
  // last CTA: fixed-order sum of the partials -> C of this pass (and the running total)
  for (int e = tid; e < k * n; e += T) {
    const int i = e / n, j = e % n;
    double s = 0.0;
    for (int b = 0; b < (int)nb; ++b) s += __ldcg(a.w.partials + (size_t)b * KC * NC + i * NC + j);
    a.w.cpass[i * n + j] = s;
    const double tot = a.pass == 1 ? s : __ldcg(a.w.cprev + i * n + j) + s;
    if (a.pass == 1) a.w.cprev[i * n + j] = s;
    a.C[j * a.ldc + i] = tot;
  }
}

// ---- W = V - Y C (C of this pass), one row per thread
template <int KC, int NC, typename S>
__global__ void __launch_bounds__(kProjT, 1) update_kernel(ProjArgs<S> a) {
  constexpr int T = kProjT;
  extern __shared__ __align__(16) unsigned char smem[];
  double* Cf = reinterpret_cast<double*>(smem);     // [KC][NC]
  df* Cd = reinterpret_cast<df*>(Cf + KC * NC);      // [KC][NC]
  df* ys = Cd + KC * NC;                             // [KC][T]
  const int tid = threadIdx.x, k = a.k, n = a.n;
  bool cbad = false;
  for (int e = tid; e < KC * NC; e += T) {
    const int i = e / NC, j = e % NC;
    const double c = (i < k && j < n) ? __ldcg(a.w.cpass + i * n + j) : 0.0;
    Cf[e] = c;
    const int E = (int)((__double_as_longlong(c) >> 52) & 0x7ff);
    if (c != 0.0 && (E < 1023 - 80 || E > 1023 + 80)) cbad = true;  // products with Y stay normal floats
    Cd[e] = df_from_double_rn(c);
  }
  const bool c64 = __syncthreads_or(cbad);
  const int64_t nb = gridDim.x, bid = blockIdx.x;
  const int64_t t0 = a.tiles * bid / nb, t1 = a.tiles * (bid + 1) / nb;
  for (int64_t t = t0; t < t1; ++t) {
    const int64_t row = t * T + tid;
    const bool live = row < a.m;
    bool bad = false;
    for (int i = 0; i < k; ++i) {
      int E = 0;
      df y = df{0.0f, 0.0f};
      if (live) y = load_df(a.Y[i * a.ldy + row], E);
      if (!df_range_ok_dev(E)) bad = true;
      ys[i * T + tid] = y;
    }
    const bool f64 = __syncthreads_or(bad) || c64;
#pragma unroll 1
    for (int jb = 0; jb < n; jb += 8) {
      if (!f64) {
        ArithDF::Acc acc[8];
#pragma unroll
        for (int jj = 0; jj < 8; ++jj) acc[jj] = ArithDF::acc_zero();
#pragma unroll 1
        for (int i = 0; i < k; ++i) {
          const df y = ys[i * T + tid];
#pragma unroll
          for (int jj = 0; jj < 8; ++jj) ArithDF::acc_fma(acc[jj], y, Cd[i * NC + jb + jj]);
        }
        if (live) {
#pragma unroll
          for (int jj = 0; jj < 8; ++jj) {
            const int j = jb + jj;
            if (j < n) {
              int E;
              const df v = load_df(a.V[j * a.ldv + row], E);
              bool vbad = !df_range_ok_dev(E);
              if (!vbad) {
                const df w = df_sub(v, ArithDF::acc_get(acc[jj]));
                if constexpr (sizeof(S) == 8)
                  a.W[j * a.ldw + row] = (double)w.hi + (double)w.lo;
                else
                  a.W[j * a.ldw + row] = __fadd_rn(w.hi, w.lo);
              } else {  // this entry alone is out of range: FP64
                double s = (double)a.V[j * a.ldv + row];
                for (int i = 0; i < k; ++i) s = fma(-(double)a.Y[i * a.ldy + row], Cf[i * NC + j], s);
                a.W[j * a.ldw + row] = (S)s;
              }
            }
          }
        }
      } else if (live) {
        for (int jj = 0; jj < 8 && jb + jj < n; ++jj) {
          const int j = jb + jj;
          double s = (double)a.V[j * a.ldv + row];
          for (int i = 0; i < k; ++i) s = fma(-(double)a.Y[i * a.ldy + row], Cf[i * NC + j], s);
          a.W[j * a.ldw + row] = (S)s;
        }
      }
    }
    __syncthreads();  // ys is rewritten by the next tile
  }
}

static int cls(int v) { return v <= 8 ? 8 : v <= 16 ? 16 : v <= 32 ? 32 : 64; }

template <int KC, int NC>
struct ProjSmem {
  static constexpr int NBLK = (KC / 4) * (NC / 4);
  static constexpr int SL = kProjT / NBLK >= 1 ? kProjT / NBLK : 1;
  static constexpr size_t kCross = 8 * (size_t)(KC + NC) * kProjB + 8 * (size_t)SL * KC * NC + 64;
  static constexpr size_t kUpdate = 16 * (size_t)KC * NC + 8 * (size_t)KC * kProjT;
};

static size_t proj_parts_bytes() { return (size_t)device_sm_count() * 64 * 64 * sizeof(double); }

size_t project_workspace_bytes(int k, int n) {
  if (k < 1 || k > kMaxN || n < 1 || n > kMaxN) return 0;
  return 256 + 2 * (size_t)kMaxN * kMaxN * sizeof(double) + proj_parts_bytes();
}

template <int KC, int NC, typename S>
static ql_status proj_run(ProjArgs<S> a, cudaStream_t st) {
  using Sm = ProjSmem<KC, NC>;
  auto ck = cross_kernel<KC, NC, S>;
  auto uk = update_kernel<KC, NC, S>;
  static bool ready = false;
  static std::mutex mu;
  {
    std::lock_guard<std::mutex> lk(mu);
    if (!ready) {
      if (cudaFuncSetAttribute(ck, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)Sm::kCross) != cudaSuccess ||
          cudaFuncSetAttribute(uk, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)Sm::kUpdate) != cudaSuccess)
        return QL_ERR_CUDA;
      ready = true;
    }
  }
  const int64_t ctiles = (a.m + kProjB - 1) / kProjB, utiles = (a.m + kProjT - 1) / kProjT;
  int64_t gc = device_sm_count(), gu = device_sm_count();
  if (gc > ctiles) gc = ctiles;
  if (gu > utiles) gu = utiles;
  if (gc < 1) gc = 1;
  if (gu < 1) gu = 1;
  const S* X = a.V;
  const int64_t ldx = a.ldv;
  for (int pass = 1; pass <= 2; ++pass) {
    a.pass = pass;
    if (pass == 2) {  // the second phase projects the first one's result again
      a.V = a.W;
      a.ldv = a.ldw;
    } else {
      a.V = X;
      a.ldv = ldx;
    }
    a.tiles = ctiles;
    count_launch();
    ck<<<(int)gc, kProjT, Sm::kCross, st>>>(a);
    if (cudaPeekAtLastError() != cudaSuccess) return QL_ERR_CUDA;
    a.tiles = utiles;
    count_launch();
    uk<<<(int)gu, kProjT, Sm::kUpdate, st>>>(a);
    if (cudaPeekAtLastError() != cudaSuccess) return QL_ERR_CUDA;
  }
  return QL_OK;
}

template <typename S>
static ql_status proj_dispatch(ProjArgs<S> a, cudaStream_t st) {
  const int kc = cls(a.k), nc = cls(a.n);
#define QL_PROJ_CASE(K, N) \
  if (kc == K && nc == N) return proj_run<K, N, S>(a, st);
#define QL_PROJ_ROW(K) QL_PROJ_CASE(K, 8) QL_PROJ_CASE(K, 16) QL_PROJ_CASE(K, 32) QL_PROJ_CASE(K, 64)
  QL_PROJ_ROW(8) QL_PROJ_ROW(16) QL_PROJ_ROW(32) QL_PROJ_ROW(64)
#undef QL_PROJ_ROW
#undef QL_PROJ_CASE
  return QL_ERR_ARG;
}

}  // namespace ql

using namespace ql;

extern "C" {

size_t ql_project_workspace_bytes(int64_t k, int64_t n) { return project_workspace_bytes((int)k, (int)n); }

ql_status ql_project_out(int64_t m, int64_t k, const void* Y, int64_t ldy, int64_t n, const void* X, int64_t ldx,
                         ql_dtype dtype, void* W, int64_t ldw, double* C, int64_t ldc, void* ws, size_t ws_bytes,
                         void* stream) {
  const int64_t lmin = m > 1 ? m : 1;
  if (m < 0 || k < 1 || k > kMaxN || n < 1 || n > kMaxN || (dtype != QL_F64 && dtype != QL_F32) || ldy < lmin ||
      ldx < lmin || ldw < lmin || ldc < k || !C || (m > 0 && (!Y || !X || !W)))
    return QL_ERR_ARG;
  const size_t el = dtype == QL_F64 ? 8 : 4;
  if ((reinterpret_cast<uintptr_t>(Y) % el) || (reinterpret_cast<uintptr_t>(X) % el) ||
      (reinterpret_cast<uintptr_t>(W) % el) || (reinterpret_cast<uintptr_t>(C) % 8))
    return QL_ERR_ALIGN;
  if (!ws || ws_bytes < project_workspace_bytes((int)k, (int)n)) return QL_ERR_WORKSPACE;
  cudaStream_t st = (cudaStream_t)stream;
  unsigned char* b = static_cast<unsigned char*>(ws);
  ProjWs w;
  w.flags = reinterpret_cast<int*>(b);
  w.cprev = reinterpret_cast<double*>(b + 256);
  w.cpass = w.cprev + (size_t)kMaxN * kMaxN;
  w.partials = w.cpass + (size_t)kMaxN * kMaxN;
  if (cudaMemsetAsync(w.flags, 0, 256, st) != cudaSuccess) return QL_ERR_CUDA;
  if (dtype == QL_F64) {
    ProjArgs<double> a{m, (int)k, (int)n, static_cast<const double*>(Y), ldy, static_cast<const double*>(X), ldx,
                       static_cast<double*>(W), ldw, C, ldc, 1, w, 0};
    return proj_dispatch(a, st);
  }
  ProjArgs<float> a{m, (int)k, (int)n, static_cast<const float*>(Y), ldy, static_cast<const float*>(X), ldx,
                    static_cast<float*>(W), ldw, C, ldc, 1, w, 0};
  return proj_dispatch(a, st);
}

}  // extern "C"
