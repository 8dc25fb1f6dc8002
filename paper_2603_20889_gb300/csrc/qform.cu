// Q reconstruction: Q = X R^{-1}, the orthonormal factor of X = Q R from the R that any of
// the Q-less calls returned (the explicit Q of Sec. 1 that block iterative solvers use).
//
// One launch.  Every CTA inverts R (FP64, shared memory; n <= 64 so this is cheap) and then
// streams row tiles of T rows: each thread owns one row, converts it once to double-float
// (shared memory, conflict-free), and forms its row of Q = X M eight columns at a time from
// the M rows above the diagonal.  A tile whose X or whose M lies outside the double-float
// exponent range is formed in FP64 instead (decided per tile, the same for the whole CTA),
// so no second launch and no workspace are needed.
#include <mutex>

#include "internal.h"
#include "small_dense.cuh"

namespace ql {

template <typename S>
struct QformArgs {
  int64_t m;
  int n;
  const S* X;
  int64_t ldx;
  const double* R;
  int64_t ldr;
  S* Q;
  int64_t ldq;
  int32_t* info;
  int64_t tiles;
};

template <int NC>
struct QformSmem {
  static constexpr int T = 256;                              // rows per tile, one per thread
  static constexpr int LDM = NC + 1;                         // odd stride: column walks of the inverse
  static constexpr size_t kM = 8 * (size_t)NC * LDM;         // FP64 M = R^{-1}
  static constexpr size_t kMd = 8 * (size_t)NC * NC;         // double-float M (row k, 8 columns per load)
  static constexpr size_t kX = 8 * (size_t)NC * T;           // the tile as double-float, [k][row]
  static constexpr size_t kOffMd = kM;
  static constexpr size_t kOffX = kOffMd + kMd;
  static constexpr size_t kOffMisc = kOffX + kX;
  static constexpr size_t kBytes = kOffMisc + 64;
};

template <int NC, typename S>
__global__ void __launch_bounds__(256, 1) qform_kernel(QformArgs<S> a) {
  using Sm = QformSmem<NC>;
  constexpr int T = Sm::T, LDM = Sm::LDM;
  extern __shared__ __align__(16) unsigned char smem[];
  double* Mf = reinterpret_cast<double*>(smem);
  df* Md = reinterpret_cast<df*>(smem + Sm::kOffMd);
  df* xs = reinterpret_cast<df*>(smem + Sm::kOffX);
  int* misc = reinterpret_cast<int*>(smem + Sm::kOffMisc);
  const int tid = threadIdx.x, n = a.n;

  // ---- M = R^{-1} (FP64).  A zero diagonal entry (rank-deficient R) gives no inverse.
  double* Rs = reinterpret_cast<double*>(smem + Sm::kOffX);  // the tile area is free here
  for (int e = tid; e < n * n; e += T) {
    const int i = e % n, j = e / n;
    Rs[i * LDM + j] = i <= j ? __ldcg(a.R + (int64_t)j * a.ldr + i) : 0.0;
  }
  if (tid == 0) {
    int zi = 0;
    for (int i = 0; i < n; ++i)
      if (!(__ldcg(a.R + (int64_t)i * a.ldr + i) != 0.0)) {
        zi = i + 1;
        break;
      }
    misc[0] = zi;
  }
  __syncthreads();
  const int zi = misc[0];
  if (zi) {  // Q would not be finite: NaN columns from the first zero pivot on, and the status
    const int64_t k = gridDim.x;
    const int64_t r0 = a.tiles * blockIdx.x / k * T, r1 = min(a.m, a.tiles * (blockIdx.x + 1) / k * T);
    for (int j = 0; j < n; ++j)
      for (int64_t r = r0 + tid; r < r1; r += T) a.Q[j * a.ldq + r] = (S)__longlong_as_double(0x7ff8000000000000ll);
    if (blockIdx.x == 0 && tid == 0 && a.info) {
      a.info[0] = QL_ERR_NOT_SPD;
      a.info[1] = zi;
    }
    return;
  }
  tri_upper_inverse<T>(Rs, LDM, Mf, LDM, n);
  // double-float copy (zero below the diagonal and past n) and its range verdict
  bool mbad = false;
  for (int e = tid; e < NC * NC; e += T) {
    const int k = e / NC, j = e % NC;
    const double v = (k < n && j < n && k <= j) ? Mf[k * LDM + j] : 0.0;
    if (v != 0.0) {
      const int E = (int)((__double_as_longlong(v) >> 52) & 0x7ff);
      if (E < 1023 - 60 || E > 1023 + 60) mbad = true;
    }
    Md[k * NC + j] = df_from_double_rn(v);
  }
  const bool m_f64 = __syncthreads_or(mbad);
  if (blockIdx.x == 0 && tid == 0 && a.info) {
    a.info[0] = QL_OK;
    a.info[1] = 0;
  }

  const int64_t k = gridDim.x, bid = blockIdx.x;
  const int64_t t0 = a.tiles * bid / k, t1 = a.tiles * (bid + 1) / k;
  for (int64_t t = t0; t < t1; ++t) {
    const int64_t row = t * T + tid;
    const bool live = row < a.m;
    // this thread's row as double-float, [k][row] in shared memory (conflict-free)
    bool xbad = false;
    for (int c = 0; c < n; ++c) {
      int E = 0;
      df v = df{0.0f, 0.0f};
      if (live) {
        const S x = a.X[c * a.ldx + row];
        if constexpr (sizeof(S) == 8) {
          v = df_split_double((double)x, E);
        } else {
          const int e = (__float_as_int((float)x) >> 23) & 0xff;
          E = e == 0 ? 0 : e + 896;
          v = df{(float)x, 0.0f};
        }
      }
      if (E != 0 && (E < kDfEminLimit || E > kDfEmaxLimit)) xbad = true;
      xs[c * T + tid] = v;
    }
    const bool f64 = __syncthreads_or(xbad) || m_f64;
    if (!f64) {
#pragma unroll 1
      for (int jb = 0; jb < n; jb += 8) {
        ArithDF::Acc acc[8];
#pragma unroll
        for (int jj = 0; jj < 8; ++jj) acc[jj] = ArithDF::acc_zero();
        const int kend = min(n, jb + 8);  // M is upper triangular: rows past column jb + 7 are zero
#pragma unroll 1
        for (int kk = 0; kk < kend; ++kk) {
          const df xk = xs[kk * T + tid];
#pragma unroll
          for (int jj = 0; jj < 8; ++jj) ArithDF::acc_fma(acc[jj], xk, Md[kk * NC + jb + jj]);
        }
        if (live) {
#pragma unroll
          for (int jj = 0; jj < 8; ++jj) {
            if (jb + jj < n) {
              const df q = ArithDF::acc_get(acc[jj]);
              if constexpr (sizeof(S) == 8)
                a.Q[(jb + jj) * a.ldq + row] = (double)q.hi + (double)q.lo;
              else
                a.Q[(jb + jj) * a.ldq + row] = __fadd_rn(q.hi, q.lo);
            }
          }
        }
      }
    } else {
      // FP64 for this tile: outside the double-float range, or M is
#pragma unroll 1
      for (int jb = 0; jb < n; jb += 8) {
        double acc[8];
#pragma unroll
        for (int jj = 0; jj < 8; ++jj) acc[jj] = 0.0;
        const int kend = min(n, jb + 8);
#pragma unroll 1
        for (int kk = 0; kk < kend; ++kk) {
          const double xk = live ? (double)a.X[kk * a.ldx + row] : 0.0;
#pragma unroll
          for (int jj = 0; jj < 8; ++jj)
            acc[jj] = fma(xk, (kk < n && jb + jj < n && kk <= jb + jj) ? Mf[kk * LDM + jb + jj] : 0.0, acc[jj]);
        }
        if (live) {
#pragma unroll
          for (int jj = 0; jj < 8; ++jj)
            if (jb + jj < n) a.Q[(jb + jj) * a.ldq + row] = (S)acc[jj];
        }
      }
    }
    __syncthreads();  // the tile area is rewritten by the next tile
  }
}

template <int NC, typename S>
static ql_status qform_launch_one(const QformArgs<S>& a, cudaStream_t stream) {
  using Sm = QformSmem<NC>;
  auto kern = qform_kernel<NC, S>;
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
  int occ = 0;
  if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, kern, Sm::T, Sm::kBytes) != cudaSuccess) return QL_ERR_CUDA;
  int64_t g = (int64_t)device_sm_count() * (occ < 1 ? 1 : occ);
  if (g > a.tiles) g = a.tiles;
  if (g < 1) g = 1;
  count_launch();
  kern<<<(int)g, Sm::T, Sm::kBytes, stream>>>(a);
  return cudaPeekAtLastError() == cudaSuccess ? QL_OK : QL_ERR_CUDA;
}

template <typename S>
static ql_status qform_dispatch(QformArgs<S> a, cudaStream_t stream) {
  a.tiles = (a.m + QformSmem<8>::T - 1) / QformSmem<8>::T;
  if (a.tiles < 1) a.tiles = 1;
  const int n = a.n;
  if (n <= 8) return qform_launch_one<8, S>(a, stream);
  if (n <= 16) return qform_launch_one<16, S>(a, stream);
  if (n <= 32) return qform_launch_one<32, S>(a, stream);
  return qform_launch_one<64, S>(a, stream);
}

// dst <- the first nonzero {status, index} pair of src[0 .. count) (or {QL_OK, 0})
__global__ void first_status_kernel(int32_t* dst, const int32_t* src, int count) {
  if (threadIdx.x != 0 || blockIdx.x != 0) return;
  int32_t s = 0, i = 0;
  for (int c = 0; c < count; ++c)
    if (src[2 * c] != 0) {
      s = src[2 * c];
      i = src[2 * c + 1];
      break;
    }
  dst[0] = s;
  dst[1] = i;
}

ql_status first_status_async(int32_t* dst, const int32_t* src, int count, cudaStream_t stream) {
  count_launch();
  first_status_kernel<<<1, 32, 0, stream>>>(dst, src, count);
  return cudaPeekAtLastError() == cudaSuccess ? QL_OK : QL_ERR_CUDA;
}

}  // namespace ql

using namespace ql;

extern "C" ql_status ql_q_from_r(int64_t m, int64_t n, const void* X, ql_dtype dtype, int64_t ldx, const double* R,
                                 int64_t ldr, void* Q, int64_t ldq, int32_t* info, void* stream) {
  if (m < 0 || n < 1 || n > kMaxN || (dtype != QL_F64 && dtype != QL_F32) || ldx < (m > 1 ? m : 1) ||
      ldq < (m > 1 ? m : 1) || (m > 0 && (!X || !Q)) || !R || ldr < n)
    return QL_ERR_ARG;
  const size_t el = dtype == QL_F64 ? 8 : 4;
  if ((reinterpret_cast<uintptr_t>(X) % el) || (reinterpret_cast<uintptr_t>(Q) % el) ||
      (reinterpret_cast<uintptr_t>(R) % 8))
    return QL_ERR_ALIGN;
  cudaStream_t st = (cudaStream_t)stream;
  if (dtype == QL_F64) {
    QformArgs<double> a{m, (int)n, static_cast<const double*>(X), ldx, R, ldr, static_cast<double*>(Q), ldq, info, 0};
    return qform_dispatch(a, st);
  }
  QformArgs<float> a{m, (int)n, static_cast<const float*>(X), ldx, R, ldr, static_cast<float*>(Q), ldq, info, 0};
  return qform_dispatch(a, st);
}
