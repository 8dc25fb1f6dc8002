// Compute-pipe throughput of the current GPU, measured with long streams of independent
// multiply-adds: the denominators of the roofline of the kernels that are bound by
// arithmetic rather than by HBM (double-float arithmetic on the FP32 pipes, native FP64,
// FP64 tensor-core MMA).  Measurement support, not part of the paper's method.
//
// Each kernel runs a fixed number of iterations over 8 independent accumulators per thread
// (enough instruction-level parallelism to cover the pipe latency) on 4 CTAs of 256
// threads per SM, and writes its accumulators to global memory so that nothing is
// optimised away.  The host times each kernel with CUDA events on the caller's stream after
// one warm-up launch.
#include <cuda_runtime.h>

#include "common.cuh"
#include "internal.h"

namespace ql {

constexpr int kPeakThreads = 256;
constexpr int kPeakCtasPerSm = 4;

__global__ void __launch_bounds__(kPeakThreads) peak_fp32_kernel(float* out, int iters, float x, float y) {
  float a[8];
#pragma unroll
  for (int k = 0; k < 8; ++k) a[k] = (float)(threadIdx.x + k);
#pragma unroll 1
  for (int i = 0; i < iters; ++i) {
#pragma unroll
    for (int r = 0; r < 16; ++r)
#pragma unroll
      for (int k = 0; k < 8; ++k) a[k] = __fmaf_rn(a[k], x, y);
  }
  float s = 0.0f;
#pragma unroll
  for (int k = 0; k < 8; ++k) s += a[k];
  out[blockIdx.x * blockDim.x + threadIdx.x] = s;
}

__global__ void __launch_bounds__(kPeakThreads) peak_fp64_kernel(double* out, int iters, double x, double y) {
  double a[8];
#pragma unroll
  for (int k = 0; k < 8; ++k) a[k] = (double)(threadIdx.x + k);
#pragma unroll 1
  for (int i = 0; i < iters; ++i) {
#pragma unroll
    for (int r = 0; r < 16; ++r)
#pragma unroll
      for (int k = 0; k < 8; ++k) a[k] = fma(a[k], x, y);
  }
  double s = 0.0;
#pragma unroll
  for (int k = 0; k < 8; ++k) s += a[k];
  out[blockIdx.x * blockDim.x + threadIdx.x] = s;
}

// The double-float multiply-accumulate of the Householder and Gram loops (ArithDF::acc_fma),
// 2 FP64-equivalent flops each.
__global__ void __launch_bounds__(kPeakThreads) peak_df_kernel(float* out, int iters, float xh, float xl) {
  ArithDF::Acc a[8];
  const df x{xh, xl};
#pragma unroll
  for (int k = 0; k < 8; ++k) a[k] = ArithDF::Acc{(float)(threadIdx.x + k), 0.0f};
  df y[8];
#pragma unroll
  for (int k = 0; k < 8; ++k) y[k] = df{1.0f + 0x1p-20f * (float)k, 0x1p-30f};
#pragma unroll 1
  for (int i = 0; i < iters; ++i) {
#pragma unroll
    for (int r = 0; r < 4; ++r)
#pragma unroll
      for (int k = 0; k < 8; ++k) ArithDF::acc_fma(a[k], x, y[k]);
  }
  float s = 0.0f;
#pragma unroll
  for (int k = 0; k < 8; ++k) s += a[k].hi + a[k].lo;
  out[blockIdx.x * blockDim.x + threadIdx.x] = s;
}

// Packed FP32 FMA (fma.rn.f32x2: two lanes per instruction, sm_100 and later).
__global__ void __launch_bounds__(kPeakThreads) peak_fp32x2_kernel(float* out, int iters, float xs, float ys) {
  unsigned long long a[8], x, y;
  asm("mov.b64 %0, {%1, %2};" : "=l"(x) : "f"(xs), "f"(xs));
  asm("mov.b64 %0, {%1, %2};" : "=l"(y) : "f"(ys), "f"(ys));
#pragma unroll
  for (int k = 0; k < 8; ++k) {
    const float t = (float)(threadIdx.x + k);
    asm("mov.b64 %0, {%1, %2};" : "=l"(a[k]) : "f"(t), "f"(t));
  }
#pragma unroll 1
  for (int i = 0; i < iters; ++i) {
#pragma unroll
    for (int r = 0; r < 16; ++r)
#pragma unroll
      for (int k = 0; k < 8; ++k) asm volatile("fma.rn.f32x2 %0, %0, %1, %2;" : "+l"(a[k]) : "l"(x), "l"(y));
  }
  float s = 0.0f;
#pragma unroll
  for (int k = 0; k < 8; ++k) {
    float lo, hi;
    asm("mov.b64 {%0, %1}, %2;" : "=f"(lo), "=f"(hi) : "l"(a[k]));
    s += lo + hi;
  }
  out[blockIdx.x * blockDim.x + threadIdx.x] = s;
}

// FP64 tensor-core MMA (mma.sync m8n8k4, 512 flops per warp instruction), 4 independent
// accumulator tiles per warp.
__global__ void __launch_bounds__(kPeakThreads) peak_dmma_kernel(double* out, int iters) {
  double acc[4][2];
#pragma unroll
  for (int k = 0; k < 4; ++k) acc[k][0] = acc[k][1] = 0.0;
  const double a = 1.0 + 1e-9 * threadIdx.x, b = 1.0 - 1e-9 * threadIdx.x;
#pragma unroll 1
  for (int i = 0; i < iters; ++i) {
#pragma unroll
    for (int r = 0; r < 8; ++r)
#pragma unroll
      for (int k = 0; k < 4; ++k)
        asm volatile("mma.sync.aligned.m8n8k4.row.col.f64.f64.f64.f64 {%0,%1}, {%2}, {%3}, {%0,%1};\n"
                     : "+d"(acc[k][0]), "+d"(acc[k][1])
                     : "d"(a), "d"(b));
  }
  double s = 0.0;
#pragma unroll
  for (int k = 0; k < 4; ++k) s += acc[k][0] + acc[k][1];
  out[blockIdx.x * blockDim.x + threadIdx.x] = s;
}

}  // namespace ql

using namespace ql;

extern "C" ql_status ql_measure_peaks(double* out, void* stream_) {
  if (!out) return QL_ERR_ARG;
  cudaStream_t stream = (cudaStream_t)stream_;
  const int grid = device_sm_count() * kPeakCtasPerSm;
  const size_t nthr = (size_t)grid * kPeakThreads;
  void* buf = nullptr;
  if (cudaMalloc(&buf, nthr * sizeof(double)) != cudaSuccess) return QL_ERR_CUDA;
  cudaEvent_t e0 = nullptr, e1 = nullptr;
  ql_status st = QL_OK;
  if (cudaEventCreate(&e0) != cudaSuccess || cudaEventCreate(&e1) != cudaSuccess) st = QL_ERR_CUDA;
  // (flops per thread and iteration, iterations): each timed launch runs a few tens of ms
  auto timed = [&](auto launch, double flops_per_thread_iter, int iters) -> double {
    launch(iters / 8);  // warm-up
    cudaEventRecord(e0, stream);
    launch(iters);
    cudaEventRecord(e1, stream);
    if (cudaEventSynchronize(e1) != cudaSuccess) return -1.0;
    float ms = 0.0f;
    cudaEventElapsedTime(&ms, e0, e1);
    count_launch();
    count_launch();
    return flops_per_thread_iter * iters * (double)nthr / (ms * 1e-3) / 1e12;
  };
  if (st == QL_OK) {
    out[0] = timed([&](int it) { peak_fp32_kernel<<<grid, kPeakThreads, 0, stream>>>((float*)buf, it, 0.999f, 1e-3f); },
                   2.0 * 16 * 8, 40000);
    out[1] = timed([&](int it) { peak_fp64_kernel<<<grid, kPeakThreads, 0, stream>>>((double*)buf, it, 0.999, 1e-3); },
                   2.0 * 16 * 8, 1000);
    out[2] = timed([&](int it) { peak_dmma_kernel<<<grid, kPeakThreads, 0, stream>>>((double*)buf, it); },
                   512.0 / 32 * 8 * 4, 500);
    out[3] = timed([&](int it) { peak_df_kernel<<<grid, kPeakThreads, 0, stream>>>((float*)buf, it, 0.999f, 1e-9f); },
                   2.0 * 4 * 8, 20000);
    out[4] = timed([&](int it) { peak_fp32x2_kernel<<<grid, kPeakThreads, 0, stream>>>((float*)buf, it, 0.999f, 1e-3f); },
                   2.0 * 2 * 16 * 8, 40000);
    if (cudaGetLastError() != cudaSuccess) st = QL_ERR_CUDA;
    for (int i = 0; i < 5; ++i)
      if (!(out[i] > 0.0)) st = QL_ERR_CUDA;
  }
  if (e0) cudaEventDestroy(e0);
  if (e1) cudaEventDestroy(e1);
  cudaFree(buf);
  return st;
}
