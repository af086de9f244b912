// Arithmetic-pipe throughput probe: the FP64 (DFMA) and FP32 (FFMA) rates of the current GPU,
// measured with CUDA events around kernels that keep every pipe busy. They are the denominators
// of the roofline fractions of the FP64-pipe kernels (products, sweep) and of the double-float
// kernels. Not part of the method; exported for the benchmark (hbs_probe_peaks in hbs.h).
#include <cuda_runtime.h>

#include "../../include/hbs.h"
#include "hbs_internal.cuh"

namespace hbs {
namespace {

constexpr int kProbeThreads = 256;
constexpr int kChains = 8;          // independent multiply-add chains per thread

template <class Real>
__global__ void __launch_bounds__(kProbeThreads) fma_probe(Real seed, int iters, Real* sink) {
  Real a[kChains];
#pragma unroll
  for (int c = 0; c < kChains; ++c) a[c] = seed + Real(threadIdx.x + c);
  const Real m = Real(0.999), d = Real(0.001);
#pragma unroll 4
  for (int i = 0; i < iters; ++i)
#pragma unroll
    for (int c = 0; c < kChains; ++c) a[c] = fma(a[c], m, d);
  Real acc = 0;
#pragma unroll
  for (int c = 0; c < kChains; ++c) acc += a[c];
  if (acc == Real(-1)) *sink = acc;   // never true: keeps the chains alive
}

// The FP64 tensor instruction (DMMA, mma.sync m8n8k4 with FP64 operands): 2 x 8 x 8 x 4 = 512
// flops per warp instruction, kChains independent accumulators per warp.
__global__ void __launch_bounds__(kProbeThreads) dmma_probe(double seed, int iters, double* sink) {
  double c[kChains][2];
#pragma unroll
  for (int k = 0; k < kChains; ++k) c[k][0] = c[k][1] = seed + threadIdx.x + k;
  const double a = 0.999, b = 0.5;
#pragma unroll 2
  for (int i = 0; i < iters; ++i)
#pragma unroll
    for (int k = 0; k < kChains; ++k)
      asm volatile("mma.sync.aligned.m8n8k4.row.col.f64.f64.f64.f64 {%0, %1}, {%2}, {%3}, {%0, %1};"
                   : "+d"(c[k][0]), "+d"(c[k][1])
                   : "d"(a), "d"(b));
  double acc = 0;
#pragma unroll
  for (int k = 0; k < kChains; ++k) acc += c[k][0] + c[k][1];
  if (acc == -1.0) *sink = acc;   // never true: keeps the chains alive
}

template <class Real>
cudaError_t time_probe(int blocks, int iters, Real* sink, cudaStream_t st, double* tflops) {
  cudaEvent_t e0, e1;
  cudaError_t e = cudaEventCreate(&e0);
  if (e == cudaSuccess) e = cudaEventCreate(&e1);
  if (e != cudaSuccess) return e;
  fma_probe<Real><<<blocks, kProbeThreads, 0, st>>>(Real(1), iters, sink);   // warm-up
  e = cudaEventRecord(e0, st);
  constexpr int kReps = 5;
  for (int i = 0; i < kReps && e == cudaSuccess; ++i) {
    fma_probe<Real><<<blocks, kProbeThreads, 0, st>>>(Real(1), iters, sink);
    e = cudaGetLastError();
  }
  if (e == cudaSuccess) e = cudaEventRecord(e1, st);
  if (e == cudaSuccess) e = cudaEventSynchronize(e1);
  float ms = 0.f;
  if (e == cudaSuccess) e = cudaEventElapsedTime(&ms, e0, e1);
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  const double flops = 2.0 * kReps * double(blocks) * kProbeThreads * kChains * iters;
  *tflops = e == cudaSuccess ? flops / (ms * 1e-3) / 1e12 : 0.0;
  return e;
}

cudaError_t time_dmma(int blocks, int iters, double* sink, cudaStream_t st, double* tflops) {
  cudaEvent_t e0, e1;
  cudaError_t e = cudaEventCreate(&e0);
  if (e == cudaSuccess) e = cudaEventCreate(&e1);
  if (e != cudaSuccess) return e;
  dmma_probe<<<blocks, kProbeThreads, 0, st>>>(1.0, iters, sink);   // warm-up
  e = cudaEventRecord(e0, st);
  constexpr int kReps = 5;
  for (int i = 0; i < kReps && e == cudaSuccess; ++i) {
    dmma_probe<<<blocks, kProbeThreads, 0, st>>>(1.0, iters, sink);
    e = cudaGetLastError();
  }
  if (e == cudaSuccess) e = cudaEventRecord(e1, st);
  if (e == cudaSuccess) e = cudaEventSynchronize(e1);
  float ms = 0.f;
  if (e == cudaSuccess) e = cudaEventElapsedTime(&ms, e0, e1);
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  const double flops = 512.0 * kReps * double(blocks) * (kProbeThreads / 32) * kChains * iters;
  *tflops = e == cudaSuccess ? flops / (ms * 1e-3) / 1e12 : 0.0;
  return e;
}

}  // namespace
}  // namespace hbs

extern "C" int hbs_probe_dmma(double* tflops, void* cuda_stream) {
  if (!tflops) return HBS_ERR_ARG;
  int dev = 0, sms = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e == cudaSuccess) e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  if (e != cudaSuccess) return HBS_ERR_CUDA;
  void* sink = nullptr;
  e = cudaMalloc(&sink, 16);
  if (e != cudaSuccess) return HBS_ERR_NOMEM;
  // 8 CTAs of 8 warps per SM, 8 independent accumulators per warp (~60 ms per timed launch)
  e = hbs::time_dmma(8 * sms, 16, static_cast<double*>(sink), static_cast<cudaStream_t>(cuda_stream), tflops);
  cudaFree(sink);
  return e == cudaSuccess ? HBS_OK : HBS_ERR_CUDA;
}

extern "C" int hbs_probe_peaks(double* fp64_tflops, double* fp32_tflops, void* cuda_stream) {
  if (!fp64_tflops || !fp32_tflops) return HBS_ERR_ARG;
  cudaStream_t st = static_cast<cudaStream_t>(cuda_stream);
  int dev = 0, sms = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e == cudaSuccess) e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  if (e != cudaSuccess) return HBS_ERR_CUDA;
  void* sink = nullptr;
  e = cudaMalloc(&sink, 16);
  if (e != cudaSuccess) return HBS_ERR_NOMEM;
  // 8 CTAs of 256 threads per SM: 64 warps, 8 chains each, enough to hide both pipes' latency
  // (about 40 ms of work per timed launch on each pipe)
  e = hbs::time_probe<double>(8 * sms, 2048, static_cast<double*>(sink), st, fp64_tflops);
  if (e == cudaSuccess)
    e = hbs::time_probe<float>(8 * sms, 2048 * 64, static_cast<float*>(sink), st, fp32_tflops);
  cudaFree(sink);
  return e == cudaSuccess ? HBS_OK : HBS_ERR_CUDA;
}
