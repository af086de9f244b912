// Arithmetic-pipe throughput probe: the FP64 (DFMA) and FP32 (FFMA) rates of the current GPU,
// measured with CUDA events around kernels that keep every pipe busy. They are the denominators
// of the roofline fractions of the FP64-pipe kernels (products, sweep) and of the double-float
// kernels. Not part of the method; exported for the benchmark (hbs_probe_peaks in hbs.h).
#include <cuda_runtime.h>

#include <vector>

#include "../../include/hbs.h"
#include "hbs_internal.cuh"
#include "tc_ptx.cuh"

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

// tcgen05 MMA issue rate: one thread of warp 1 issues back-to-back M = N = 128, K = 16 MMAs
// (kind::f16, zeroed FP16 operands in shared memory, four accumulators in tensor memory); the
// other eight warps (4 .. 11) do nothing (mode 0), run FP32 TwoSum chains (mode 1), or run them
// only where they do not share warp 1's scheduler, warp % 4 != 1 (mode 2). One CTA per SM.
// cycles[blockIdx.x] = clock cycles from the first issue to the completion of the last MMA.
constexpr int kMmaProbeThreads = 384;
constexpr int kMmaProbeSmem = 200 * 1024;      // one CTA per SM

__global__ void __launch_bounds__(kMmaProbeThreads, 1)
    mma_issue_probe(int iters, int mode, unsigned long long* cycles, float* sink, int* status) {
  extern __shared__ uint8_t smem_raw[];
  uint8_t* smem = smem_raw + ((1024u - (su32(smem_raw) & 1023u)) & 1023u);
  uint8_t* A = smem;                       // 128 x 64 FP16, 128-byte swizzle
  uint8_t* B = smem + 16384;               // 128 x 64 FP16
  __shared__ uint64_t bar;
  __shared__ uint32_t tslot;
  __shared__ volatile int done;
  const int warp = threadIdx.x / 32;
  if (threadIdx.x == 0) {
    mbar_init(&bar, 1);
    done = 0;
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  for (int i = threadIdx.x; i < 32768 / 4; i += blockDim.x) reinterpret_cast<uint32_t*>(smem)[i] = 0u;
  asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
  if (warp == 1) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(
                     su32(&tslot)),
                 "r"(512)
                 : "memory");
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
  }
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  const uint32_t tmem = tslot;
  if (threadIdx.x == 32) {
    const uint64_t ad = sw128_desc(su32(A)), bd = sw128_desc(su32(B));
    const uint32_t idesc = idesc_f16(128, 128);
    const unsigned long long t0 = clock64();
    for (int i = 0; i < iters; ++i) {
#pragma unroll
      for (int kk = 0; kk < 4; ++kk) {
        const uint32_t acc = tmem + static_cast<uint32_t>((i & 3) * 128);
        asm volatile(
            "{\n\t.reg .pred p;\n\tsetp.ne.b32 p, %4, 0;\n\t"
            "tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n\t}" ::"r"(acc),
            "l"(ad + 2 * kk), "l"(bd + 2 * kk), "r"(idesc), "r"(kk)
            : "memory");
      }
    }
    mma_commit(&bar);
    mbar_wait(&bar, 0, status, false);
    cycles[blockIdx.x] = clock64() - t0;
    done = 1;
  } else if (warp >= 4 && (mode == 1 || (mode == 2 && (warp & 3) != 1))) {
    float hi[16], lo[16];
#pragma unroll
    for (int j = 0; j < 16; ++j) {
      hi[j] = 1e-3f * threadIdx.x + j;
      lo[j] = 0.f;
    }
    while (!done) {
#pragma unroll
      for (int j = 0; j < 16; ++j) {              // TwoSum of hi[j] and a neighbour's multiple
        const float v = __fmul_rn(hi[(j + 1) & 15], 1.0001f);
        const float t = __fadd_rn(hi[j], v);
        const float bp = __fsub_rn(t, hi[j]);
        lo[j] = __fadd_rn(lo[j], __fadd_rn(__fsub_rn(hi[j], __fsub_rn(t, bp)), __fsub_rn(v, bp)));
        hi[j] = __fmul_rn(t, 0.5f);
      }
    }
    float acc = 0.f;
#pragma unroll
    for (int j = 0; j < 16; ++j) acc += hi[j] + lo[j];
    if (acc == -1.f) *sink = acc;                  // never true: keeps the chains alive
  }
  tc_fence_before();
  __syncthreads();
  if (warp == 1) {
    tc_fence_after();
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(512)
                 : "memory");
  }
}

}  // namespace
}  // namespace hbs

extern "C" int hbs_probe_mma_issue(double* cycles_per_mma, void* cuda_stream) {
  if (!cycles_per_mma) return HBS_ERR_ARG;
  cudaStream_t st = static_cast<cudaStream_t>(cuda_stream);
  int dev = 0, sms = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e == cudaSuccess) e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  if (e != cudaSuccess) return HBS_ERR_CUDA;
  unsigned long long* cyc = nullptr;
  int* status = nullptr;
  float* sink = nullptr;
  e = cudaMalloc(&cyc, sizeof(unsigned long long) * sms);
  if (e == cudaSuccess) e = cudaMalloc(&status, 2 * sizeof(int));
  if (e == cudaSuccess) e = cudaMalloc(&sink, sizeof(float));
  if (e == cudaSuccess) e = cudaMemsetAsync(status, 0, 2 * sizeof(int), st);
  if (e == cudaSuccess)
    e = cudaFuncSetAttribute(hbs::mma_issue_probe, cudaFuncAttributeMaxDynamicSharedMemorySize,
                             hbs::kMmaProbeSmem);
  constexpr int kIters = 2000;                     // 8000 MMAs per CTA
  std::vector<unsigned long long> h(sms);
  for (int mode = 0; mode < 3 && e == cudaSuccess; ++mode) {
    for (int rep = 0; rep < 2 && e == cudaSuccess; ++rep) {   // the first launch warms up
      hbs::mma_issue_probe<<<sms, hbs::kMmaProbeThreads, hbs::kMmaProbeSmem, st>>>(
          kIters, mode, cyc, sink, status);
      e = cudaGetLastError();
    }
    if (e == cudaSuccess)
      e = cudaMemcpyAsync(h.data(), cyc, sizeof(unsigned long long) * sms, cudaMemcpyDeviceToHost, st);
    if (e == cudaSuccess) e = cudaStreamSynchronize(st);
    double mean = 0.0;
    for (int b = 0; b < sms; ++b) mean += static_cast<double>(h[b]);
    cycles_per_mma[mode] = e == cudaSuccess ? mean / sms / (4.0 * kIters) : 0.0;
  }
  int stat = 0;
  if (e == cudaSuccess) e = cudaMemcpy(&stat, status, sizeof(int), cudaMemcpyDeviceToHost);
  cudaFree(cyc);
  cudaFree(status);
  cudaFree(sink);
  if (e != cudaSuccess) return HBS_ERR_CUDA;
  return (stat & hbs::kStatusTimeout) ? HBS_ERR_TIMEOUT : HBS_OK;
}

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
