// Small per-node products of Algorithm 1 (apply): C = op1(A1) B1 [+ op2(A2) B2], one CTA per
// task, one thread per output element with a K loop. The apply of one level is one launch.
// At large N the pass is bound by reading X and writing Out once (HBM); factors are small.
#include "hbs_internal.cuh"

namespace hbs {
namespace {

constexpr int THREADS = 256;

__global__ void __launch_bounds__(THREADS) gemm_tasks_f64(const GemmTask* __restrict__ tasks,
                                                          int ncols) {
  const GemmTask t = tasks[blockIdx.x];
  if (t.ncols > 0) ncols = t.ncols;
  const int total = t.m * ncols;
  for (int e = threadIdx.x; e < total; e += THREADS) {
    const int i = e / ncols, b = e % ncols;
    double acc = 0.0;
    if (t.t1) {
      for (int k = 0; k < t.k1; ++k)
        acc = fma(t.A1[static_cast<size_t>(k) * t.lda1 + i], t.B1[static_cast<size_t>(k) * t.ldb1 + b], acc);
    } else {
      for (int k = 0; k < t.k1; ++k)
        acc = fma(t.A1[static_cast<size_t>(i) * t.lda1 + k], t.B1[static_cast<size_t>(k) * t.ldb1 + b], acc);
    }
    if (t.A2 != nullptr) {
      if (t.t2) {
        for (int k = 0; k < t.k2; ++k)
          acc = fma(t.A2[static_cast<size_t>(k) * t.lda2 + i], t.B2[static_cast<size_t>(k) * t.ldb2 + b], acc);
      } else {
        for (int k = 0; k < t.k2; ++k)
          acc = fma(t.A2[static_cast<size_t>(i) * t.lda2 + k], t.B2[static_cast<size_t>(k) * t.ldb2 + b], acc);
      }
    }
    t.C[static_cast<size_t>(i) * t.ldc + b] = acc;
  }
}

}  // namespace

cudaError_t launch_gemm_tasks_f64(const GemmTask* d_tasks, int ntasks, int ncols, cudaStream_t st) {
  if (ntasks <= 0) return cudaSuccess;
  gemm_tasks_f64<<<ntasks, THREADS, 0, st>>>(d_tasks, ncols);
  return cudaGetLastError();
}

}  // namespace hbs
