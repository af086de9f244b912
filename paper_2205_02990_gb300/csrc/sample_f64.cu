// Dense FP64 sampling Y = A Omega, Z = A^* Psi (Algorithm 2, first block) on the FP64 pipe.
//
// C (N x s) = op(A) B with op(A) = A (Y) or A^T (Z); A row-major N x N (leading dimension
// lda), B and C row-major N x s. One CTA computes a 64 x 128 tile of C (s <= 128 needs one
// column tile) over one slice of the reduction; the K loop walks BK = 16 columns (Y) or rows
// (Z) of A through shared memory, so that both products read A in coalesced 128-byte rows.
// Each thread accumulates a 4 x 8 register tile. FP64 FMA is the bound: 2 N^2 s FMAs per
// product. The reduction is cut into as many slices as make the CTA count a whole number of
// waves (two CTAs per SM), so that no SM idles in a last partial wave; the slices' FP64
// partials are summed in a fixed order, keeping the result deterministic.
#include <algorithm>
#include <cmath>
#include <mutex>
#include <utility>
#include <vector>

#include "hbs_internal.cuh"

namespace hbs {
namespace {

constexpr int BM = 64, BN = 128, BK = 16, THREADS = 256;
constexpr int ASTRIDE = BM + 1;   // padded so that the transposing stores of op(A) = A hit
                                  // distinct banks

template <bool TRANS>
__global__ void __launch_bounds__(THREADS)
    sample_gemm_f64(const double* __restrict__ A, int64_t lda, int64_t N,
                    const double* __restrict__ B, int s, double* __restrict__ C, int64_t kslice,
                    int64_t ldc_split) {
  __shared__ double As[BK][ASTRIDE];   // As[k][m] = op(A)[m0 + m][k0 + k]
  __shared__ double Bs[BK][BN];        // Bs[k][c] = B[k0 + k][c0 + c]
  const int tid = threadIdx.x;
  const int tx = tid % 16, ty = tid / 16;
  const int64_t m0 = static_cast<int64_t>(blockIdx.x) * BM;
  const int c0 = blockIdx.y * BN;
  const int64_t kbeg = static_cast<int64_t>(blockIdx.z) * kslice;
  const int64_t kend = min(N, kbeg + kslice);
  C += static_cast<int64_t>(blockIdx.z) * ldc_split;        // this slice's partial (or C itself)

  double acc[4][8];
#pragma unroll
  for (int i = 0; i < 4; ++i)
#pragma unroll
    for (int j = 0; j < 8; ++j) acc[i][j] = 0.0;

  for (int64_t k0 = kbeg; k0 < kend; k0 += BK) {
    // op(A) tile: BK x BM = 1024 doubles, 4 per thread
#pragma unroll
    for (int e = 0; e < 4; ++e) {
      const int idx = tid + e * THREADS;
      if (!TRANS) {            // A[m0 + m][k0 + k]: 16 consecutive threads read one row
        const int k = idx % BK, m = idx / BK;
        const int64_t gm = m0 + m, gk = k0 + k;
        As[k][m] = (gm < N && gk < kend) ? A[gm * lda + gk] : 0.0;
      } else {                 // A[k0 + k][m0 + m]: 64 consecutive threads read one row
        const int m = idx % BM, k = idx / BM;
        const int64_t gm = m0 + m, gk = k0 + k;
        As[k][m] = (gm < N && gk < kend) ? A[gk * lda + gm] : 0.0;
      }
    }
    // B tile: BK x BN = 2048 doubles, 8 per thread
#pragma unroll
    for (int e = 0; e < 8; ++e) {
      const int idx = tid + e * THREADS;
      const int c = idx % BN, k = idx / BN;
      const int64_t gk = k0 + k;
      const int gc = c0 + c;
      Bs[k][c] = (gk < kend && gc < s) ? B[gk * s + gc] : 0.0;
    }
    __syncthreads();
#pragma unroll
    for (int k = 0; k < BK; ++k) {
      double a[4], b[8];
#pragma unroll
      for (int i = 0; i < 4; ++i) a[i] = As[k][ty * 4 + i];
#pragma unroll
      for (int j = 0; j < 8; ++j) b[j] = Bs[k][tx + 16 * j];
#pragma unroll
      for (int i = 0; i < 4; ++i)
#pragma unroll
        for (int j = 0; j < 8; ++j) acc[i][j] = fma(a[i], b[j], acc[i][j]);
    }
    __syncthreads();
  }
#pragma unroll
  for (int i = 0; i < 4; ++i) {
    const int64_t gm = m0 + ty * 4 + i;
    if (gm >= N) continue;
#pragma unroll
    for (int j = 0; j < 8; ++j) {
      const int gc = c0 + tx + 16 * j;
      if (gc < s) C[gm * s + gc] = acc[i][j];
    }
  }
}

// C = sum over slices of the partials, in slice order.
__global__ void sum_slices(const double* __restrict__ part, int slices, int64_t count,
                           double* __restrict__ C) {
  for (int64_t i = blockIdx.x * static_cast<int64_t>(blockDim.x) + threadIdx.x; i < count;
       i += static_cast<int64_t>(gridDim.x) * blockDim.x) {
    double acc = 0.0;
    for (int z = 0; z < slices; ++z) acc += part[z * count + i];
    C[i] = acc;
  }
}

// Per-device buffer for the slices' partials, grown on demand.
std::mutex g_part_mutex;
std::vector<std::pair<double*, size_t>> g_part;

cudaError_t partial_buffer(size_t doubles, double** out) {
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return e;
  std::lock_guard<std::mutex> lock(g_part_mutex);
  if (static_cast<int>(g_part.size()) <= dev) g_part.resize(dev + 1, {nullptr, 0});
  auto& b = g_part[dev];
  if (b.second < doubles) {
    if (b.first) {
      e = cudaDeviceSynchronize();
      if (e != cudaSuccess) return e;
      cudaFree(b.first);
      b = {nullptr, 0};
    }
    e = cudaMalloc(&b.first, doubles * sizeof(double));
    if (e != cudaSuccess) return e;
    b.second = doubles;
  }
  *out = b.first;
  return cudaSuccess;
}

// Reduction slices that make tiles x slices a whole number of waves of 2 x SM CTAs (about 16
// waves; a slice keeps at least 64 reduction steps).
int reduction_slices(int64_t N, int64_t tiles, int sms) {
  const int64_t slots = 2 * static_cast<int64_t>(sms);
  const int64_t max_slices = std::max<int64_t>(1, N / (64 * BK));
  int best = 1;
  double best_eff = 0.0;
  for (int64_t z = 1; z <= std::min<int64_t>(max_slices, 64); ++z) {
    const int64_t ctas = tiles * z;
    const double waves = static_cast<double>(ctas) / slots;
    const double eff = waves / std::ceil(waves);
    if (eff > best_eff + 1e-3 || (eff > best_eff - 1e-3 && ctas <= 16 * slots && z < best)) {
      if (eff > best_eff + 1e-3 || z < best) {
        best_eff = eff;
        best = static_cast<int>(z);
      }
    }
    if (best_eff > 0.985 && ctas >= 8 * slots) break;
  }
  return best;
}

}  // namespace

cudaError_t launch_sample_dense_f64(const double* A, int64_t lda, int64_t N, const double* Om,
                                    const double* Ps, int s, double* Y, double* Z,
                                    cudaStream_t st) {
  int dev = 0, sms = 0;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  if (sms <= 0) sms = 152;
  const int64_t mt = (N + BM - 1) / BM, nt = (s + BN - 1) / BN;
  const int slices = reduction_slices(N, mt * nt, sms);
  const int64_t kslice = ((N + slices - 1) / slices + BK - 1) / BK * BK;
  const int nslices = static_cast<int>((N + kslice - 1) / kslice);
  const dim3 grid(static_cast<unsigned>(mt), static_cast<unsigned>(nt), static_cast<unsigned>(nslices));
  const int64_t count = N * s;
  double* part = nullptr;
  if (nslices > 1) {
    cudaError_t e = partial_buffer(static_cast<size_t>(nslices) * count, &part);
    if (e != cudaSuccess) return e;
  }
  const unsigned rg = static_cast<unsigned>(std::min<int64_t>((count + 255) / 256, 8 * sms));
  for (int which = 0; which < 2; ++which) {
    double* C = which ? Z : Y;
    double* dst = nslices > 1 ? part : C;
    if (which == 0)
      sample_gemm_f64<false><<<grid, THREADS, 0, st>>>(A, lda, N, Om, s, dst, kslice, count);
    else
      sample_gemm_f64<true><<<grid, THREADS, 0, st>>>(A, lda, N, Ps, s, dst, kslice, count);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    if (nslices > 1) {
      sum_slices<<<rg, 256, 0, st>>>(part, nslices, count, C);
      e = cudaGetLastError();
      if (e != cudaSuccess) return e;
    }
  }
  return cudaSuccess;
}

}  // namespace hbs
