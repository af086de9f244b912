// Dense FP64 sampling Y = A Omega, Z = A^* Psi (Algorithm 2, first block) on the FP64 pipe.
//
// C (N x s) = op(A) B with op(A) = A (Y) or A^T (Z); A row-major N x N (leading dimension
// lda), B and C row-major N x s. One CTA computes a 64 x 128 tile of C (s <= 128 needs one
// column tile); the K loop walks BK = 16 columns (Y) or rows (Z) of A through shared memory,
// so that both products read A in coalesced 128-byte rows. Each thread accumulates a 4 x 8
// register tile. FP64 FMA is the bound: 2 N^2 s FMAs per product.
#include "hbs_internal.cuh"

namespace hbs {
namespace {

constexpr int BM = 64, BN = 128, BK = 16, THREADS = 256;
constexpr int ASTRIDE = BM + 1;   // padded so that the transposing stores of op(A) = A hit
                                  // distinct banks

template <bool TRANS>
__global__ void __launch_bounds__(THREADS)
    sample_gemm_f64(const double* __restrict__ A, int64_t lda, int64_t N,
                    const double* __restrict__ B, int s, double* __restrict__ C) {
  __shared__ double As[BK][ASTRIDE];   // As[k][m] = op(A)[m0 + m][k0 + k]
  __shared__ double Bs[BK][BN];        // Bs[k][c] = B[k0 + k][c0 + c]
  const int tid = threadIdx.x;
  const int tx = tid % 16, ty = tid / 16;
  const int64_t m0 = static_cast<int64_t>(blockIdx.x) * BM;
  const int c0 = blockIdx.y * BN;

  double acc[4][8];
#pragma unroll
  for (int i = 0; i < 4; ++i)
#pragma unroll
    for (int j = 0; j < 8; ++j) acc[i][j] = 0.0;

  for (int64_t k0 = 0; k0 < N; k0 += BK) {
    // op(A) tile: BK x BM = 1024 doubles, 4 per thread
#pragma unroll
    for (int e = 0; e < 4; ++e) {
      const int idx = tid + e * THREADS;
      if (!TRANS) {            // A[m0 + m][k0 + k]: 16 consecutive threads read one row
        const int k = idx % BK, m = idx / BK;
        const int64_t gm = m0 + m, gk = k0 + k;
        As[k][m] = (gm < N && gk < N) ? A[gm * lda + gk] : 0.0;
      } else {                 // A[k0 + k][m0 + m]: 64 consecutive threads read one row
        const int m = idx % BM, k = idx / BM;
        const int64_t gm = m0 + m, gk = k0 + k;
        As[k][m] = (gm < N && gk < N) ? A[gk * lda + gm] : 0.0;
      }
    }
    // B tile: BK x BN = 2048 doubles, 8 per thread
#pragma unroll
    for (int e = 0; e < 8; ++e) {
      const int idx = tid + e * THREADS;
      const int c = idx % BN, k = idx / BN;
      const int64_t gk = k0 + k;
      const int gc = c0 + c;
      Bs[k][c] = (gk < N && gc < s) ? B[gk * s + gc] : 0.0;
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

}  // namespace

cudaError_t launch_sample_dense_f64(const double* A, int64_t lda, int64_t N, const double* Om,
                                    const double* Ps, int s, double* Y, double* Z,
                                    cudaStream_t st) {
  const dim3 grid(static_cast<unsigned>((N + BM - 1) / BM), static_cast<unsigned>((s + BN - 1) / BN));
  sample_gemm_f64<false><<<grid, THREADS, 0, st>>>(A, lda, N, Om, s, Y);
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return e;
  sample_gemm_f64<true><<<grid, THREADS, 0, st>>>(A, lda, N, Ps, s, Z);
  return cudaGetLastError();
}

}  // namespace hbs
