// Dense FP64 sampling Y = A Omega, Z = A^* Psi (Algorithm 2, first block) on the FP64 pipe.
//
// C (M x s) = op(A) B with op(A) = A (Y; A stored M x K) or A^T (Z; A stored K x M); A
// row-major with leading dimension lda, B (K x s) and C row-major. One CTA computes a 64 x 128
// tile of C (s <= 128 needs one column tile) over one slice of the reduction; the K loop walks
// BK = 16 columns (Y) or rows (Z) of A through shared memory, so that both products read A in
// coalesced 128-byte rows. Each thread accumulates a 4 x 8 register tile. FP64 FMA is the
// bound: 2 M K s FMAs per product. The reduction is cut into as many slices as make the CTA
// count a whole number of waves (two CTAs per SM), so that no SM idles in a last partial wave;
// the slices' FP64 partials are summed in a fixed order, keeping the result deterministic.
//
// A in page-locked host memory is streamed through the device in row blocks on a second
// stream, each block's copy overlapping the products of the previous one: block b gives the
// rows b of Y and reduction slices of Z = sum_b A_b^* Psi_b; Z's slices are summed in block
// order at the end.
#include <algorithm>
#include <cmath>
#include <mutex>
#include <utility>
#include <vector>

#include "hbs_internal.cuh"

namespace hbs {
namespace {

constexpr int BM = 64, BK = 16, THREADS = 256;   // rows of a tile, reduction step, threads
constexpr int ASTRIDE = BM + 1;   // padded so that the transposing stores of op(A) = A hit
                                  // distinct banks

// TJ = column slots per thread: the CTA's column tile is 8 TJ wide (TJ = ceil(s/8) <= 16, wider s
// in tiles of 128), 8 column lanes x 32 row pairs per CTA. A warp covers 8 columns of each slot,
// so a slot lies wholly inside or wholly past s: s = 120 computes 120 columns, not 128. (Each
// FP64 warp instruction occupies its scheduler's FP64 unit for the same time however many of its
// lanes do useful work, so a half-used slot would cost a whole one.)
template <bool TRANS, int TJ>
__global__ void __launch_bounds__(THREADS, 2)
    sample_gemm_f64(const double* __restrict__ A, int64_t lda, int64_t M, int64_t K,
                    const double* __restrict__ B, int s, double* __restrict__ C, int64_t kslice,
                    int64_t ldc_split) {
  constexpr int TBN = 8 * TJ;
  constexpr int kBLoads = (BK * TBN + THREADS - 1) / THREADS;
  __shared__ double As[BK][ASTRIDE];   // As[k][m] = op(A)[m0 + m][k0 + k]
  __shared__ double Bs[BK][TBN];       // Bs[k][c] = B[k0 + k][c0 + c]
  const int tid = threadIdx.x;
  const int tx = tid % 8, ty = tid / 8;                     // column lane, row pair
  const int64_t m0 = static_cast<int64_t>(blockIdx.x) * BM;
  const int c0 = blockIdx.y * TBN;
  const int64_t kbeg = static_cast<int64_t>(blockIdx.z) * kslice;
  const int64_t kend = min(K, kbeg + kslice);
  C += static_cast<int64_t>(blockIdx.z) * ldc_split;        // this slice's partial (or C itself)

  double acc[2][TJ];
#pragma unroll
  for (int i = 0; i < 2; ++i)
#pragma unroll
    for (int j = 0; j < TJ; ++j) acc[i][j] = 0.0;

  for (int64_t k0 = kbeg; k0 < kend; k0 += BK) {
    // op(A) tile: BK x BM = 1024 doubles, 4 per thread
#pragma unroll
    for (int e = 0; e < 4; ++e) {
      const int idx = tid + e * THREADS;
      if (!TRANS) {            // A[m0 + m][k0 + k]: 16 consecutive threads read one row
        const int k = idx % BK, m = idx / BK;
        const int64_t gm = m0 + m, gk = k0 + k;
        As[k][m] = (gm < M && gk < kend) ? A[gm * lda + gk] : 0.0;
      } else {                 // A[k0 + k][m0 + m]: 64 consecutive threads read one row
        const int m = idx % BM, k = idx / BM;
        const int64_t gm = m0 + m, gk = k0 + k;
        As[k][m] = (gm < M && gk < kend) ? A[gk * lda + gm] : 0.0;
      }
    }
    // B tile: BK x TBN doubles
#pragma unroll
    for (int e = 0; e < kBLoads; ++e) {
      const int idx = tid + e * THREADS;
      if (idx < BK * TBN) {
        const int c = idx % TBN, k = idx / TBN;
        const int64_t gk = k0 + k;
        const int gc = c0 + c;
        Bs[k][c] = (gk < kend && gc < s) ? B[gk * s + gc] : 0.0;
      }
    }
    __syncthreads();
#pragma unroll
    for (int k = 0; k < BK; ++k) {
      double a[2], b[TJ];
#pragma unroll
      for (int i = 0; i < 2; ++i) a[i] = As[k][ty * 2 + i];
#pragma unroll
      for (int j = 0; j < TJ; ++j) b[j] = Bs[k][tx + 8 * j];
#pragma unroll
      for (int i = 0; i < 2; ++i)
#pragma unroll
        for (int j = 0; j < TJ; ++j) acc[i][j] = fma(a[i], b[j], acc[i][j]);
    }
    __syncthreads();
  }
#pragma unroll
  for (int i = 0; i < 2; ++i) {
    const int64_t gm = m0 + ty * 2 + i;
    if (gm >= M) continue;
#pragma unroll
    for (int j = 0; j < TJ; ++j) {
      const int gc = c0 + tx + 8 * j;
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
int reduction_slices(int64_t K, int64_t tiles, int sms) {
  const int64_t slots = 2 * static_cast<int64_t>(sms);
  const int64_t max_slices = std::max<int64_t>(1, K / (64 * BK));
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

int sm_count() {
  int dev = 0, sms = 0;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  return sms > 0 ? sms : 152;
}

// Column slots per thread of the product's tile: 8 TJ >= s up to TJ = 16 (wider s: tiles of 128).
int col_per_thread(int s) { return std::min(16, std::max(1, (s + 7) / 8)); }

// Slices of the reduction and their length (a multiple of BK) for an M x K product.
void plan_slices(int64_t M, int64_t K, int s, int* nslices, int64_t* kslice) {
  const int tbn = 8 * col_per_thread(s);
  const int64_t tiles = ((M + BM - 1) / BM) * ((s + tbn - 1) / tbn);
  const int slices = reduction_slices(K, tiles, sm_count());
  *kslice = ((K + slices - 1) / slices + BK - 1) / BK * BK;
  *nslices = static_cast<int>((K + *kslice - 1) / *kslice);
}

// Launches C (+ z * ldc) = the slices of op(A) B; C is M x s, slice z starts at C + z * ldc.
template <int TJ>
void launch_tj(bool trans, const dim3& grid, cudaStream_t st, const double* A, int64_t lda,
               int64_t M, int64_t K, const double* B, int s, double* C, int64_t kslice,
               int64_t ldc) {
  if (trans) sample_gemm_f64<true, TJ><<<grid, THREADS, 0, st>>>(A, lda, M, K, B, s, C, kslice, ldc);
  else sample_gemm_f64<false, TJ><<<grid, THREADS, 0, st>>>(A, lda, M, K, B, s, C, kslice, ldc);
}

cudaError_t launch_slices(bool trans, const double* A, int64_t lda, int64_t M, int64_t K,
                          const double* B, int s, double* C, int nslices, int64_t kslice,
                          int64_t ldc, cudaStream_t st) {
  const int tj = col_per_thread(s), tbn = 8 * tj;
  const dim3 grid(static_cast<unsigned>((M + BM - 1) / BM), static_cast<unsigned>((s + tbn - 1) / tbn),
                  static_cast<unsigned>(nslices));
  switch (tj) {
    case 1: launch_tj<1>(trans, grid, st, A, lda, M, K, B, s, C, kslice, ldc); break;
    case 2: launch_tj<2>(trans, grid, st, A, lda, M, K, B, s, C, kslice, ldc); break;
    case 3: launch_tj<3>(trans, grid, st, A, lda, M, K, B, s, C, kslice, ldc); break;
    case 4: launch_tj<4>(trans, grid, st, A, lda, M, K, B, s, C, kslice, ldc); break;
    case 5: launch_tj<5>(trans, grid, st, A, lda, M, K, B, s, C, kslice, ldc); break;
    case 6: launch_tj<6>(trans, grid, st, A, lda, M, K, B, s, C, kslice, ldc); break;
    case 7: launch_tj<7>(trans, grid, st, A, lda, M, K, B, s, C, kslice, ldc); break;
    case 8: launch_tj<8>(trans, grid, st, A, lda, M, K, B, s, C, kslice, ldc); break;
    case 9: launch_tj<9>(trans, grid, st, A, lda, M, K, B, s, C, kslice, ldc); break;
    case 10: launch_tj<10>(trans, grid, st, A, lda, M, K, B, s, C, kslice, ldc); break;
    case 11: launch_tj<11>(trans, grid, st, A, lda, M, K, B, s, C, kslice, ldc); break;
    case 12: launch_tj<12>(trans, grid, st, A, lda, M, K, B, s, C, kslice, ldc); break;
    case 13: launch_tj<13>(trans, grid, st, A, lda, M, K, B, s, C, kslice, ldc); break;
    case 14: launch_tj<14>(trans, grid, st, A, lda, M, K, B, s, C, kslice, ldc); break;
    case 15: launch_tj<15>(trans, grid, st, A, lda, M, K, B, s, C, kslice, ldc); break;
    default: launch_tj<16>(trans, grid, st, A, lda, M, K, B, s, C, kslice, ldc); break;
  }
  return cudaGetLastError();
}

// C = op(A) B, through the partial buffer when the reduction is split.
cudaError_t product(bool trans, const double* A, int64_t lda, int64_t M, int64_t K,
                    const double* B, int s, double* C, cudaStream_t st) {
  int nslices;
  int64_t kslice;
  plan_slices(M, K, s, &nslices, &kslice);
  const int64_t count = M * s;
  if (nslices == 1) return launch_slices(trans, A, lda, M, K, B, s, C, 1, kslice, 0, st);
  double* part = nullptr;
  cudaError_t e = partial_buffer(static_cast<size_t>(nslices) * count, &part);
  if (e != cudaSuccess) return e;
  e = launch_slices(trans, A, lda, M, K, B, s, part, nslices, kslice, count, st);
  if (e != cudaSuccess) return e;
  const unsigned rg = static_cast<unsigned>(std::min<int64_t>((count + 255) / 256, 8 * sm_count()));
  sum_slices<<<rg, 256, 0, st>>>(part, nslices, count, C);
  return cudaGetLastError();
}

// ---- host-resident A: per-device staging, copy stream and events ----------------------------

struct HostStream {
  double* stage[2] = {nullptr, nullptr};
  size_t stage_doubles = 0;
  double* zpart = nullptr;
  size_t zpart_doubles = 0;
  cudaStream_t copy = nullptr;
  cudaEvent_t start = nullptr, copied[2] = {nullptr, nullptr}, consumed[2] = {nullptr, nullptr};
};
std::mutex g_host_mutex;
std::vector<HostStream> g_host;

cudaError_t grow(double** p, size_t* have, size_t want) {
  if (*have >= want) return cudaSuccess;
  if (*p) {
    cudaError_t e = cudaDeviceSynchronize();
    if (e != cudaSuccess) return e;
    cudaFree(*p);
    *p = nullptr;
    *have = 0;
  }
  cudaError_t e = cudaMalloc(p, want * sizeof(double));
  if (e == cudaSuccess) *have = want;
  return e;
}

cudaError_t host_stream(size_t stage_doubles, size_t zpart_doubles, HostStream** out) {
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return e;
  std::lock_guard<std::mutex> lock(g_host_mutex);
  if (static_cast<int>(g_host.size()) <= dev) g_host.resize(dev + 1);
  HostStream& h = g_host[dev];
  if (!h.copy) {
    e = cudaStreamCreateWithFlags(&h.copy, cudaStreamNonBlocking);
    if (e == cudaSuccess) e = cudaEventCreateWithFlags(&h.start, cudaEventDisableTiming);
    for (int i = 0; i < 2 && e == cudaSuccess; ++i) {
      e = cudaEventCreateWithFlags(&h.copied[i], cudaEventDisableTiming);
      if (e == cudaSuccess) e = cudaEventCreateWithFlags(&h.consumed[i], cudaEventDisableTiming);
    }
    if (e != cudaSuccess) return e;
  }
  size_t have0 = h.stage_doubles, have1 = h.stage_doubles;
  e = grow(&h.stage[0], &have0, stage_doubles);
  if (e == cudaSuccess) e = grow(&h.stage[1], &have1, stage_doubles);
  if (e != cudaSuccess) return e;
  h.stage_doubles = std::min(have0, have1);
  e = grow(&h.zpart, &h.zpart_doubles, zpart_doubles);
  if (e != cudaSuccess) return e;
  *out = &h;
  return cudaSuccess;
}

}  // namespace

cudaError_t launch_sample_dense_f64(const double* A, int64_t lda, int64_t N, const double* Om,
                                    const double* Ps, int s, double* Y, double* Z,
                                    cudaStream_t st) {
  cudaError_t e = product(false, A, lda, N, N, Om, s, Y, st);
  if (e != cudaSuccess) return e;
  return product(true, A, lda, N, N, Ps, s, Z, st);
}

cudaError_t launch_sample_host_f64(const double* A, int64_t lda, int64_t N, const double* Om,
                                   const double* Ps, int s, double* Y, double* Z,
                                   cudaStream_t st) {
  // Row blocks (multiples of the 64-row tile) doubling from ~N/32 rows up to ~N/4 rows (at most
  // 2 GiB of staging each): the first copy, which nothing hides, stays short, and few blocks are
  // small (a small block's products fill the GPU less well: at N = 32768 the streamed products
  // took 456, 427 and 424 ms with blocks of up to N/16, N/8 and N/4 rows, against 416 ms from
  // device memory).
  const int64_t cap = std::max<int64_t>(BM, (int64_t(1) << 28) / std::max<int64_t>(1, N) / BM * BM);
  const int64_t nb_max = std::min(N, std::max<int64_t>(BM, std::min(((N + 3) / 4 + BM - 1) / BM * BM, cap)));
  std::vector<int64_t> rows_of;
  std::vector<int> zs_of;
  int64_t total_slices = 0;
  for (int64_t r0 = 0, nb = std::min(nb_max, ((N + 31) / 32 + BM - 1) / BM * BM); r0 < N;) {
    const int64_t rows = std::min(nb, N - r0);
    int zs = 0;                                        // Z slices of this block
    int64_t zk = 0;
    plan_slices(N, rows, s, &zs, &zk);
    rows_of.push_back(rows);
    zs_of.push_back(zs);
    total_slices += zs;
    r0 += rows;
    nb = std::min(nb_max, 2 * nb);
  }
  const int64_t count = N * s;
  HostStream* h = nullptr;
  cudaError_t e = host_stream(static_cast<size_t>(nb_max) * N,
                              static_cast<size_t>(total_slices) * count, &h);
  if (e != cudaSuccess) return e;
  e = cudaEventRecord(h->start, st);                   // the stages are free once st is here
  if (e == cudaSuccess) e = cudaStreamWaitEvent(h->copy, h->start, 0);
  int64_t r0 = 0, slice0 = 0;
  for (size_t b = 0; b < rows_of.size() && e == cudaSuccess; ++b) {
    const int slot = static_cast<int>(b & 1);
    const int64_t rows = rows_of[b];
    const int zs = zs_of[b];
    if (b >= 2) e = cudaStreamWaitEvent(h->copy, h->consumed[slot], 0);
    if (e == cudaSuccess)                              // contiguous rows: one 1D copy
      e = lda == N ? cudaMemcpyAsync(h->stage[slot], A + r0 * lda, rows * N * sizeof(double),
                                     cudaMemcpyHostToDevice, h->copy)
                   : cudaMemcpy2DAsync(h->stage[slot], N * sizeof(double), A + r0 * lda,
                                       lda * sizeof(double), N * sizeof(double), rows,
                                       cudaMemcpyHostToDevice, h->copy);
    if (e == cudaSuccess) e = cudaEventRecord(h->copied[slot], h->copy);
    if (e == cudaSuccess) e = cudaStreamWaitEvent(st, h->copied[slot], 0);
    if (e == cudaSuccess) e = product(false, h->stage[slot], N, rows, N, Om, s, Y + r0 * s, st);
    if (e == cudaSuccess) {
      const int64_t zkb = ((rows + zs - 1) / zs + BK - 1) / BK * BK;
      double* zb = h->zpart + static_cast<size_t>(slice0) * count;
      e = launch_slices(true, h->stage[slot], N, N, rows, Ps + r0 * s, s, zb, zs, zkb, count, st);
    }
    if (e == cudaSuccess) e = cudaEventRecord(h->consumed[slot], st);
    r0 += rows;
    slice0 += zs;
  }
  if (e != cudaSuccess) return e;
  const unsigned rg = static_cast<unsigned>(std::min<int64_t>((count + 255) / 256, 8 * sm_count()));
  sum_slices<<<rg, 256, 0, st>>>(h->zpart, static_cast<int>(total_slices), count, Z);
  return cudaGetLastError();
}

}  // namespace hbs
