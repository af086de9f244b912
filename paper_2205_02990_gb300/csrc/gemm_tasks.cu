// Small per-node products of Algorithm 1 (apply): C = op1(A1) B1 [+ op2(A2) B2]. The apply of
// one level is one launch.
//
// Wide right-hand sides (more than kSkinny columns): one CTA per task, one thread per output
// element with a K loop; the products then bound the pass on the FP64 pipe (measured at 93 - 94 %
// of it for 16 and 150 columns).
//
// Skinny right-hand sides (1 .. kSkinny columns, a matvec and its neighbours): every factor entry
// is used by at most kSkinny multiply-adds, so the pass is bound by the FP64 pipe (one DFMA per
// 8-byte entry is slower on GB300 than reading the entry from HBM), provided the factor, read
// once from HBM, arrives fast enough: a warp owns 32 rows of C with all their columns and reads
// the factor coalesced in either storage order (below).
#include <algorithm>

#include "hbs_internal.cuh"

namespace hbs {
namespace {

constexpr int THREADS = 256;
constexpr int kSkinny = 4;          // widest right-hand side of the skinny path

// acc[b] += sum_k op(A)[i][k] B[k][b] over k < K for row i = i0 + lane (< m) of this warp's 32
// rows. The additions run in k order, as in the wide path, so both give the same bits.
// op(A) = A^* (entry (i, k) at A[k][i]) is read coalesced along the rows, kUnroll loads ahead of
// their multiply-adds (the factor is read once from HBM). op(A) = A (entry at A[i][k]) would have
// each lane walk its own row, one cache line per lane per load (measured: long-scoreboard stalls,
// the FP64 pipe 55 % busy); instead the warp brings 32 x 32 blocks through two shared-memory
// tiles, one coalesced row segment per copy, the next block in flight while one is used. NC (the
// columns) is a template parameter, so that no multiply-add is issued for an absent column
// (predicated ones ran 2.4x slower).
constexpr int kUnroll = 8;
template <int NC>
__device__ __forceinline__ void skinny_term(const double* __restrict__ A, int lda, int t, int K,
                                            const double* __restrict__ B, int ldb, int m, int i0,
                                            double* tile, double (&acc)[NC]) {
  const int lane = threadIdx.x % 32, i = i0 + lane;
  if (t) {
    if (i >= m) return;
    const double* a0 = A + i;
    int k = 0;
    for (; k + kUnroll <= K; k += kUnroll) {
      double a[kUnroll];
#pragma unroll
      for (int u = 0; u < kUnroll; ++u) a[u] = a0[static_cast<size_t>(k + u) * lda];
#pragma unroll
      for (int u = 0; u < kUnroll; ++u)
#pragma unroll
        for (int b = 0; b < NC; ++b) acc[b] = fma(a[u], B[static_cast<size_t>(k + u) * ldb + b], acc[b]);
    }
    for (; k < K; ++k) {
      const double a = a0[static_cast<size_t>(k) * lda];
#pragma unroll
      for (int b = 0; b < NC; ++b) acc[b] = fma(a, B[static_cast<size_t>(k) * ldb + b], acc[b]);
    }
    return;
  }
  // two tiles: the next 32 x 32 block streams in by asynchronous copies while this one is used
  const int rows = min(32, m - i0);
  auto fetch = [&](int k0, double* tl) {
    const int kw = min(32, K - k0);
    if (lane < kw) {
#pragma unroll 8
      for (int rr = 0; rr < rows; ++rr)
        asm volatile("cp.async.ca.shared.global [%0], [%1], 8;" ::"r"(
                         static_cast<uint32_t>(__cvta_generic_to_shared(tl + rr * 33 + lane))),
                     "l"(A + static_cast<size_t>(i0 + rr) * lda + k0 + lane)
                     : "memory");
    }
    asm volatile("cp.async.commit_group;" ::: "memory");
  };
  __syncwarp();
  fetch(0, tile);
  for (int k0 = 0, c = 0; k0 < K; k0 += 32, ++c) {
    double* cur = tile + (c & 1) * 32 * 33;
    if (k0 + 32 < K) {
      fetch(k0 + 32, tile + ((c + 1) & 1) * 32 * 33);
      asm volatile("cp.async.wait_group 1;" ::: "memory");
    } else {
      asm volatile("cp.async.wait_group 0;" ::: "memory");
    }
    __syncwarp();
    const int kw = min(32, K - k0);
    if (i < m)
      for (int k = 0; k < kw; ++k) {
        const double a = cur[lane * 33 + k];
#pragma unroll
        for (int b = 0; b < NC; ++b) acc[b] = fma(a, B[static_cast<size_t>(k0 + k) * ldb + b], acc[b]);
      }
    __syncwarp();                            // before the tile is refilled
  }
}

// A launch whose tasks are all skinny: each warp takes 32 rows of a task (a task of m rows
// occupies ceil(m / 32) warp slots), slots grid-strided over a few CTAs per SM. (One CTA per
// task, at ~260,000 tasks per apply, paid the start-up of a CTA, the load of its task and the
// first memory latency each time.)
constexpr int kSkinnyThreads = 64;      // two warps: 2 x 2 tiles of 32 x 33 doubles
template <int NC>
__global__ void __launch_bounds__(kSkinnyThreads)
    gemm_tasks_skinny(const GemmTask* __restrict__ tasks, int ntasks, int slots_per_task) {
  __shared__ double tiles[kSkinnyThreads / 32][2 * 32 * 33];
  const int warp = threadIdx.x / 32, lane = threadIdx.x % 32;
  double* tile = tiles[warp];
  const long long nslots = static_cast<long long>(ntasks) * slots_per_task;
  for (long long sl = static_cast<long long>(blockIdx.x) * (kSkinnyThreads / 32) + warp; sl < nslots;
       sl += static_cast<long long>(gridDim.x) * (kSkinnyThreads / 32)) {
    const GemmTask t = tasks[sl / slots_per_task];
    for (int i0 = 32 * static_cast<int>(sl % slots_per_task); i0 < t.m; i0 += 32 * slots_per_task) {
      double acc[NC];
#pragma unroll
      for (int b = 0; b < NC; ++b) acc[b] = 0.0;
      skinny_term<NC>(t.A1, t.lda1, t.t1, t.k1, t.B1, t.ldb1, t.m, i0, tile, acc);
      if (t.A2 != nullptr) skinny_term<NC>(t.A2, t.lda2, t.t2, t.k2, t.B2, t.ldb2, t.m, i0, tile, acc);
      const int i = i0 + lane;
      if (i < t.m) {
#pragma unroll
        for (int b = 0; b < NC; ++b) t.C[static_cast<size_t>(i) * t.ldc + b] = acc[b];
      }
    }
  }
}

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

// One task of Algorithm 1's work list per thread (layout in hbs_internal.cuh).
__global__ void build_apply_tasks(const ApplyNode* __restrict__ nodes, int L, int r, int64_t N,
                                  int trans, int c, const double* arena, const double* X,
                                  double* Out, double* ws, GemmTask* __restrict__ out) {
  const int64_t up = (L == 0) ? 0 : (int64_t(2) << L) - 2;          // upward tasks
  const int64_t total = (L == 0) ? 1 : up + (int64_t(2) << L) - 1;
  const int64_t i = static_cast<int64_t>(blockIdx.x) * blockDim.x + threadIdx.x;
  if (i >= total) return;
  const int64_t rc = static_cast<int64_t>(r) * c;
  auto qhat = [&](int64_t t) { return ws + (t - 2) * rc; };
  auto uhat = [&](int64_t t) { return ws + up * rc + (t - 2) * rc; };
  GemmTask g{};
  if (L == 0) {                                                      // A = D
    g.A1 = arena + nodes[1].oD; g.lda1 = static_cast<int>(N); g.t1 = trans;
    g.k1 = static_cast<int>(N); g.m = static_cast<int>(N);
    g.B1 = X; g.ldb1 = c; g.C = Out; g.ldc = c;
  } else if (i < up) {                                               // upward: q-hat_t = V_t^* ..
    int l = L;
    while (i >= (int64_t(2) << L) - (int64_t(1) << l)) --l;          // levels L, L-1, .. in order
    const int64_t t = (int64_t(1) << l) + (i - ((int64_t(2) << L) - (int64_t(2) << l)));
    const ApplyNode nd = nodes[t];
    g.A1 = arena + (trans ? nd.oU : nd.oV); g.lda1 = r; g.t1 = 1; g.k1 = nd.n; g.m = r;
    g.B1 = (l == L) ? X + nd.off * c : qhat(2 * t);
    g.ldb1 = c; g.C = qhat(t); g.ldc = c;
  } else {                                                           // downward, node t = j + 1
    const int64_t t = i - up + 1;
    const int l = 63 - __clzll(static_cast<long long>(t));
    const ApplyNode nd = nodes[t];
    if (l == 0) {
      g.A1 = arena + nd.oD; g.lda1 = nd.n; g.t1 = trans; g.k1 = nd.n; g.m = nd.n;
      g.B1 = qhat(2); g.ldb1 = c; g.C = uhat(2); g.ldc = c;
    } else {
      g.A1 = arena + (trans ? nd.oV : nd.oU); g.lda1 = r; g.t1 = 0; g.k1 = r; g.m = nd.n;
      g.B1 = uhat(t); g.ldb1 = c;
      g.A2 = arena + nd.oD; g.lda2 = nd.n; g.t2 = trans; g.k2 = nd.n;
      if (l < L) {
        g.B2 = qhat(2 * t); g.ldb2 = c; g.C = uhat(2 * t); g.ldc = c;
      } else {
        g.B2 = X + nd.off * c; g.ldb2 = c; g.C = Out + nd.off * c; g.ldc = c;
      }
    }
  }
  out[i] = g;
}

}  // namespace

cudaError_t launch_build_apply_tasks(const ApplyNode* nodes, int L, int r, int64_t N, int trans,
                                     int c, const double* arena, const double* X, double* Out,
                                     double* ws, GemmTask* out, cudaStream_t st) {
  const int64_t total = (L == 0) ? 1 : (int64_t(4) << L) - 3;
  const int64_t blocks = (total + THREADS - 1) / THREADS;
  build_apply_tasks<<<static_cast<unsigned>(blocks), THREADS, 0, st>>>(nodes, L, r, N, trans, c,
                                                                       arena, X, Out, ws, out);
  return cudaGetLastError();
}

cudaError_t launch_gemm_tasks_f64(const GemmTask* d_tasks, int ntasks, int ncols, cudaStream_t st) {
  if (ntasks <= 0) return cudaSuccess;
  if (ncols >= 1 && ncols <= kSkinny) {          // every task has ncols columns
    // warp slots per task: 2 (rows 0-31 and 32-63 of a task, then 64-95 ... by the same two)
    const int spt = 2;
    const long long slots = static_cast<long long>(ntasks) * spt;
    const int grid = static_cast<int>(std::min<long long>((slots + 1) / 2, 152 * 32));
    switch (ncols) {
      case 1: gemm_tasks_skinny<1><<<grid, kSkinnyThreads, 0, st>>>(d_tasks, ntasks, spt); break;
      case 2: gemm_tasks_skinny<2><<<grid, kSkinnyThreads, 0, st>>>(d_tasks, ntasks, spt); break;
      case 3: gemm_tasks_skinny<3><<<grid, kSkinnyThreads, 0, st>>>(d_tasks, ntasks, spt); break;
      default: gemm_tasks_skinny<4><<<grid, kSkinnyThreads, 0, st>>>(d_tasks, ntasks, spt); break;
    }
    return cudaGetLastError();
  }
  gemm_tasks_f64<<<ntasks, THREADS, 0, st>>>(d_tasks, ncols);
  return cudaGetLastError();
}

}  // namespace hbs
