// Mixed-precision sampling Y = A Omega, Z = A^* Psi (Algorithm 2, first block) on the
// 5th-generation tensor cores (tcgen05, sm_103a) with split-BF16 compensated products.
//
// A is FP32 (row-major N x N). Each FP32 value a is split into P bfloat16 slices by repeated
// round-to-nearest (a = a_0 + a_1 + ... up to the last slice's rounding), each FP64 entry of
// Omega/Psi into Q slices the same way. C = sum over slice pairs (p, q) with p + q < max(P, Q)
// of A_p B_q^*: P = Q = 2 gives 3 products ("bf16x3", ~16 significant bits), P = Q = 3 gives 6
// ("bf16x6", ~24 bits).
//
// Accumulation. The tensor core adds each MMA result into its FP32 accumulator with a
// truncating rounding, so an accumulator that collects many MMAs drifts by ~0.5 ulp per MMA
// (measured: relative error growing linearly with the reduction length). Here an accumulator
// collects only the MMAs of DR reduction steps of 64 columns: the small slice products first,
// the leading pair (0, 0) last, so only the last few MMAs truncate at full magnitude. It is
// then drained into a double-float (hi + lo, TwoSum in FP32) running sum kept in tensor
// memory, while the tensor core fills the other accumulator of a ping-pong pair. The running
// sum goes out as FP64; reduction splits exist only to balance the grid and are summed in FP64.
//
// CTA (448 threads, one per SM): warp 0 issues the TMA loads of the Q pre-split B tiles
// (128-byte swizzled); warp 1 owns the tensor memory and one thread issues tcgen05.mma
// (M = 128, N = BN <= 128, K = 16 per instruction); warps 2-9 read the FP32 A tile straight
// from global memory (the next tile held in registers, the two after it prefetched into L2)
// and write its P bf16 slices in the 128-byte-swizzled K-major layout the MMA reads
// (transposing it on the way for Z = A^* Psi); warps 10-13 drain the accumulators
// (tcgen05.ld / tcgen05.st) and write the result. The operand stages (P A slices + Q B slices)
// form a ring of SO buffers (2 for bf16x6, 3 for bf16x3), so splitting the next tile overlaps
// the current MMAs. Tensor memory: two accumulators, hi, lo (4 x 128 columns). mbarriers hand
// buffers between the roles; every wait is bounded in time and sets the timeout bit of the
// status word instead of hanging. (Measured: 4 converter warps leave the MMAs waiting for
// slices; 8 drain warps next to 8 converters spill registers; this split is the fastest.)
#include <cuda.h>
#include <cuda_bf16.h>
#include <cudaTypedefs.h>

#include <mutex>
#include <vector>

#include "hbs_internal.cuh"
#include "tc_ptx.cuh"

namespace hbs {
namespace {

constexpr int kConvWarps = 8;                 // FP32 A -> bf16 slices
constexpr int kDrainWarps = 4;                // per quarter of tensor-memory lanes: kDrainWarps / 4
constexpr int kDrainParts = kDrainWarps / 4;  // column chunks c of a warp: c % kDrainParts == part
constexpr int kTcThreads = 64 + 32 * (kConvWarps + kDrainWarps);
constexpr int BM = 128;                       // MMA M: rows of C per CTA
constexpr int BK = 64;                        // reduction columns per stage (128 B of bf16)
constexpr int kSliceABytes = BM * BK * 2;     // one bf16 slice of the A tile
constexpr int kUnitsPerThread = BM * BK / 8 / (32 * kConvWarps);   // (row, 8-column) units
static_assert(kUnitsPerThread == 4, "the Z mapping gives a thread 4 neighbouring rows of op(A)");
// Unit `it` of converter thread ct is (row m, 8-column chunk c) of op(A); the thread holds its 8
// FP32 values. Y = A Omega: u = ct + 256 it, m = u / 8, c = u % 8 (8 lanes cover one 256-byte row
// of A). Z = A^* Psi: the thread's 4 units are 4 neighbouring columns of A (m = 4 mb + it), read
// as one 16-byte vector per row of A; lane l of warp w takes c = l % 4 + 4 (w % 2) and
// mb = l / 4 + 8 (w / 2), so that a warp reads whole 128-byte lines (4 rows of A, 32 columns)
// and the 8 lanes of a shared-memory store phase write two rows of the tile whose m % 8 differ
// in bit 2 (8 distinct swizzled chunks: no bank conflict).
template <bool TRANS>
__device__ __forceinline__ void unit_coords(int ct, int it, int& m, int& c) {
  if (!TRANS) {
    const int u = ct + 32 * kConvWarps * it;
    m = u >> 3;
    c = u & 7;
  } else {
    const int w = ct >> 5, l = ct & 31;
    m = 4 * ((l >> 2) + 8 * (w >> 1)) + it;
    c = (l & 3) + 4 * (w & 1);
  }
}

// Loads the thread's units of the A tile (rows m0.., reduction columns k0..). Y reads
// A[m0 + m][k0 + 8c ..] as two float4; Z reads, for each e < 8, A[k0 + 8c + e][m0 + 4 mb ..]
// as one float4. A is 16-byte aligned and lda % 4 == 0. Entries outside M x K read as zero.
template <bool TRANS>
__device__ __forceinline__ void load_units(const float* __restrict__ A, int64_t lda, int M, int K,
                                           int m0, int k0, int ct,
                                           float (&v)[kUnitsPerThread][8]) {
  if (!TRANS) {
#pragma unroll
    for (int it = 0; it < kUnitsPerThread; ++it) {
      int m, c;
      unit_coords<false>(ct, it, m, c);
      const int64_t gm = m0 + m, gk = k0 + 8 * c;
      if (gm < M && gk + 8 <= K) {
        const float4* q = reinterpret_cast<const float4*>(A + gm * lda + gk);
        const float4 lo = q[0], hi = q[1];
        v[it][0] = lo.x; v[it][1] = lo.y; v[it][2] = lo.z; v[it][3] = lo.w;
        v[it][4] = hi.x; v[it][5] = hi.y; v[it][6] = hi.z; v[it][7] = hi.w;
      } else {
#pragma unroll
        for (int e = 0; e < 8; ++e) v[it][e] = (gm < M && gk + e < K) ? A[gm * lda + gk + e] : 0.f;
      }
    }
  } else {
    int m, c;
    unit_coords<true>(ct, 0, m, c);
    const int64_t gm = m0 + m;
#pragma unroll
    for (int e = 0; e < 8; ++e) {
      const int64_t gk = k0 + 8 * c + e;
      if (gk < K && gm + 4 <= M) {
        const float4 q = *reinterpret_cast<const float4*>(A + gk * lda + gm);
        v[0][e] = q.x; v[1][e] = q.y; v[2][e] = q.z; v[3][e] = q.w;
      } else {
#pragma unroll
        for (int i = 0; i < 4; ++i) v[i][e] = (gk < K && gm + i < M) ? A[gk * lda + gm + i] : 0.f;
      }
    }
  }
}

// Brings the A tile at (m0, k0) towards L2 ahead of its loads: its 256 lines of 128 bytes
// (128 rows of 256 B for Y; 64 rows of A of 512 B for Z) spread over the converter threads.
template <bool TRANS>
__device__ __forceinline__ void prefetch_tile(const float* A, int64_t lda, int M, int K, int m0,
                                              int k0, int ct) {
#pragma unroll
  for (int l = ct; l < 256; l += 32 * kConvWarps) {
    int64_t row, col;
    if (!TRANS) {
      row = m0 + (l >> 1);
      col = k0 + 32 * (l & 1);
      if (row >= M || col >= K) continue;
    } else {
      row = k0 + (l >> 2);
      col = m0 + 32 * (l & 3);
      if (row >= K || col >= M) continue;
    }
    asm volatile("prefetch.global.L2 [%0];" ::"l"(A + row * lda + col));
  }
}

// Splits the units into P bf16 slices in the K-major 128-byte swizzled layout: row m at byte
// m*128, 16-byte chunk c (columns 8c..8c+7) at chunk c ^ (m%8).
template <int P, bool TRANS>
__device__ __forceinline__ void store_units(const float (&v)[kUnitsPerThread][8], uint8_t* slices,
                                            int ct) {
#pragma unroll
  for (int it = 0; it < kUnitsPerThread; ++it) {
    int m, c;
    unit_coords<TRANS>(ct, it, m, c);
    uint32_t w[P][4];
#pragma unroll
    for (int e = 0; e < 4; ++e) {
      float x0 = v[it][2 * e], x1 = v[it][2 * e + 1];
#pragma unroll
      for (int p = 0; p < P; ++p) {
        const __nv_bfloat162 h = __floats2bfloat162_rn(x0, x1);
        w[p][e] = *reinterpret_cast<const uint32_t*>(&h);
        const float2 f = __bfloat1622float2(h);
        x0 -= f.x;
        x1 -= f.y;
      }
    }
    const uint32_t off = static_cast<uint32_t>(m) * 128u +
                         ((static_cast<uint32_t>(c) ^ (static_cast<uint32_t>(m) & 7u)) << 4);
#pragma unroll
    for (int p = 0; p < P; ++p)
      *reinterpret_cast<uint4*>(slices + p * kSliceABytes + off) =
          make_uint4(w[p][0], w[p][1], w[p][2], w[p][3]);
  }
}

struct TcArgs {
  const float* A;  // FP32 A, row-major, lda % 4 == 0
  int64_t lda;
  int M, K;        // rows of C, reduction length
  int BN;          // columns per CTA (multiple of 32, <= 128); blockIdx.z picks the column tile
  int BNt;         // padded columns of the whole product (BN x column tiles)
  int kchunk;      // reduction columns per split (multiple of BK)
  double* partial; // [splits][M][BNt] FP64
  int* status;
};

template <int P, int Q, bool TRANS, int SO, int DR>
__global__ void __launch_bounds__(kTcThreads, 1)
    sliced_gemm_tc(const __grid_constant__ CUtensorMap tmB, TcArgs a) {
  extern __shared__ uint8_t smem_raw[];
  if (aborted(a.status)) return;              // a CTA of this run timed out: nothing issued yet
  uint8_t* smem = smem_raw + ((1024u - (su32(smem_raw) & 1023u)) & 1023u);
  const int BN = a.BN;
  const int slice_b_bytes = BN * 128;
  uint8_t* opA = smem;                                           // SO x P bf16 A slices
  uint8_t* opB = opA + SO * P * kSliceABytes;                    // SO x Q bf16 B slices
  uint64_t* b_full = reinterpret_cast<uint64_t*>(opB + SO * Q * slice_b_bytes);
  uint64_t* o_empty = b_full + SO;                               // the stage's MMAs are done
  uint64_t* a_ready = o_empty + SO;                              // the stage's A slices written
  uint64_t* acc_full = a_ready + SO;                             // 2: accumulator ping-pong
  uint64_t* acc_empty = acc_full + 2;                            // 2
  uint64_t* mma_done = acc_empty + 2;                            // every issued MMA finished
  uint32_t* tmem_slot = reinterpret_cast<uint32_t*>(mma_done + 1);

  const int warp = threadIdx.x / 32, lane = threadIdx.x % 32;
  const int m0 = blockIdx.x * BM;
  const int n0 = blockIdx.z * BN;                                // first column of this tile
  const int k_begin = blockIdx.y * a.kchunk;
  const int k_end = min(a.K, k_begin + a.kchunk);
  const int nk = (k_end - k_begin + BK - 1) / BK;
  const int ngroups = (nk + DR - 1) / DR;                        // accumulator drains
  constexpr uint32_t kTmemCols = 512;                            // acc0, acc1, hi, lo
  constexpr uint32_t kHi = 256, kLo = 384;

  if (threadIdx.x == 0) {
    for (int i = 0; i < SO; ++i) {
      mbar_init(&b_full[i], 1);
      mbar_init(&o_empty[i], 1);
      mbar_init(&a_ready[i], kConvWarps);
    }
    for (int i = 0; i < 2; ++i) {
      mbar_init(&acc_full[i], 1);
      mbar_init(&acc_empty[i], kDrainWarps);
    }
    mbar_init(mma_done, 1);
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  if (warp == 1) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(
                     su32(tmem_slot)),
                 "r"(kTmemCols)
                 : "memory");
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
  }
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  const uint32_t tmem = *tmem_slot;

  if (warp == 0) {
    if (lane == 0) {                                            // ---- TMA producer (B) ----
      bool ok = true;
      int issued = 0;
      for (int ks = 0; ks < nk && ok; ++ks) {
        const int so = ks % SO, uo = ks / SO;
        const int k0 = k_begin + ks * BK;
        if (ks >= SO) ok = mbar_wait(&o_empty[so], (uo - 1) & 1, a.status);
        if (!ok) break;
        mbar_expect_tx(&b_full[so], Q * slice_b_bytes);
#pragma unroll
        for (int q = 0; q < Q; ++q)
          tma_load_2d(opB + (so * Q + q) * slice_b_bytes, &tmB, &b_full[so], k0, q * a.BNt + n0);
        issued = ks + 1;
      }
      // the last copies into each buffer must have landed before the CTA may exit
      for (int ks = max(0, issued - SO); ks < issued; ++ks)
        mbar_wait(&b_full[ks % SO], (ks / SO) & 1, a.status, false);
    }
  } else if (warp == 1) {
    if (lane == 0) {                                            // ---- MMA issuer ----
      const uint32_t idesc = idesc_bf16(BM, BN);
      bool ok = true;
      for (int g = 0; g < ngroups && ok; ++g) {
        const int b = g & 1;
        if (g >= 2) ok = mbar_wait(&acc_empty[b], ((g >> 1) - 1) & 1, a.status);
        if (!ok) break;
        tc_fence_after();
        const uint32_t acc = tmem + static_cast<uint32_t>(b * 128);
        const int ks_end = min(nk, (g + 1) * DR);
        for (int ks = g * DR; ks < ks_end && ok; ++ks) {
          const int so = ks % SO, uo = ks / SO;
          ok = mbar_wait(&b_full[so], uo & 1, a.status) && mbar_wait(&a_ready[so], uo & 1, a.status);
          if (!ok) break;
          tc_fence_after();
          const uint32_t abase = su32(opA + so * P * kSliceABytes);
          const uint32_t bbase = su32(opB + so * Q * slice_b_bytes);
          const bool fresh = (ks == g * DR);
          int term = 0;
          // small slice products first, the leading pair (0, 0) last
#pragma unroll
          for (int level = (P > Q ? P : Q) - 1; level >= 0; --level) {
#pragma unroll
            for (int p = 0; p < P; ++p) {
              const int q = level - p;
              if (q < 0 || q >= Q) continue;
              const uint64_t ad = sw128_desc(abase + p * kSliceABytes);
              const uint64_t bd = sw128_desc(bbase + q * slice_b_bytes);
#pragma unroll
              for (int kk = 0; kk < BK / 16; ++kk)
                mma_bf16(acc, ad + 2 * kk, bd + 2 * kk, idesc, (fresh && term == 0 && kk == 0) ? 0u : 1u);
              ++term;
            }
          }
          mma_commit(&o_empty[so]);
        }
        if (!ok) break;
        mma_commit(&acc_full[b]);
      }
      // every MMA this thread issued must have finished before tensor memory is freed
      mma_commit(mma_done);
      mbar_wait(mma_done, 0, a.status, false);
    }
  } else if (warp < 2 + kConvWarps) {                           // ---- A converters ----
    const int ct = threadIdx.x - 64;
    float cur[kUnitsPerThread][8], nxt[kUnitsPerThread][8];
    for (int d = 1; d <= 2 && d < nk; ++d)                      // first tiles towards L2
      prefetch_tile<TRANS>(a.A, a.lda, a.M, a.K, m0, k_begin + d * BK, ct);
    if (nk > 0) load_units<TRANS>(a.A, a.lda, a.M, a.K, m0, k_begin, ct, cur);
    bool ok = true;
    for (int ks = 0; ks < nk && ok; ++ks) {
      const int so = ks % SO, uo = ks / SO;
      if (ks + 3 < nk)                                          // three tiles ahead into L2
        prefetch_tile<TRANS>(a.A, a.lda, a.M, a.K, m0, k_begin + (ks + 3) * BK, ct);
      if (ks + 1 < nk)                                          // the next tile in registers
        load_units<TRANS>(a.A, a.lda, a.M, a.K, m0, k_begin + (ks + 1) * BK, ct, nxt);
      if (ks >= SO) ok = mbar_wait(&o_empty[so], (uo - 1) & 1, a.status);
      if (!ok) break;
      store_units<P, TRANS>(cur, opA + so * P * kSliceABytes, ct);
      asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
      __syncwarp();
      if (lane == 0) mbar_arrive(&a_ready[so]);
#pragma unroll
      for (int it = 0; it < kUnitsPerThread; ++it)
#pragma unroll
        for (int e = 0; e < 8; ++e) cur[it][e] = nxt[it][e];
    }
  } else {                                                      // ---- accumulator drain ----
    const int quarter = warp & 3;                               // TMEM lanes 32*quarter..+31
    const int part = (warp - 2 - kConvWarps) >> 2;              // 32-column chunks of this warp
    const uint32_t lane_base = static_cast<uint32_t>(quarter * 32) << 16;
    bool ok = true;
    int drained = 0;
    for (int g = 0; g < ngroups && ok; ++g) {
      const int b = g & 1;
      ok = mbar_wait(&acc_full[b], (g >> 1) & 1, a.status);
      if (!ok) break;
      tc_fence_after();
      for (int c0 = 32 * part; c0 < BN; c0 += 32 * kDrainParts) {
        uint32_t x[32], hi[32], lo[32];
        tmem_ld32(tmem + lane_base + static_cast<uint32_t>(b * 128 + c0), x);
        if (g == 0) {
#pragma unroll
          for (int j = 0; j < 32; ++j) {
            hi[j] = x[j];
            lo[j] = 0u;
          }
        } else {
          tmem_ld32(tmem + lane_base + kHi + static_cast<uint32_t>(c0), hi);
          tmem_ld32(tmem + lane_base + kLo + static_cast<uint32_t>(c0), lo);
#pragma unroll
          for (int j = 0; j < 32; ++j) {                        // (hi, lo) += x, TwoSum
            const float h = __uint_as_float(hi[j]), v = __uint_as_float(x[j]);
            const float s = h + v;
            const float bp = s - h;
            const float err = (h - (s - bp)) + (v - bp);
            hi[j] = __float_as_uint(s);
            lo[j] = __float_as_uint(__uint_as_float(lo[j]) + err);
          }
        }
        tmem_st32(tmem + lane_base + kHi + static_cast<uint32_t>(c0), hi);
        tmem_st32(tmem + lane_base + kLo + static_cast<uint32_t>(c0), lo);
      }
      tc_fence_before();
      __syncwarp();
      if (lane == 0) mbar_arrive(&acc_empty[b]);
      drained = g + 1;
    }
    tc_fence_after();
    const int row = m0 + quarter * 32 + lane;
    double* out = a.partial + (static_cast<size_t>(blockIdx.y) * a.M + row) * a.BNt + n0;
    if (ok && drained == ngroups && ngroups > 0) {
      for (int c0 = 32 * part; c0 < BN; c0 += 32 * kDrainParts) {
        uint32_t hi[32], lo[32];
        tmem_ld32(tmem + lane_base + kHi + static_cast<uint32_t>(c0), hi);
        tmem_ld32(tmem + lane_base + kLo + static_cast<uint32_t>(c0), lo);
        if (row < a.M) {
#pragma unroll
          for (int j = 0; j < 32; j += 2)
            *reinterpret_cast<double2*>(out + c0 + j) = make_double2(
                static_cast<double>(__uint_as_float(hi[j])) + static_cast<double>(__uint_as_float(lo[j])),
                static_cast<double>(__uint_as_float(hi[j + 1])) + static_cast<double>(__uint_as_float(lo[j + 1])));
        }
      }
    } else if (ngroups == 0 && row < a.M && part == 0) {
      for (int c = 0; c < BN; ++c) out[c] = 0.0;
    }
  }
  tc_fence_before();
  __syncthreads();
  if (warp == 1) {
    tc_fence_after();
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(kTmemCols)
                 : "memory");
  }
}

// Omega (N x s FP64, row-major) -> Q bf16 slices of Omega^*: out[q*BN + c][j], rows c >= s and
// columns j >= N zero. 32 x 32 tiles through shared memory so both sides stay coalesced.
template <int Q>
__global__ void split_rhs(const double* __restrict__ X, int64_t N, int s, int BN, int64_t ldb,
                          __nv_bfloat16* __restrict__ out) {
  __shared__ double tile[32][33];
  const int64_t j0 = static_cast<int64_t>(blockIdx.x) * 32;
  const int c0 = blockIdx.y * 32;
  for (int e = threadIdx.y; e < 32; e += blockDim.y) {
    const int64_t j = j0 + e;
    const int c = c0 + threadIdx.x;
    tile[e][threadIdx.x] = (j < N && c < s) ? X[j * s + c] : 0.0;
  }
  __syncthreads();
  for (int e = threadIdx.y; e < 32; e += blockDim.y) {
    const int c = c0 + e;
    const int64_t j = j0 + threadIdx.x;
    if (c >= BN || j >= ldb) continue;
    double x = tile[threadIdx.x][e];
#pragma unroll
    for (int q = 0; q < Q; ++q) {
      const __nv_bfloat16 h = __double2bfloat16(x);
      out[(static_cast<int64_t>(q) * BN + c) * ldb + j] = h;
      x -= static_cast<double>(__bfloat162float(h));
    }
  }
}

__global__ void reduce_partials(const double* __restrict__ partial, int splits, int64_t M, int BN,
                                int s, double* __restrict__ C) {
  const int64_t total = M * s;
  for (int64_t idx = blockIdx.x * static_cast<int64_t>(blockDim.x) + threadIdx.x; idx < total;
       idx += static_cast<int64_t>(gridDim.x) * blockDim.x) {
    const int64_t i = idx / s;
    const int c = static_cast<int>(idx % s);
    double acc = 0.0;
    for (int sp = 0; sp < splits; ++sp) acc += partial[(sp * M + i) * BN + c];
    C[idx] = acc;
  }
}

// ---- host side ------------------------------------------------------------------------------

// Per-device scratch of the tensor-core sampling (B slices and split partials), grown on demand.
struct TcScratch {
  void* ptr = nullptr;
  size_t bytes = 0;
};
std::mutex g_tc_mutex;
std::vector<TcScratch> g_tc_scratch;

cudaError_t tc_scratch(size_t bytes, void** out) {
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return e;
  std::lock_guard<std::mutex> lock(g_tc_mutex);
  if (static_cast<int>(g_tc_scratch.size()) <= dev) g_tc_scratch.resize(dev + 1);
  TcScratch& s = g_tc_scratch[dev];
  if (s.bytes < bytes) {
    if (s.ptr) {
      e = cudaDeviceSynchronize();
      if (e != cudaSuccess) return e;
      cudaFree(s.ptr);
      s.ptr = nullptr;
      s.bytes = 0;
    }
    e = cudaMalloc(&s.ptr, bytes);
    if (e != cudaSuccess) return e;
    s.bytes = bytes;
    e = cudaMemset(s.ptr, 0, 1024);          // status word starts clear
    if (e != cudaSuccess) return e;
  }
  *out = s.ptr;
  return cudaSuccess;
}

size_t smem_bytes(int P, int Q, int SO, int BN) {
  return static_cast<size_t>(SO) * (P * kSliceABytes + Q * BN * 128) + 256 + 1024;
}

template <int P, int Q, bool TRANS, int SO>
cudaError_t launch_one(const CUtensorMap& mb, const TcArgs& args, int splits, cudaStream_t st) {
  constexpr int DR = (P >= 3) ? 1 : 2;        // reduction steps per accumulator drain
  auto kernel = sliced_gemm_tc<P, Q, TRANS, SO, DR>;
  const size_t bytes = smem_bytes(P, Q, SO, args.BN);
  cudaError_t e = cudaFuncSetAttribute(kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                       static_cast<int>(bytes));
  if (e != cudaSuccess) return e;
  const dim3 grid(static_cast<unsigned>((args.M + BM - 1) / BM), static_cast<unsigned>(splits),
                  static_cast<unsigned>(args.BNt / args.BN));
  kernel<<<grid, kTcThreads, bytes, st>>>(mb, args);
  return cudaGetLastError();
}

template <int P, bool TRANS>
cudaError_t launch_pq(const CUtensorMap& mb, const TcArgs& args, int splits, cudaStream_t st) {
  // the deepest operand ring that fits 227 KB
  if (smem_bytes(P, P, 3, args.BN) <= kMaxNodeSmemBytes)
    return launch_one<P, P, TRANS, 3>(mb, args, splits, st);
  if (smem_bytes(P, P, 2, args.BN) <= kMaxNodeSmemBytes)
    return launch_one<P, P, TRANS, 2>(mb, args, splits, st);
  return launch_one<P, P, TRANS, 1>(mb, args, splits, st);
}

}  // namespace

// Column tiling: s <= 128 runs as one tile of BN = s rounded up to 32; wider s as tiles of 128.
void column_tiles(int s, int* BN, int* BNt) {
  *BNt = (s <= 128) ? (s + 31) / 32 * 32 : (s + 127) / 128 * 128;
  *BN = (*BNt < 128) ? *BNt : 128;
}

// Reduction splits: only to fill the GPU (about 8 CTAs per SM in total), each split >= 64 wide.
int reduction_splits(int64_t N, int BNt, int BN) {
  const int64_t tiles = ((N + BM - 1) / BM) * (BNt / BN);
  int64_t splits = (8 * 152 + tiles - 1) / tiles;
  const int64_t ksteps = (N + BK - 1) / BK;
  if (splits > ksteps) splits = ksteps;
  return static_cast<int>(splits < 1 ? 1 : splits);
}

// Scratch layout: [0, 1024) status word; then Q x BNt x ldb bf16 slices of Omega^* and of
// Psi^*; then the FP64 split partials.
size_t sample_tc_scratch_bytes(int64_t N, int s, int kchunk) {
  int BN, BNt;
  column_tiles(s, &BN, &BNt);
  const int64_t ldb = (N + 7) / 8 * 8;
  const int64_t splits = (N + kchunk - 1) / kchunk;
  return 1024 + static_cast<size_t>(2 * 3 * BNt * ldb * 2) +
         static_cast<size_t>(splits * N * BNt * 8);
}

cudaError_t sample_tc_status(int* host_status, bool clear) {
  *host_status = 0;
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return e;
  int* status = nullptr;
  {
    std::lock_guard<std::mutex> lock(g_tc_mutex);
    if (dev < static_cast<int>(g_tc_scratch.size())) status = static_cast<int*>(g_tc_scratch[dev].ptr);
  }
  if (!status) return cudaSuccess;
  e = cudaMemcpy(host_status, status, sizeof(int), cudaMemcpyDeviceToHost);
  if (e == cudaSuccess && clear) e = cudaMemset(status, 0, kStatusWords * sizeof(int));
  return e;
}

cudaError_t sample_tc_inject(int bits) {
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return e;
  int* status = nullptr;
  {
    std::lock_guard<std::mutex> lock(g_tc_mutex);
    if (dev < static_cast<int>(g_tc_scratch.size())) status = static_cast<int*>(g_tc_scratch[dev].ptr);
  }
  if (!status) return cudaSuccess;
  const int words[kStatusWords] = {bits, (bits & kStatusTimeout) ? 1 : 0};
  int now[kStatusWords];
  e = cudaMemcpy(now, status, sizeof(now), cudaMemcpyDeviceToHost);
  now[0] |= words[0];
  now[kAbortWord] |= words[kAbortWord];
  if (e == cudaSuccess) e = cudaMemcpy(status, now, sizeof(now), cudaMemcpyHostToDevice);
  return e;
}

cudaError_t launch_sample_dense_tc(const float* A, int64_t lda, int64_t N, const double* Om,
                                   const double* Ps, int s, double* Y, double* Z, int slices,
                                   int kchunk_hint, cudaStream_t st) {
  if (slices != 2 && slices != 3) return cudaErrorInvalidValue;
  if (s < 1 || s > 256 || N < 1 || N > (int64_t(1) << 30) || lda % 4 != 0)
    return cudaErrorInvalidValue;
  int BN, BNt;
  column_tiles(s, &BN, &BNt);
  const int64_t ldb = (N + 7) / 8 * 8;
  int kchunk;
  if (kchunk_hint > 0) {
    kchunk = (kchunk_hint + BK - 1) / BK * BK;
  } else {
    const int splits_wanted = reduction_splits(N, BNt, BN);
    kchunk = static_cast<int>(((N + splits_wanted - 1) / splits_wanted + BK - 1) / BK * BK);
  }
  const int splits = static_cast<int>((N + kchunk - 1) / kchunk);
  void* scratch = nullptr;
  cudaError_t e = tc_scratch(sample_tc_scratch_bytes(N, s, kchunk), &scratch);
  if (e != cudaSuccess) return e;
  int* status = static_cast<int*>(scratch);
  auto* bY = reinterpret_cast<__nv_bfloat16*>(static_cast<uint8_t*>(scratch) + 1024);
  auto* bZ = bY + 3 * BNt * ldb;
  double* partial = reinterpret_cast<double*>(bZ + 3 * BNt * ldb);
  // a new run: clear the abort flag an earlier run may have left (the report bits stay)
  e = cudaMemsetAsync(status + kAbortWord, 0, sizeof(int), st);
  if (e != cudaSuccess) return e;

  const dim3 tb(32, 8), tg(static_cast<unsigned>((ldb + 31) / 32), static_cast<unsigned>((BNt + 31) / 32));
  if (slices == 2) {
    split_rhs<2><<<tg, tb, 0, st>>>(Om, N, s, BNt, ldb, bY);
    split_rhs<2><<<tg, tb, 0, st>>>(Ps, N, s, BNt, ldb, bZ);
  } else {
    split_rhs<3><<<tg, tb, 0, st>>>(Om, N, s, BNt, ldb, bY);
    split_rhs<3><<<tg, tb, 0, st>>>(Ps, N, s, BNt, ldb, bZ);
  }
  e = cudaGetLastError();
  if (e != cudaSuccess) return e;

  CUtensorMap mBy, mBz;
  const uint64_t brow = static_cast<uint64_t>(ldb) * 2;
  const uint64_t brows = static_cast<uint64_t>(slices) * BNt;
  if (!make_map(&mBy, CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, bY, N, brows, brow, BK, BN, CU_TENSOR_MAP_SWIZZLE_128B) ||
      !make_map(&mBz, CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, bZ, N, brows, brow, BK, BN, CU_TENSOR_MAP_SWIZZLE_128B))
    return cudaErrorInvalidValue;

  TcArgs args{A, lda, static_cast<int>(N), static_cast<int>(N), BN, BNt, kchunk, partial, status};
  const unsigned rg = 152u * 8u;
  e = (slices == 2) ? launch_pq<2, false>(mBy, args, splits, st)
                    : launch_pq<3, false>(mBy, args, splits, st);
  if (e != cudaSuccess) return e;
  reduce_partials<<<rg, 256, 0, st>>>(partial, splits, N, BNt, s, Y);
  e = cudaGetLastError();
  if (e != cudaSuccess) return e;
  e = (slices == 2) ? launch_pq<2, true>(mBz, args, splits, st)
                    : launch_pq<3, true>(mBz, args, splits, st);
  if (e != cudaSuccess) return e;
  reduce_partials<<<rg, 256, 0, st>>>(partial, splits, N, BNt, s, Z);
  return cudaGetLastError();
}

}  // namespace hbs
