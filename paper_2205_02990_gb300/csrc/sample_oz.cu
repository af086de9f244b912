// FP64-class sampling Y = A Omega, Z = A^* Psi (Algorithm 2, first block) on the tcgen05 tensor
// cores by exact products of 8-bit digits: an error-free splitting in the manner of Ozaki,
// Ogita, Oishi and Rump (Numer. Algorithms 59, 2012), with bfloat16 digits and FP32
// accumulation instead of FP64 slices.
//
// Digits. A block of FP64 entries that shares one exponent E (every |x| < 2^(E-1), the largest
// >= 2^(E-2)) is scaled to the integers X = round(x 2^(8S-E)), |X| <= 2^(8S-1), and each X is
// written in balanced base 256: X = sum_{i<S} d_i 256^(S-1-i), d_i in [-128, 128]. Then
// x = sum_i d_i 2^(E-8(i+1)) to within 2^(E-8S-1), and every digit is exact in bfloat16.
// A has one exponent per row and 64-column window (the blocks of Y = A Omega) and one per column
// and 64-row window (the blocks of Z = A^* Psi, whose reduction runs over the rows of A); the
// test matrices have one per 64-row window. Digit planes are written once per call by a split
// pass: A's in both orientations, each plane row-major so that the reduction index is the
// contiguous one (the K-major operand layout of the MMA).
//
// Exact products. Digit products are integers of magnitude <= 2^14. For one output entry, the
// products of the digit pairs (i, j) with i + j = d over one 64-wide window all carry the scale
// 2^(E_a + E_b - 8d - 16) and sum to an integer of magnitude <= (d + 1) * 64 * 2^14 < 2^23
// (d < S <= 7), so the tensor core's FP32 accumulator holds every partial sum exactly, in any
// order and under any rounding of its adder. Pairs with i + j <= S - 1 are formed, S(S+1)/2
// bf16 tile products per window; each dropped pair weighs at most 2^(2-8S) of max|a| max|b|.
//
// Accumulation. The diagonal d of a window is one accumulator in tensor memory (two of them,
// ping-pong): the MMA thread fills one while eight drain warps scale the other by its power of
// two (exact) and add it to a double-float running sum kept in tensor memory (hi + lo: TwoSum in
// FP32, then a Fast2Sum renormalisation that keeps |lo| <= ulp(hi) / 2, so that every addition
// errs by at most ~2^-48 of the running sum). A CTA's reduction range is at most 32 windows (2048 indices); the ranges are summed
// in FP64 by the reduce kernel. Within a range, scales are taken relative to the largest block
// exponents of the output row's entries of A and of the test matrix over that range; the
// reduce kernel scales each range's sum back in FP64. Every output row keeps the full FP64
// exponent range; only blocks more than ~2^100 below the largest block of their row and range
// are flushed (they are below its rounding).
//
// CTA (320 threads, one per SM): warp 0 issues the TMA loads of a window's S A-digit tiles
// (128 x 64) and S test-digit tiles (BN x 64), one mbarrier per digit so that the products of
// low diagonals start before the high digits land; warp 1 allocates tensor memory and one
// thread issues tcgen05.mma (M = 128, N = BN, K = 16); warps 2-9 drain. Every wait is bounded
// and sets the timeout bit of the status word instead of hanging.
#include <cuda.h>
#include <cudaTypedefs.h>

#include <algorithm>
#include <mutex>
#include <vector>

#include "hbs_internal.cuh"
#include "tc_ptx.cuh"

namespace hbs {
namespace {

constexpr int kOzThreads = 320;
constexpr int OBM = 128;                       // rows of C per CTA (MMA M)
constexpr int OBK = 64;                        // window: reduction indices per digit tile
constexpr int kDigitTileA = OBM * OBK * 2;     // one bf16 digit tile of A
constexpr int kMaxWindowsPerSplit = 32;        // double-float sums span at most 2048 indices
constexpr int16_t kNoExp = -32768;             // exponent of an all-zero block (the smallest)

// ---- digit splitting -------------------------------------------------------------------------

__device__ __forceinline__ uint64_t abs_bits(double x) {
  return static_cast<uint64_t>(__double_as_longlong(x)) & 0x7fffffffffffffffull;
}

// E with 2^(E-2) <= m < 2^(E-1) for the magnitude bits m of a finite nonzero double; kNoExp for
// zero. Infinities and NaNs set the numeric bit.
__device__ __forceinline__ int block_exponent(uint64_t m, int* status) {
  if (m == 0) return kNoExp;
  const int e = static_cast<int>(m >> 52);
  if (e == 0x7ff) {
    atomicOr(status, kStatusNumeric);
    return 1026;
  }
  if (e == 0) return (63 - __clzll(static_cast<long long>(m))) - 1073 + 1;
  return e - 1021;
}

// Balanced base-256 digits of round(x 2^(8S - E)) (|x| < 2^(E-1)), most significant first.
template <int S>
__device__ __forceinline__ void to_digits(double x, int E, int (&d)[S]) {
  const uint64_t u = static_cast<uint64_t>(__double_as_longlong(x));
  const int ex = static_cast<int>((u >> 52) & 0x7ff);
  uint64_t m = u & ((1ull << 52) - 1);
  int p = -1074;                                        // |x| = m 2^p
  if (ex != 0) {
    m |= 1ull << 52;
    p = ex - 1075;
  }
  const int sh = p + 8 * S - E;
  int64_t X = 0;
  if (E != kNoExp && m != 0 && ex != 0x7ff) {
    if (sh >= 0) X = static_cast<int64_t>(m << min(sh, 10));
    else if (sh > -60) X = static_cast<int64_t>((m + (1ull << (-sh - 1))) >> (-sh));
  }
  if (u >> 63) X = -X;
#pragma unroll
  for (int i = S - 1; i > 0; --i) {
    const int di = static_cast<int>((X + 128) & 255) - 128;
    d[i] = di;
    X = (X - di) >> 8;
  }
  d[0] = static_cast<int>(X);
}

// bfloat16 bits of an integer |v| <= 128 (exact: at most 8 significant bits).
__device__ __forceinline__ uint32_t digit_bf16(int v) {
  const float f = __int_as_float(0x4B000000 + v + 256) - 8388864.0f;   // 2^23 + 256
  return __float_as_uint(f) >> 16;
}

__device__ __forceinline__ uint64_t umax64(uint64_t a, uint64_t b) { return a > b ? a : b; }

// Writes 16 consecutive digits-of-x (one per plane) for a thread's 16 elements.
template <int S>
__device__ __forceinline__ void store_digits16(const double (&x)[16], int E, uint16_t* dst,
                                               size_t plane_stride) {
  uint32_t w[S][8];
#pragma unroll
  for (int j = 0; j < 16; j += 2) {
    int d0[S], d1[S];
    to_digits<S>(x[j], E, d0);
    to_digits<S>(x[j + 1], E, d1);
#pragma unroll
    for (int i = 0; i < S; ++i) w[i][j / 2] = digit_bf16(d0[i]) | (digit_bf16(d1[i]) << 16);
  }
#pragma unroll
  for (int i = 0; i < S; ++i) {
    uint4* q = reinterpret_cast<uint4*>(dst + i * plane_stride);
    q[0] = make_uint4(w[i][0], w[i][1], w[i][2], w[i][3]);
    q[1] = make_uint4(w[i][4], w[i][5], w[i][6], w[i][7]);
  }
}

// One 64 x 64 block of A: exponents per row (EY) and per column (EZ), digit planes of A (Yd,
// row-major) and of A^* (Zd). Planes: S x N rows of ldd entries; ldd a multiple of 64.
template <int S>
__global__ void __launch_bounds__(256)
    oz_split_a(const double* __restrict__ A, int64_t lda, int64_t N, uint16_t* __restrict__ Yd,
               uint16_t* __restrict__ Zd, int64_t ldd, int16_t* __restrict__ EY,
               int16_t* __restrict__ EZ, int W, int* status) {
  __shared__ double tile[64][65];
  __shared__ int rowE[64], colE[64];
  const int64_t r0 = static_cast<int64_t>(blockIdx.y) * 64, c0 = static_cast<int64_t>(blockIdx.x) * 64;
  const int t = threadIdx.x;
  for (int e = t; e < 64 * 64; e += 256) {
    const int r = e >> 6, c = e & 63;
    const int64_t gr = r0 + r, gc = c0 + c;
    tile[r][c] = (gr < N && gc < N) ? A[gr * lda + gc] : 0.0;
  }
  __syncthreads();
  const int g = t >> 2, part = t & 3;                 // row / column g, quarter `part`
  uint64_t mr = 0, mc = 0;
#pragma unroll
  for (int j = 0; j < 16; ++j) {
    mr = umax64(mr, abs_bits(tile[g][part * 16 + j]));
    mc = umax64(mc, abs_bits(tile[part * 16 + j][g]));
  }
  mr = umax64(mr, __shfl_xor_sync(0xffffffffu, mr, 1));
  mr = umax64(mr, __shfl_xor_sync(0xffffffffu, mr, 2));
  mc = umax64(mc, __shfl_xor_sync(0xffffffffu, mc, 1));
  mc = umax64(mc, __shfl_xor_sync(0xffffffffu, mc, 2));
  if (part == 0) {
    rowE[g] = block_exponent(mr, status);
    colE[g] = block_exponent(mc, status);
  }
  __syncthreads();
  if (t < 64) {
    if (r0 + t < N) EY[(r0 + t) * W + blockIdx.x] = static_cast<int16_t>(rowE[t]);
  } else if (t < 128) {
    if (c0 + t - 64 < N) EZ[(c0 + t - 64) * W + blockIdx.y] = static_cast<int16_t>(colE[t - 64]);
  }
  const size_t plane = static_cast<size_t>(N) * ldd;
  double x[16];
  if (r0 + g < N) {                                   // row g of A: digits for Y = A Omega
#pragma unroll
    for (int j = 0; j < 16; ++j) x[j] = tile[g][part * 16 + j];
    store_digits16<S>(x, rowE[g], Yd + (r0 + g) * ldd + c0 + part * 16, plane);
  }
  if (c0 + g < N) {                                   // column g of A: digits for Z = A^* Psi
#pragma unroll
    for (int j = 0; j < 16; ++j) x[j] = tile[part * 16 + j][g];
    store_digits16<S>(x, colE[g], Zd + (c0 + g) * ldd + r0 + part * 16, plane);
  }
}

// One 64-row window of a test matrix X (N x s, row-major): its exponent and the digit planes of
// X^* (S x BNt rows of ldd entries; rows c >= s are zero).
template <int S>
__global__ void __launch_bounds__(256)
    oz_split_b(const double* __restrict__ X, int64_t N, int s, int BNt, int64_t ldd,
               uint16_t* __restrict__ out, int16_t* __restrict__ EB, int* status) {
  __shared__ uint64_t wmax[8];
  __shared__ int wexp;
  const int64_t k0 = static_cast<int64_t>(blockIdx.x) * 64;
  const int t = threadIdx.x;
  uint64_t m = 0;
  for (int e = t; e < 64 * s; e += 256) {
    const int64_t k = k0 + e / s;
    if (k < N) m = umax64(m, abs_bits(X[k * s + e % s]));
  }
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) m = umax64(m, __shfl_xor_sync(0xffffffffu, m, o));
  if ((t & 31) == 0) wmax[t >> 5] = m;
  __syncthreads();
  if (t == 0) {
    uint64_t mm = 0;
    for (int i = 0; i < 8; ++i) mm = umax64(mm, wmax[i]);
    wexp = block_exponent(mm, status);
    EB[blockIdx.x] = static_cast<int16_t>(wexp);
  }
  __syncthreads();
  const int E = wexp;
  const size_t plane = static_cast<size_t>(BNt) * ldd;
  for (int e = t; e < BNt * 64; e += 256) {
    const int c = e >> 6, kk = e & 63;
    const int64_t k = k0 + kk;
    const double x = (c < s && k < N) ? X[k * s + c] : 0.0;
    int d[S];
    to_digits<S>(x, E, d);
#pragma unroll
    for (int i = 0; i < S; ++i)
      out[i * plane + static_cast<size_t>(c) * ldd + k] = static_cast<uint16_t>(digit_bf16(d[i]));
  }
}

// ---- the digit-product kernel ----------------------------------------------------------------

struct OzArgs {
  int M;               // rows of C (= N)
  int W;               // 64-wide windows of the reduction
  int BN, BNt;         // columns per CTA tile; padded columns of the product
  int wchunk;          // windows per reduction split (<= kMaxWindowsPerSplit)
  const int16_t* EA;   // [M][W] exponent of row m of op(A) over window w
  const int16_t* EB;   // [W] exponent of the test matrix over window w
  float2* partial;     // [splits][M][BNt] (hi, lo), in units of 2^rexp
  int* rexp;           // [splits][M] reference exponent of each split's row sums
  int* status;
};

__device__ __forceinline__ float pow2f(int e) {
  return (e >= -126 && e <= 127) ? __int_as_float((e + 127) << 23) : 0.0f;
}

template <int S>
__global__ void __launch_bounds__(kOzThreads, 1)
    oz_gemm(const __grid_constant__ CUtensorMap tmA, const __grid_constant__ CUtensorMap tmB,
            OzArgs a) {
  extern __shared__ uint8_t smem_raw[];
  if (aborted(a.status)) return;
  uint8_t* smem = smem_raw + ((1024u - (su32(smem_raw) & 1023u)) & 1023u);
  const int BN = a.BN;
  const int tile_b = BN * 128;
  uint8_t* opA = smem;                                   // S digit tiles of A
  uint8_t* opB = opA + S * kDigitTileA;                  // S digit tiles of the test matrix
  uint64_t* full = reinterpret_cast<uint64_t*>(opB + S * tile_b);   // S: digit i landed
  uint64_t* empty = full + S;                            // the window's MMAs are done
  uint64_t* acc_full = empty + 1;                        // 2
  uint64_t* acc_empty = acc_full + 2;                    // 2
  uint64_t* mma_done = acc_empty + 2;
  uint32_t* tmem_slot = reinterpret_cast<uint32_t*>(mma_done + 1);

  const int warp = threadIdx.x / 32, lane = threadIdx.x % 32;
  const int m0 = blockIdx.x * OBM;
  const int n0 = blockIdx.z * BN;
  const int w_begin = blockIdx.y * a.wchunk;
  const int nw = max(0, min(a.W, w_begin + a.wchunk) - w_begin);
  constexpr uint32_t kTmemCols = 512;                    // acc0, acc1, hi, lo
  constexpr uint32_t kHi = 256, kLo = 384;

  if (threadIdx.x == 0) {
    for (int i = 0; i < S; ++i) mbar_init(&full[i], 1);
    mbar_init(empty, 1);
    for (int i = 0; i < 2; ++i) {
      mbar_init(&acc_full[i], 1);
      mbar_init(&acc_empty[i], 8);
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
    if (lane == 0) {                                     // ---- TMA producer ----
      bool ok = true;
      int issued = 0;                                    // windows whose loads were issued
      for (int w = 0; w < nw && ok; ++w) {
        if (w > 0) ok = mbar_wait(empty, (w - 1) & 1, a.status);
        if (!ok) break;
        const int k0 = (w_begin + w) * OBK;
#pragma unroll
        for (int i = 0; i < S; ++i) {
          mbar_expect_tx(&full[i], kDigitTileA + tile_b);
          tma_load_2d(opA + i * kDigitTileA, &tmA, &full[i], k0, i * a.M + m0);
          tma_load_2d(opB + i * tile_b, &tmB, &full[i], k0, i * a.BNt + n0);
        }
        issued = w + 1;
      }
      if (issued > 0)                                    // copies must land before exit
        for (int i = 0; i < S; ++i) mbar_wait(&full[i], (issued - 1) & 1, a.status, false);
    }
  } else if (warp == 1) {
    if (lane == 0) {                                     // ---- MMA issuer ----
      const uint32_t idesc = idesc_bf16(OBM, BN);
      const uint32_t abase = su32(opA), bbase = su32(opB);
      bool ok = true;
      int g = 0;                                         // diagonals issued
      for (int w = 0; w < nw && ok; ++w) {
        for (int d = 0; d < S && ok; ++d, ++g) {
          const int b = g & 1;
          if (g >= 2) ok = mbar_wait(&acc_empty[b], ((g >> 1) - 1) & 1, a.status);
          if (ok) ok = mbar_wait(&full[d], w & 1, a.status);
          if (!ok) break;
          tc_fence_after();
          const uint32_t acc = tmem + static_cast<uint32_t>(b * 128);
          for (int i = 0; i <= d; ++i) {
            const uint64_t ad = sw128_desc(abase + i * kDigitTileA);
            const uint64_t bd = sw128_desc(bbase + (d - i) * tile_b);
#pragma unroll
            for (int kk = 0; kk < OBK / 16; ++kk)
              mma_bf16(acc, ad + 2 * kk, bd + 2 * kk, idesc, (i == 0 && kk == 0) ? 0u : 1u);
          }
          mma_commit(&acc_full[b]);
        }
        if (ok) mma_commit(empty);
      }
      mma_commit(mma_done);                              // all issued MMAs finished
      mbar_wait(mma_done, 0, a.status, false);
    }
  } else {                                               // ---- drain (warps 2..9) ----
    const int quarter = warp & 3;                        // TMEM lanes 32*quarter .. +31
    const int half = (warp - 2) >> 2;                    // 32-column chunks c with c % 2 == half
    const uint32_t lane_base = static_cast<uint32_t>(quarter * 32) << 16;
    const int row = m0 + quarter * 32 + lane;
    int RA = kNoExp, RB = kNoExp;                        // largest exponents over the range
    for (int w = w_begin; w < w_begin + nw; ++w) {
      if (row < a.M) RA = max(RA, static_cast<int>(a.EA[static_cast<size_t>(row) * a.W + w]));
      RB = max(RB, static_cast<int>(a.EB[w]));
    }
    const int nchunks = BN / 32;
    bool ok = true;
    int g = 0;
    for (int w = 0; w < nw && ok; ++w) {
      const int wabs = w_begin + w;
      const int ea = row < a.M ? a.EA[static_cast<size_t>(row) * a.W + wabs] : kNoExp;
      const int eb = a.EB[wabs];
      const bool zero = (ea == kNoExp || eb == kNoExp);
      const int base = (ea - RA) + (eb - RB) - 16;
      for (int d = 0; d < S && ok; ++d, ++g) {
        const int b = g & 1;
        ok = mbar_wait(&acc_full[b], (g >> 1) & 1, a.status);
        if (!ok) break;
        tc_fence_after();
        const float scale = zero ? 0.0f : pow2f(base - 8 * d);
        for (int c = half; c < nchunks; c += 2) {
          uint32_t x[32], hi[32], lo[32];
          tmem_ld32(tmem + lane_base + static_cast<uint32_t>(b * 128 + 32 * c), x);
          if (g == 0) {
#pragma unroll
            for (int j = 0; j < 32; ++j) {
              hi[j] = __float_as_uint(__fmul_rn(__uint_as_float(x[j]), scale));
              lo[j] = 0u;
            }
          } else {
            tmem_ld32(tmem + lane_base + kHi + static_cast<uint32_t>(32 * c), hi);
            tmem_ld32(tmem + lane_base + kLo + static_cast<uint32_t>(32 * c), lo);
#pragma unroll
            for (int j = 0; j < 32; ++j) {   // (hi, lo) += x * scale: TwoSum, then renormalise
              const float h = __uint_as_float(hi[j]);
              const float v = __fmul_rn(__uint_as_float(x[j]), scale);
              const float s = __fadd_rn(h, v);
              const float bp = __fsub_rn(s, h);
              const float err = __fadd_rn(__fsub_rn(h, __fsub_rn(s, bp)), __fsub_rn(v, bp));
              const float t = __fadd_rn(__uint_as_float(lo[j]), err);
              const float h2 = __fadd_rn(s, t);
              hi[j] = __float_as_uint(h2);
              lo[j] = __float_as_uint(__fsub_rn(t, __fsub_rn(h2, s)));
            }
          }
          tmem_st32(tmem + lane_base + kHi + static_cast<uint32_t>(32 * c), hi);
          tmem_st32(tmem + lane_base + kLo + static_cast<uint32_t>(32 * c), lo);
        }
        tc_fence_before();
        __syncwarp();
        if (lane == 0) mbar_arrive(&acc_empty[b]);
      }
    }
    tc_fence_after();
    float2* out = a.partial + (static_cast<size_t>(blockIdx.y) * a.M + row) * a.BNt + n0;
    if (half == 0 && row < a.M)
      a.rexp[static_cast<size_t>(blockIdx.y) * a.M + row] =
          (RA == kNoExp || RB == kNoExp) ? 0 : RA + RB;
    if (ok && g == nw * S && nw > 0) {
      for (int c = half; c < nchunks; c += 2) {
        uint32_t hi[32], lo[32];
        tmem_ld32(tmem + lane_base + kHi + static_cast<uint32_t>(32 * c), hi);
        tmem_ld32(tmem + lane_base + kLo + static_cast<uint32_t>(32 * c), lo);
        if (row < a.M) {
#pragma unroll
          for (int j = 0; j < 32; j += 2)
            *reinterpret_cast<float4*>(out + 32 * c + j) =
                make_float4(__uint_as_float(hi[j]), __uint_as_float(lo[j]),
                            __uint_as_float(hi[j + 1]), __uint_as_float(lo[j + 1]));
        }
      }
    } else if (nw == 0 && row < a.M) {
      for (int c = half; c < nchunks; c += 2)
        for (int j = 0; j < 32; ++j) out[32 * c + j] = make_float2(0.f, 0.f);
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

// C[i][c] = sum over splits of 2^rexp (hi + lo), in FP64, in split order.
__global__ void oz_reduce(const float2* __restrict__ partial, const int* __restrict__ rexp,
                          int splits, int64_t M, int BNt, int s, double* __restrict__ C) {
  const int64_t total = M * s;
  for (int64_t idx = blockIdx.x * static_cast<int64_t>(blockDim.x) + threadIdx.x; idx < total;
       idx += static_cast<int64_t>(gridDim.x) * blockDim.x) {
    const int64_t i = idx / s;
    const int c = static_cast<int>(idx % s);
    double acc = 0.0;
    for (int sp = 0; sp < splits; ++sp) {
      const float2 p = partial[(sp * M + i) * BNt + c];
      acc += scalbn(static_cast<double>(p.x) + static_cast<double>(p.y), rexp[sp * M + i]);
    }
    C[idx] = acc;
  }
}

// ---- host side ------------------------------------------------------------------------------

std::mutex g_oz_mutex;
struct OzScratch {
  void* ptr = nullptr;
  size_t bytes = 0;
};
std::vector<OzScratch> g_oz_scratch;

cudaError_t oz_scratch(size_t bytes, void** out) {
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return e;
  std::lock_guard<std::mutex> lock(g_oz_mutex);
  if (static_cast<int>(g_oz_scratch.size()) <= dev) g_oz_scratch.resize(dev + 1);
  OzScratch& s = g_oz_scratch[dev];
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
    e = cudaMemset(s.ptr, 0, 1024);                      // status word starts clear
    if (e != cudaSuccess) return e;
  }
  *out = s.ptr;
  return cudaSuccess;
}

size_t align1k(size_t b) { return (b + 1023) / 1024 * 1024; }

size_t oz_smem_bytes(int S, int BN) {
  return static_cast<size_t>(S) * (kDigitTileA + BN * 128) + 256 + 1024;
}

template <int S>
cudaError_t launch_products(const double* A, int64_t lda, int64_t N, const double* Om,
                            const double* Ps, int s, double* Y, double* Z, cudaStream_t st) {
  int BN, BNt;
  column_tiles(s, &BN, &BNt);
  const int64_t ldd = (N + 63) / 64 * 64;
  const int W = static_cast<int>((N + OBK - 1) / OBK);
  const int64_t mtiles = (N + OBM - 1) / OBM;
  const int64_t tiles = mtiles * (BNt / BN);
  int splits = std::max<int>((W + kMaxWindowsPerSplit - 1) / kMaxWindowsPerSplit,
                             static_cast<int>((2 * 152 + tiles - 1) / tiles));
  splits = std::min(splits, W);
  const int wchunk = (W + splits - 1) / splits;
  splits = (W + wchunk - 1) / wchunk;

  const size_t a_planes = static_cast<size_t>(S) * N * ldd * 2;
  const size_t b_planes = static_cast<size_t>(S) * BNt * ldd * 2;
  const size_t etab = static_cast<size_t>(N) * W * 2;
  const size_t off_yd = 1024, off_zd = off_yd + align1k(a_planes);
  const size_t off_ey = off_zd + align1k(a_planes), off_ez = off_ey + align1k(etab);
  const size_t off_bo = off_ez + align1k(etab), off_bp = off_bo + align1k(b_planes);
  const size_t off_eo = off_bp + align1k(b_planes), off_ep = off_eo + align1k(W * 2);
  const size_t off_rexp = off_ep + align1k(W * 2);
  const size_t off_part = off_rexp + align1k(static_cast<size_t>(splits) * N * sizeof(int));
  const size_t total = off_part + static_cast<size_t>(splits) * N * BNt * sizeof(float2);
  void* scratch = nullptr;
  cudaError_t e = oz_scratch(total, &scratch);
  if (e != cudaSuccess) return e;
  uint8_t* base = static_cast<uint8_t*>(scratch);
  int* status = reinterpret_cast<int*>(base);
  auto* Yd = reinterpret_cast<uint16_t*>(base + off_yd);
  auto* Zd = reinterpret_cast<uint16_t*>(base + off_zd);
  auto* EY = reinterpret_cast<int16_t*>(base + off_ey);
  auto* EZ = reinterpret_cast<int16_t*>(base + off_ez);
  auto* Bo = reinterpret_cast<uint16_t*>(base + off_bo);
  auto* Bp = reinterpret_cast<uint16_t*>(base + off_bp);
  auto* EO = reinterpret_cast<int16_t*>(base + off_eo);
  auto* EP = reinterpret_cast<int16_t*>(base + off_ep);
  auto* rexp = reinterpret_cast<int*>(base + off_rexp);
  auto* partial = reinterpret_cast<float2*>(base + off_part);

  oz_split_a<S><<<dim3(W, W), 256, 0, st>>>(A, lda, N, Yd, Zd, ldd, EY, EZ, W, status);
  oz_split_b<S><<<W, 256, 0, st>>>(Om, N, s, BNt, ldd, Bo, EO, status);
  oz_split_b<S><<<W, 256, 0, st>>>(Ps, N, s, BNt, ldd, Bp, EP, status);
  e = cudaGetLastError();
  if (e != cudaSuccess) return e;

  CUtensorMap mAy, mAz, mBo, mBp;
  const uint64_t row_bytes = static_cast<uint64_t>(ldd) * 2;
  if (!make_map(&mAy, CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, Yd, N, S * N, row_bytes, OBK, OBM,
                CU_TENSOR_MAP_SWIZZLE_128B) ||
      !make_map(&mAz, CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, Zd, N, S * N, row_bytes, OBK, OBM,
                CU_TENSOR_MAP_SWIZZLE_128B) ||
      !make_map(&mBo, CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, Bo, N, S * BNt, row_bytes, OBK, BN,
                CU_TENSOR_MAP_SWIZZLE_128B) ||
      !make_map(&mBp, CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, Bp, N, S * BNt, row_bytes, OBK, BN,
                CU_TENSOR_MAP_SWIZZLE_128B))
    return cudaErrorInvalidValue;

  auto kernel = oz_gemm<S>;
  const size_t smem = oz_smem_bytes(S, BN);
  e = cudaFuncSetAttribute(kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                           static_cast<int>(smem));
  if (e != cudaSuccess) return e;
  const dim3 grid(static_cast<unsigned>(mtiles), static_cast<unsigned>(splits),
                  static_cast<unsigned>(BNt / BN));
  const unsigned rg = 152u * 8u;
  OzArgs ay{static_cast<int>(N), W, BN, BNt, wchunk, EY, EO, partial, rexp, status};
  kernel<<<grid, kOzThreads, smem, st>>>(mAy, mBo, ay);
  oz_reduce<<<rg, 256, 0, st>>>(partial, rexp, splits, N, BNt, s, Y);
  e = cudaGetLastError();
  if (e != cudaSuccess) return e;
  OzArgs az{static_cast<int>(N), W, BN, BNt, wchunk, EZ, EP, partial, rexp, status};
  kernel<<<grid, kOzThreads, smem, st>>>(mAz, mBp, az);
  oz_reduce<<<rg, 256, 0, st>>>(partial, rexp, splits, N, BNt, s, Z);
  return cudaGetLastError();
}

}  // namespace

cudaError_t launch_sample_dense_oz(const double* A, int64_t lda, int64_t N, const double* Om,
                                   const double* Ps, int s, double* Y, double* Z, int digits,
                                   cudaStream_t st) {
  if (s < 1 || s > 256 || N < 1 || N > (int64_t(1) << 20) || lda < N)
    return cudaErrorInvalidValue;
  int BN, BNt;
  column_tiles(s, &BN, &BNt);
  if (oz_smem_bytes(digits, BN) > kMaxNodeSmemBytes) return cudaErrorInvalidValue;
  if (digits == 6) return launch_products<6>(A, lda, N, Om, Ps, s, Y, Z, st);
  if (digits == 7) return launch_products<7>(A, lda, N, Om, Ps, s, Y, Z, st);
  return cudaErrorInvalidValue;
}

cudaError_t sample_oz_status(int* host_status, bool clear) {
  *host_status = 0;
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return e;
  int* status = nullptr;
  {
    std::lock_guard<std::mutex> lock(g_oz_mutex);
    if (dev < static_cast<int>(g_oz_scratch.size())) status = static_cast<int*>(g_oz_scratch[dev].ptr);
  }
  if (!status) return cudaSuccess;
  e = cudaMemcpy(host_status, status, sizeof(int), cudaMemcpyDeviceToHost);
  if (e == cudaSuccess && clear) e = cudaMemset(status, 0, sizeof(int));
  return e;
}

}  // namespace hbs
