// FP64-class sampling Y = A Omega, Z = A^* Psi (Algorithm 2, first block) on the tcgen05 tensor
// cores by exact products of 8-bit digits: an error-free splitting in the manner of Ozaki,
// Ogita, Oishi and Rump (Numer. Algorithms 59, 2012), with FP16 digits and FP32
// accumulation instead of FP64 slices.
//
// Digits. A block of FP64 entries that shares one exponent E (every |x| < 2^(E-1), the largest
// >= 2^(E-2)) is scaled to the integers X = round(x 2^(8S-E)), |X| <= 2^(8S-1), and each X is
// written in balanced base 256: X = sum_{i<S} d_i 256^(S-1-i), d_i in [-128, 128]. Then
// x = sum_i d_i 2^(E-8(i+1)) to within 2^(E-8S-1), and every digit is exact in FP16.
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
// FP16 tile products per window; each dropped pair weighs at most 2^(2-8S) of max|a| max|b|.
//
// Accumulation. The diagonal d of a window is one accumulator in tensor memory (four of them,
// several): the MMA thread fills one while eight drain warps scale another by its power of
// two (exact) and add it to a double-float running sum kept in registers (hi + lo: the leading
// diagonals by TwoSum in FP32, hi exact and its rounding error collected in lo; the trailing
// ones, far below the sum, by one FMA into lo). A CTA's reduction range is at most 32 windows
// (2048 indices); the ranges are summed in FP64 by the reduce kernel. Within a range, scales are taken relative to the largest block
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
#include <cuda_fp16.h>
#include <cudaTypedefs.h>

#include <algorithm>
#include <mutex>
#include <vector>

#include "hbs_internal.cuh"
#include "tc_ptx.cuh"

namespace hbs {
namespace {

constexpr int kDrainWarps = 8;                  // two per quarter of tensor-memory lanes
constexpr int kOzThreads = 64 + 32 * kDrainWarps;
constexpr int OBM = 128;                       // rows of C per CTA (MMA M)
constexpr int OBK = 64;                        // window: reduction indices per digit tile
constexpr int kDigitTileA = OBM * OBK * 2;     // one FP16 digit tile of A
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

// round(x 2^(8S - E)) for |x| < 2^(E-1): an integer of magnitude <= 2^(8S-1).
template <int S>
__device__ __forceinline__ int64_t scaled_integer(double x, int E) {
  const uint64_t u = static_cast<uint64_t>(__double_as_longlong(x));
  const int ex = static_cast<int>((u >> 52) & 0x7ff);
  uint64_t m = u & ((1ull << 52) - 1);
  int p = -1074;                                        // |x| = m 2^p
  if (ex != 0) {
    m |= 1ull << 52;
    p = ex - 1075;
  }
  // m 2^sh < 2^(8S-1): sh <= 2 for normal x, up to 8S - 2 for a block of subnormals
  const int sh = p + 8 * S - E;
  uint64_t X = 0;
  if (E != kNoExp && m != 0 && ex != 0x7ff) {
    if (sh >= 0) X = m << min(sh, 63);
    else if (sh > -60) X = (m + (1ull << (-sh - 1))) >> (-sh);
  }
  return (u >> 63) ? -static_cast<int64_t>(X) : static_cast<int64_t>(X);
}

// The balanced base-256 digits of X (d_i in [-128, 127], the leading one in [-128, 128]) are
// the bytes of V = X + 128 (256^(S-1) + ... + 1) less 128 each (the leading one: V's bits from
// 8(S-1) up), with no carries to propagate.
template <int S>
__device__ __forceinline__ uint64_t digit_offset() {
  uint64_t c = 0;
#pragma unroll
  for (int i = 0; i < S; ++i) c = (c << 8) | 128u;
  return c;
}

// V for one entry, as two 32-bit words. Normal entries (and zeros) take a branch-free integer
// path: |x| = m 2^(ex - 1075) with m < 2^53, and X = round(m 2^(2 - t)) with
// t = E + 1077 - 8S - ex >= 0 (E bounds the block), i.e. ((8m >> t) + 1) >> 1, round half up.
// Subnormal and non-finite entries take the general form.
template <int S>
__device__ __forceinline__ void offset_value(double x, int E, uint32_t& vl, uint32_t& vh) {
  const uint32_t lx = static_cast<uint32_t>(__double2loint(x));
  const uint32_t hx = static_cast<uint32_t>(__double2hiint(x));
  const int ex = static_cast<int>((hx >> 20) & 0x7ffu);
  uint64_t X;
  if ((ex == 0 && ((hx & 0xfffffu) | lx) != 0u) || ex == 0x7ff) {
    const int64_t xi = scaled_integer<S>(x, E);
    X = static_cast<uint64_t>(xi < 0 ? -xi : xi);
  } else {
    const uint32_t mh = (hx & 0xfffffu) | (ex != 0 ? 0x100000u : 0u);
    const uint64_t u = ((static_cast<uint64_t>(mh) << 32) | lx) << 3;
    const int t = min(63, max(0, E + 1077 - 8 * S - ex));
    X = ((u >> t) + 1) >> 1;
  }
  const uint64_t sgn = (hx >> 31) ? ~0ull : 0ull;
  const uint64_t V = digit_offset<S>() + ((X ^ sgn) - sgn);
  vl = static_cast<uint32_t>(V);
  vh = static_cast<uint32_t>(V >> 32);
}

// FP16 bits of digit i (0: most significant) of two entries from their V words, packed (the
// first entry in the low half): the byte (9 bits for the leading digit) goes under the FP16
// exponent of 1024 (0x6400 | b = 1024 + b) and 1024 + 128 is subtracted, exactly, two at once.
template <int S>
__device__ __forceinline__ uint32_t digit_pair_f16(uint32_t l0, uint32_t h0, uint32_t l1,
                                                   uint32_t h1, int i) {
  static_assert(S >= 4 && S <= 7, "4 to 7 digits");
  const int k = S - 1 - i;                              // byte position from the bottom
  uint32_t w, mask = 0x00ff00ffu;
  if (S == 4 && k == S - 1) {                           // leading 9 bits straddle the two words
    const uint32_t b0 = __funnelshift_r(l0, h0, 24) & 0x1ffu;
    const uint32_t b1 = __funnelshift_r(l1, h1, 24) & 0x1ffu;
    w = b0 | (b1 << 16);
    mask = 0x01ff01ffu;
  } else if (k == S - 1) {
    const uint32_t b = static_cast<uint32_t>(S - 5);    // leading byte in the high word
    w = __byte_perm(h0, h1, b | ((b + 1) << 4) | ((b + 4) << 8) | ((b + 5) << 12));
    mask = 0x01ff01ffu;
  } else if (k < 4) {
    const uint32_t b = static_cast<uint32_t>(k);
    w = __byte_perm(l0, l1, b | (b << 4) | ((b + 4) << 8) | ((b + 4) << 12));
  } else {
    const uint32_t b = static_cast<uint32_t>(k - 4);
    w = __byte_perm(h0, h1, b | (b << 4) | ((b + 4) << 8) | ((b + 4) << 12));
  }
  w = (w & mask) | 0x64006400u;
  const __half2 d = __hsub2(*reinterpret_cast<const __half2*>(&w),
                            __halves2half2(__ushort_as_half(0x6480), __ushort_as_half(0x6480)));
  return *reinterpret_cast<const uint32_t*>(&d);
}

// V for one entry of a block whose exponent E lies above 8S - 1020: there every subnormal
// entry (< 2^-1022) scales to below 1/2 and rounds to 0, so one select replaces the general
// form's test. Normal entries take the integer path of offset_value (t >= 56 - 8S >= 0 since the
// entry is below 2^(E-1)); an Inf or NaN, already flagged by the block exponent, gives a value
// that is not used.
template <int S>
__device__ __forceinline__ void offset_value_normal(double x, int E, uint32_t& vl, uint32_t& vh) {
  const uint32_t lx = static_cast<uint32_t>(__double2loint(x));
  const uint32_t hx = static_cast<uint32_t>(__double2hiint(x));
  const int ex = static_cast<int>((hx >> 20) & 0x7ffu);
  const uint32_t mh = (hx & 0xfffffu) | 0x100000u;
  const uint64_t u = ((static_cast<uint64_t>(mh) << 32) | lx) << 3;
  const int t = min(63, E + 1077 - 8 * S - ex);
  const uint64_t X = ex == 0 ? 0ull : ((u >> t) + 1) >> 1;
  const uint64_t V = (hx >> 31) ? digit_offset<S>() - X : digit_offset<S>() + X;
  vl = static_cast<uint32_t>(V);
  vh = static_cast<uint32_t>(V >> 32);
}

template <int S>
__device__ __forceinline__ bool block_is_normal(int E) { return E > 8 * S - 1020; }

// FP16 digits of two neighbouring entries into S planes (plane_stride apart), one 32-bit store
// per plane. E is the same for the whole warp, so the choice of path is warp-uniform.
template <int S>
__device__ __forceinline__ void store_digit_pair(double x0, double x1, int E, uint16_t* dst,
                                                 size_t plane_stride) {
  uint32_t l0, h0, l1, h1;
  if (block_is_normal<S>(E)) {
    offset_value_normal<S>(x0, E, l0, h0);
    offset_value_normal<S>(x1, E, l1, h1);
  } else {
    offset_value<S>(x0, E, l0, h0);
    offset_value<S>(x1, E, l1, h1);
  }
#pragma unroll
  for (int i = 0; i < S; ++i)
    *reinterpret_cast<uint32_t*>(dst + i * plane_stride) = digit_pair_f16<S>(l0, h0, l1, h1, i);
}

__device__ __forceinline__ uint64_t umax64(uint64_t a, uint64_t b) { return a > b ? a : b; }

// The block exponent of 64 entries held two per lane: the largest magnitude's high word is
// found with one warp reduction (its exponent field, and its leading bit when subnormal); the
// low words matter only when every high word is zero.
__device__ __forceinline__ int pair_block_exponent(double x0, double x1, int* status) {
  const uint32_t a0 = static_cast<uint32_t>(__double2hiint(x0)) & 0x7fffffffu;
  const uint32_t a1 = static_cast<uint32_t>(__double2hiint(x1)) & 0x7fffffffu;
  const uint32_t hm = __reduce_max_sync(0xffffffffu, max(a0, a1));
  if (hm != 0u) return block_exponent(static_cast<uint64_t>(hm) << 32, status);
  const uint32_t lm = __reduce_max_sync(0xffffffffu, max(static_cast<uint32_t>(__double2loint(x0)),
                                                          static_cast<uint32_t>(__double2loint(x1))));
  return block_exponent(static_cast<uint64_t>(lm), status);
}

// One 64 x 64 block of A: exponents per row (EY) and per column (EZ), digit planes of A (Yd,
// row-major) and of A^* (Zd). Planes: S x N rows of ldd entries; ldd a multiple of 64.
// Warp w handles rows (then columns) 8w .. 8w+7; lane l the neighbouring entries 2l and 2l + 1
// along them, so that each digit plane gets one 32-bit store per lane (128 contiguous bytes
// per warp).
template <int S>
__global__ void __launch_bounds__(256)
    oz_split_a(const double* __restrict__ A, int64_t lda, int64_t N, uint16_t* __restrict__ Yd,
               uint16_t* __restrict__ Zd, int64_t ldd, int16_t* __restrict__ EY,
               int16_t* __restrict__ EZ, int W, int* status) {
  __shared__ double tile[64][65];
  const int64_t r0 = static_cast<int64_t>(blockIdx.y) * 64, c0 = static_cast<int64_t>(blockIdx.x) * 64;
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
#pragma unroll
  for (int rr = 0; rr < 8; ++rr) {
    const int r = warp * 8 + rr;
    const int64_t gr = r0 + r;
#pragma unroll
    for (int h = 0; h < 2; ++h) {
      const int64_t gc = c0 + lane + 32 * h;
      tile[r][lane + 32 * h] = (gr < N && gc < N) ? A[gr * lda + gc] : 0.0;
    }
  }
  __syncthreads();
  const size_t plane = static_cast<size_t>(N) * ldd;
#pragma unroll 1
  for (int rr = 0; rr < 8; ++rr) {                    // rows of A: digits for Y = A Omega
    const int r = warp * 8 + rr;
    const double x0 = tile[r][2 * lane], x1 = tile[r][2 * lane + 1];
    const int E = pair_block_exponent(x0, x1, status);
    if (r0 + r >= N) continue;
    if (lane == 0) EY[(r0 + r) * W + blockIdx.x] = static_cast<int16_t>(E);
    store_digit_pair<S>(x0, x1, E, Yd + (r0 + r) * ldd + c0 + 2 * lane, plane);
  }
#pragma unroll 1
  for (int cc = 0; cc < 8; ++cc) {                    // columns of A: digits for Z = A^* Psi
    const int c = warp * 8 + cc;
    const double x0 = tile[2 * lane][c], x1 = tile[2 * lane + 1][c];
    const int E = pair_block_exponent(x0, x1, status);
    if (c0 + c >= N) continue;
    if (lane == 0) EZ[(c0 + c) * W + blockIdx.y] = static_cast<int16_t>(E);
    store_digit_pair<S>(x0, x1, E, Zd + (c0 + c) * ldd + r0 + 2 * lane, plane);
  }
}

// One 64 x 64 block of A with a single exponent for the whole block: the digit planes of A in
// row-major order only (the product with A^* reads them transposed, an MN-major operand), and
// that exponent as the per-row (EY) and per-column (EZ) exponents of the block. Half the
// digit work of oz_split_a; entries far below their block's largest lose the corresponding
// low bits (used with 5 digits, whose products are not FP64-class anyway).
template <int S>
__global__ void __launch_bounds__(256)
    oz_split_shared(const double* __restrict__ A, int64_t lda, int64_t N, uint16_t* __restrict__ Yd,
                    int64_t ldd, int16_t* __restrict__ EY, int16_t* __restrict__ EZ, int W,
                    int* status) {
  __shared__ double tile[64][65];
  __shared__ int wexp[8];
  const int64_t r0 = static_cast<int64_t>(blockIdx.y) * 64, c0 = static_cast<int64_t>(blockIdx.x) * 64;
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
#pragma unroll
  for (int rr = 0; rr < 8; ++rr) {
    const int r = warp * 8 + rr;
    const int64_t gr = r0 + r;
#pragma unroll
    for (int h = 0; h < 2; ++h) {
      const int64_t gc = c0 + lane + 32 * h;
      tile[r][lane + 32 * h] = (gr < N && gc < N) ? A[gr * lda + gc] : 0.0;
    }
  }
  __syncthreads();
  int Em = kNoExp;                                     // the block's exponent: the largest row's
#pragma unroll 1
  for (int rr = 0; rr < 8; ++rr) {
    const int r = warp * 8 + rr;
    Em = max(Em, pair_block_exponent(tile[r][2 * lane], tile[r][2 * lane + 1], status));
  }
  if (lane == 0) wexp[warp] = Em;
  __syncthreads();
  int E = wexp[0];
#pragma unroll
  for (int w = 1; w < 8; ++w) E = max(E, wexp[w]);
  const size_t plane = static_cast<size_t>(N) * ldd;
#pragma unroll 1
  for (int rr = 0; rr < 8; ++rr) {
    const int r = warp * 8 + rr;
    if (r0 + r >= N) continue;
    if (lane == 0) EY[(r0 + r) * W + blockIdx.x] = static_cast<int16_t>(E);
    store_digit_pair<S>(tile[r][2 * lane], tile[r][2 * lane + 1], E, Yd + (r0 + r) * ldd + c0 + 2 * lane,
                        plane);
  }
  if (threadIdx.x < 64 && c0 + threadIdx.x < N)
    EZ[(c0 + threadIdx.x) * W + blockIdx.y] = static_cast<int16_t>(E);
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
    uint32_t vl, vh;
    if (block_is_normal<S>(E)) offset_value_normal<S>(x, E, vl, vh);
    else offset_value<S>(x, E, vl, vh);
#pragma unroll
    for (int i = 0; i < S; ++i)
      out[i * plane + static_cast<size_t>(c) * ldd + k] =
          static_cast<uint16_t>(digit_pair_f16<S>(vl, vh, vl, vh, i));
  }
}

// ---- the digit-product kernel ----------------------------------------------------------------

struct OzArgs {
  int M;               // rows of C (= N)
  int W;               // 64-wide windows of the reduction
  int BN, BNt;         // columns per CTA tile; padded columns of the product
  int wchunk;          // windows per reduction split (<= kMaxWindowsPerSplit)
  int slots;           // digit slots of the shared-memory ring (S .. kMaxSlots)
  const int16_t* EA;   // [M][W] exponent of row m of op(A) over window w
  const int16_t* EB;   // [W] exponent of the test matrix over window w
  float2* partial;     // [splits][M][BNt] (hi, lo), in units of 2^rexp
  int* rexp;           // [splits][M] reference exponent of each split's row sums (kEmptyRange: 0)
  int* status;
};

constexpr int kAccBufs = 4;          // accumulators in tensor memory, 128 columns each
constexpr int kMaxSlots = 11;        // digit slots: 2 mbarriers each in the 256-byte barrier area
// Diagonals added to the running sum by TwoSum (hi exact, its rounding error into lo); the later
// ones weigh < 2^-8 kExactDiags of diagonal 0 and go into lo with one FMA. FP64-class products
// (S >= 6) take 4 (later terms < 2^-32 of the sum, each rounded to 2^-56 of it); the 5-digit
// products, whose own truncation is ~2^-38, take 3 (later terms < 2^-24, rounded to 2^-48).
template <int S>
__host__ __device__ constexpr int exact_diags() { return S >= 6 ? 4 : 3; }
constexpr int kEmptyRange = -(1 << 20);

__device__ __forceinline__ float pow2f(int e) {
  return (e >= -126 && e <= 127) ? __int_as_float((e + 127) << 23) : 0.0f;
}

// (hi, lo) += v: TwoSum, then a Fast2Sum renormalisation that keeps |lo| <= ulp(hi) / 2.
__device__ __forceinline__ void df_add(float& hi, float& lo, float v) {
  const float s = __fadd_rn(hi, v);
  const float bp = __fsub_rn(s, hi);
  const float err = __fadd_rn(__fsub_rn(hi, __fsub_rn(s, bp)), __fsub_rn(v, bp));
  const float t = __fadd_rn(lo, err);
  const float h2 = __fadd_rn(s, t);
  lo = __fsub_rn(t, __fsub_rn(h2, s));
  hi = h2;
}

// hi += v exactly by TwoSum, the rounding error of hi added to lo (no renormalisation: each
// error is at most ulp(hi) / 2, so over the <= 32 windows of a split |lo| stays below ~2^6 ulp(hi)
// and its own roundings below 2^-40 of hi).
__device__ __forceinline__ void two_sum_acc(float& hi, float& lo, float v) {
  const float s = __fadd_rn(hi, v);
  const float bp = __fsub_rn(s, hi);
  const float err = __fadd_rn(__fsub_rn(hi, __fsub_rn(s, bp)), __fsub_rn(v, bp));
  hi = s;
  lo = __fadd_rn(lo, err);
}

template <bool ACC>
__device__ __forceinline__ void mma_f16_c(uint32_t tmem_d, uint64_t adesc, uint64_t bdesc,
                                           uint32_t idesc) {
  asm volatile(
      "{\n\t.reg .pred p;\n\t"
      "setp.ne.b32 p, %4, 0;\n\t"
      "tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n\t}" ::"r"(tmem_d),
      "l"(adesc), "l"(bdesc), "r"(idesc), "n"(ACC ? 1 : 0)
      : "memory");
}

// The MMAs of diagonal D: pairs (i, D - i), four K = 16 steps each; on the last diagonal in
// groups (k, S-1-k), (S-1-k, k), each group committed to the slots of digits k and S-1-k
// (freed[.]) so that the producer can refill them while the rest of the window runs. Fully
// unrolled with the descriptors of the digit tiles precomputed per window, so that the single
// issuing thread spends few instructions per MMA.
template <int S, int D, int ASTEP>
__device__ __forceinline__ void issue_diagonal(uint32_t acc, const uint64_t (&ad)[S],
                                               const uint64_t (&bd)[S], uint32_t idesc,
                                               uint64_t* (&freed)[S]) {
  if constexpr (D >= S) {
    return;                                             // no such diagonal (never called)
  } else if constexpr (D < S - 1) {
#pragma unroll
    for (int i = 0; i <= D; ++i)
#pragma unroll
      for (int kk = 0; kk < OBK / 16; ++kk) {
        if (i == 0 && kk == 0) mma_f16_c<false>(acc, ad[i] + ASTEP * kk, bd[D - i] + 2 * kk, idesc);
        else mma_f16_c<true>(acc, ad[i] + ASTEP * kk, bd[D - i] + 2 * kk, idesc);
      }
  } else {
    constexpr int G = (S + 1) / 2;
#pragma unroll
    for (int k = 0; k < G; ++k) {
#pragma unroll
      for (int t = 0; t < 2; ++t) {
        const int i = t == 0 ? k : S - 1 - k;
        if (t == 1 && i == k) continue;
#pragma unroll
        for (int kk = 0; kk < OBK / 16; ++kk) {
          if (k == 0 && t == 0 && kk == 0) mma_f16_c<false>(acc, ad[i] + ASTEP * kk, bd[D - i] + 2 * kk, idesc);
          else mma_f16_c<true>(acc, ad[i] + ASTEP * kk, bd[D - i] + 2 * kk, idesc);
        }
      }
      mma_commit(freed[k]);                             // digits k and S-1-k: their last use
      if (S - 1 - k != k) mma_commit(freed[S - 1 - k]);
    }
  }
}

// Drain warps: warp w covers TMEM lanes 32 (w % 4) .. + 31 (rows of the tile) and the 16-column
// chunks c = part + P cc of the BN columns (part = (w - 2) / 4, P = drain warps / 4); its running
// sums stay in registers. The drain shares each scheduler with the producer or the MMA thread,
// whose issue slots must not be crowded out, so it stays at two warps per scheduler.
// MN = true: the A operand is read transposed from row-major digit planes of A (Z = A^* Psi
// from the planes of A itself): each 128 x 64 digit tile is two TMA boxes of 64 reduction rows
// x 64 output columns (128-byte swizzled rows), an MN-major operand (instruction descriptor bit
// 15) whose two 64-column atoms lie 8 KB apart (leading byte offset) with 8-row groups 1 KB
// apart (stride byte offset); a K = 16 step advances 16 rows = 2 KB.
template <int S, bool MN = false>
__global__ void __launch_bounds__(kOzThreads, 1)
    oz_gemm(const __grid_constant__ CUtensorMap tmA, const __grid_constant__ CUtensorMap tmB,
            OzArgs a) {
  extern __shared__ uint8_t smem_raw[];
  if (aborted(a.status)) return;              // a CTA of this run timed out: nothing issued yet
  uint8_t* smem = smem_raw + ((1024u - (su32(smem_raw) & 1023u)) & 1023u);
  const int BN = a.BN;
  const int tile_b = BN * 128;
  const int NS = a.slots;                                // ring of digit slots (>= S)
  uint8_t* opA = smem;                                   // NS digit tiles of A
  uint8_t* opB = opA + NS * kDigitTileA;                 // NS digit tiles of the test matrix
  uint64_t* full = reinterpret_cast<uint64_t*>(opB + NS * tile_b);  // NS: slot's tiles landed
  uint64_t* empty = full + NS;                           // NS: slot's last MMAs are done
  uint64_t* acc_full = empty + NS;                       // kAccBufs
  uint64_t* acc_empty = acc_full + kAccBufs;             // kAccBufs
  uint64_t* mma_done = acc_empty + kAccBufs;
  uint32_t* tmem_slot = reinterpret_cast<uint32_t*>(mma_done + 1);

  const int warp = threadIdx.x / 32, lane = threadIdx.x % 32;
  const int m0 = blockIdx.x * OBM;
  const int n0 = blockIdx.z * BN;
  const int w_begin = blockIdx.y * a.wchunk;
  const int nw = max(0, min(a.W, w_begin + a.wchunk) - w_begin);
  constexpr uint32_t kTmemCols = 128 * kAccBufs;

  if (threadIdx.x == 0) {
    for (int q = 0; q < NS; ++q) {
      mbar_init(&full[q], 1);
      mbar_init(&empty[q], 1);
    }
    for (int i = 0; i < kAccBufs; ++i) {
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
    if (lane == 0) {                                     // ---- TMA producer ----
      // load j = w S + i (window w, digit i, in the order the diagonals need them) goes to
      // slot j mod NS once the slot's previous load, j - NS, has been consumed
      bool ok = true;
      int j = 0;                                         // loads issued
      int q = 0, lap = 0;                                // j mod NS, j / NS (no divisions)
      for (int w = 0; w < nw && ok; ++w) {
        const int k0 = (w_begin + w) * OBK;
        for (int i = 0; i < S; ++i, ++j) {
          if (lap > 0) ok = mbar_wait(&empty[q], (lap - 1) & 1, a.status);
          if (!ok) break;
          mbar_expect_tx(&full[q], kDigitTileA + tile_b);
          if constexpr (MN) {
            tma_load_2d(opA + q * kDigitTileA, &tmA, &full[q], m0, i * a.M + k0);
            tma_load_2d(opA + q * kDigitTileA + kDigitTileA / 2, &tmA, &full[q], m0 + 64,
                        i * a.M + k0);
          } else {
            tma_load_2d(opA + q * kDigitTileA, &tmA, &full[q], k0, i * a.M + m0);
          }
          tma_load_2d(opB + q * tile_b, &tmB, &full[q], k0, i * a.BNt + n0);
          if (++q == NS) {
            q = 0;
            ++lap;
          }
        }
        if (ok && w + 1 < nw) {                          // next window into L2 meanwhile
#pragma unroll
          for (int i = 0; i < S; ++i) {
            if constexpr (MN) {
              tma_prefetch_2d(&tmA, m0, i * a.M + k0 + OBK);
              tma_prefetch_2d(&tmA, m0 + 64, i * a.M + k0 + OBK);
            } else {
              tma_prefetch_2d(&tmA, k0 + OBK, i * a.M + m0);
            }
            tma_prefetch_2d(&tmB, k0 + OBK, i * a.BNt + n0);
          }
        }
      }
      // copies must land before exit: the last load of each slot (earlier ones were consumed
      // before the slot was refilled)
      for (int q = 0; q < NS && q < j; ++q) {
        const int loads = (j - 1 - q) / NS + 1;
        mbar_wait(&full[q], (loads - 1) & 1, a.status, false);
      }
    }
  } else if (warp == 1) {
    if (lane == 0) {                                     // ---- MMA issuer ----
      const uint32_t idesc = idesc_f16(OBM, BN) | (MN ? (1u << 15) : 0u);
      constexpr int kAStep = MN ? (16 * 128) >> 4 : 2;   // descriptor units per K = 16 step
      // descriptors of slot 0; slot q lies q tiles further (start address in 16-byte units)
      const uint64_t ad0 = MN ? sw128_desc_mn(su32(opA), kDigitTileA / 2) : sw128_desc(su32(opA));
      const uint64_t bd0 = sw128_desc(su32(opB));
      bool ok = true;
      int g = 0;                                         // diagonals issued
      int qb = 0, lb = 0;                                // slot and lap of load w S (digit 0)
      for (int w = 0; w < nw && ok; ++w) {
        uint64_t ad[S], bd[S];                           // this window's digits: slot (w S + i) mod NS
        uint64_t* freed[S];
        int qs[S], ph[S];                                // slot, and the parity of its load
#pragma unroll
        for (int i = 0; i < S; ++i) {
          const bool wrap = qb + i >= NS;                // S <= NS: at most one wrap
          qs[i] = wrap ? qb + i - NS : qb + i;
          ph[i] = (wrap ? lb + 1 : lb) & 1;
          ad[i] = ad0 + static_cast<uint64_t>(qs[i] * (kDigitTileA >> 4));
          bd[i] = bd0 + static_cast<uint64_t>(qs[i] * (tile_b >> 4));
          freed[i] = &empty[qs[i]];
        }
        qb += S;
        if (qb >= NS) {
          qb -= NS;
          ++lb;
        }
#pragma unroll
        for (int d = 0; d < S; ++d, ++g) {
          if (!ok) break;
          const int b = g % kAccBufs;
          if (g >= kAccBufs) ok = mbar_wait(&acc_empty[b], ((g / kAccBufs) - 1) & 1, a.status);
          if (ok) ok = mbar_wait(&full[qs[d]], ph[d], a.status);
          if (!ok) break;
          tc_fence_after();
          const uint32_t acc = tmem + static_cast<uint32_t>(b * 128);
          switch (d) {
            case 0: issue_diagonal<S, 0, kAStep>(acc, ad, bd, idesc, freed); break;
            case 1: issue_diagonal<S, 1, kAStep>(acc, ad, bd, idesc, freed); break;
            case 2: issue_diagonal<S, 2, kAStep>(acc, ad, bd, idesc, freed); break;
            case 3: issue_diagonal<S, 3, kAStep>(acc, ad, bd, idesc, freed); break;
            case 4: issue_diagonal<S, 4, kAStep>(acc, ad, bd, idesc, freed); break;
            case 5: issue_diagonal<S, 5, kAStep>(acc, ad, bd, idesc, freed); break;
            default: issue_diagonal<S, S - 1, kAStep>(acc, ad, bd, idesc, freed); break;
          }
          mma_commit(&acc_full[b]);
        }
      }
      mma_commit(mma_done);                              // all issued MMAs finished
      mbar_wait(mma_done, 0, a.status, false);
    }
  } else {                                               // ---- drain warps ----
    const int quarter = warp & 3;
    const int part = (warp - 2) >> 2;
    const uint32_t lane_base = static_cast<uint32_t>(quarter * 32) << 16;
    const int row = m0 + quarter * 32 + lane;
    int RA = kNoExp, RB = kNoExp;                        // largest exponents over the range
    for (int w = w_begin; w < w_begin + nw; ++w) {
      if (row < a.M) RA = max(RA, static_cast<int>(a.EA[static_cast<size_t>(row) * a.W + w]));
      RB = max(RB, static_cast<int>(a.EB[w]));
    }
    constexpr int P = kDrainWarps / 4;                   // drain warps per lane quarter
    constexpr int CPT = 8 / P;                           // 16-column chunks per thread
    const int nchunks = BN / 16;
    float hi[CPT][16], lo[CPT][16];
#pragma unroll
    for (int cc = 0; cc < CPT; ++cc)
#pragma unroll
      for (int j = 0; j < 16; ++j) hi[cc][j] = lo[cc][j] = 0.0f;
    bool ok = true;
    int g = 0;
    const size_t erow = static_cast<size_t>(row < a.M ? row : 0) * a.W;
    int ea_next = (row < a.M && nw > 0) ? a.EA[erow + w_begin] : kNoExp;
    for (int w = 0; w < nw && ok; ++w) {
      const int wabs = w_begin + w;
      const int ea = ea_next;                            // loaded a window ahead
      if (w + 1 < nw && row < a.M) ea_next = a.EA[erow + wabs + 1];
      const int eb = a.EB[wabs];
      const bool zero = (ea == kNoExp || eb == kNoExp);
      const int base = (ea - RA) + (eb - RB) - 16;
      for (int d = 0; d < S && ok; ++d, ++g) {
        const int b = g % kAccBufs;
        ok = mbar_wait(&acc_full[b], (g / kAccBufs) & 1, a.status);
        if (!ok) break;
        tc_fence_after();
        const float scale = zero ? 0.0f : pow2f(base - 8 * d);
#pragma unroll
        for (int cc = 0; cc < CPT; ++cc) {
          const int c = part + P * cc;
          if (c >= nchunks) continue;
          uint32_t x[16];
          tmem_ld16(tmem + lane_base + static_cast<uint32_t>(b * 128 + 16 * c), x);
          if (d < exact_diags<S>()) {
#pragma unroll
            for (int j = 0; j < 16; ++j)
              two_sum_acc(hi[cc][j], lo[cc][j], __fmul_rn(__uint_as_float(x[j]), scale));
          } else {                                        // below 2^-30 of the running sum
#pragma unroll
            for (int j = 0; j < 16; ++j) lo[cc][j] = __fmaf_rn(__uint_as_float(x[j]), scale, lo[cc][j]);
          }
        }
        tc_fence_before();
        __syncwarp();
        if (lane == 0) mbar_arrive(&acc_empty[b]);
      }
    }
    if (row < a.M) {
      if (part == 0)
        a.rexp[static_cast<size_t>(blockIdx.y) * a.M + row] =
            (RA == kNoExp || RB == kNoExp) ? kEmptyRange : RA + RB;
      if (ok && g == nw * S) {
        float2* out = a.partial + (static_cast<size_t>(blockIdx.y) * a.M + row) * a.BNt + n0;
#pragma unroll
        for (int cc = 0; cc < CPT; ++cc) {
          const int c = part + P * cc;
          if (c >= nchunks) continue;
#pragma unroll
          for (int j = 0; j < 16; j += 2)
            *reinterpret_cast<float4*>(out + 16 * c + j) =
                make_float4(hi[cc][j], lo[cc][j], hi[cc][j + 1], lo[cc][j + 1]);
        }
      }
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

// C[i][c] = sum over splits of 2^rexp (hi + lo): the splits' double-floats are brought to the
// row's largest split exponent R (exact powers of two), added as double-floats in split order,
// and the result is scaled by 2^R in FP64.
__global__ void oz_reduce(const float2* __restrict__ partial, const int* __restrict__ rexp,
                          int splits, int64_t M, int BNt, int s, double* __restrict__ C) {
  const int64_t total = M * s;
  for (int64_t idx = blockIdx.x * static_cast<int64_t>(blockDim.x) + threadIdx.x; idx < total;
       idx += static_cast<int64_t>(gridDim.x) * blockDim.x) {
    const int64_t i = idx / s;
    const int c = static_cast<int>(idx % s);
    int R = kEmptyRange;
    for (int sp = 0; sp < splits; ++sp) R = max(R, rexp[sp * M + i]);
    float H = 0.0f, Lo = 0.0f;
    if (R != kEmptyRange) {
      for (int sp = 0; sp < splits; ++sp) {
        const int e = rexp[sp * M + i];
        if (e == kEmptyRange) continue;
        const float scale = pow2f(e - R);
        const float2 p = partial[(sp * M + i) * BNt + c];
        df_add(H, Lo, __fmul_rn(p.x, scale));
        Lo = __fadd_rn(Lo, __fmul_rn(p.y, scale));
      }
    }
    C[idx] = R == kEmptyRange ? 0.0
                              : scalbn(static_cast<double>(H) + static_cast<double>(Lo), R);
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

size_t oz_slot_bytes(int BN) { return static_cast<size_t>(kDigitTileA) + static_cast<size_t>(BN) * 128; }

// Digit slots of the ring: as many as fit 227 KB (beyond S, the next window's first digits load
// a window ahead), at least S.
int oz_slots(int S, int BN) {
  const size_t room = (kMaxNodeSmemBytes - 256 - 1024) / oz_slot_bytes(BN);
  return std::max(S, std::min(kMaxSlots, static_cast<int>(room)));
}

size_t oz_smem_bytes(int S, int BN) {                   // tiles, barriers, alignment
  return static_cast<size_t>(oz_slots(S, BN)) * oz_slot_bytes(BN) + 256 + 1024;
}

template <int S>
cudaError_t launch_products(const double* A, int64_t lda, int64_t N, const double* Om,
                            const double* Ps, int s, double* Y, double* Z, bool shared,
                            cudaStream_t st) {
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
  const size_t off_ey = off_zd + (shared ? 0 : align1k(a_planes)), off_ez = off_ey + align1k(etab);
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
  // a new run: clear the abort flag an earlier run may have left (the report bits stay)
  e = cudaMemsetAsync(status + kAbortWord, 0, sizeof(int), st);
  if (e != cudaSuccess) return e;

  if (shared)
    oz_split_shared<S><<<dim3(W, W), 256, 0, st>>>(A, lda, N, Yd, ldd, EY, EZ, W, status);
  else
    oz_split_a<S><<<dim3(W, W), 256, 0, st>>>(A, lda, N, Yd, Zd, ldd, EY, EZ, W, status);
  oz_split_b<S><<<W, 256, 0, st>>>(Om, N, s, BNt, ldd, Bo, EO, status);
  oz_split_b<S><<<W, 256, 0, st>>>(Ps, N, s, BNt, ldd, Bp, EP, status);
  e = cudaGetLastError();
  if (e != cudaSuccess) return e;

  CUtensorMap mAy, mAz, mBo, mBp;
  const uint64_t row_bytes = static_cast<uint64_t>(ldd) * 2;
  if (!make_map(&mAy, CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, Yd, N, S * N, row_bytes, OBK, OBM,
                CU_TENSOR_MAP_SWIZZLE_128B, CU_TENSOR_MAP_L2_PROMOTION_L2_128B) ||
      !(shared ? make_map(&mAz, CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, Yd, N, S * N, row_bytes, 64,
                          OBK, CU_TENSOR_MAP_SWIZZLE_128B, CU_TENSOR_MAP_L2_PROMOTION_L2_128B)
               : make_map(&mAz, CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, Zd, N, S * N, row_bytes, OBK,
                          OBM, CU_TENSOR_MAP_SWIZZLE_128B, CU_TENSOR_MAP_L2_PROMOTION_L2_128B)) ||
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
  const int slots = oz_slots(S, BN);
  OzArgs ay{static_cast<int>(N), W, BN, BNt, wchunk, slots, EY, EO, partial, rexp, status};
  kernel<<<grid, kOzThreads, smem, st>>>(mAy, mBo, ay);
  oz_reduce<<<rg, 256, 0, st>>>(partial, rexp, splits, N, BNt, s, Y);
  e = cudaGetLastError();
  if (e != cudaSuccess) return e;
  OzArgs az{static_cast<int>(N), W, BN, BNt, wchunk, slots, EZ, EP, partial, rexp, status};
  if (shared) {
    auto kernel_mn = oz_gemm<S, true>;
    e = cudaFuncSetAttribute(kernel_mn, cudaFuncAttributeMaxDynamicSharedMemorySize,
                             static_cast<int>(smem));
    if (e != cudaSuccess) return e;
    kernel_mn<<<grid, kOzThreads, smem, st>>>(mAz, mBp, az);
  } else {
    kernel<<<grid, kOzThreads, smem, st>>>(mAz, mBp, az);
  }
  oz_reduce<<<rg, 256, 0, st>>>(partial, rexp, splits, N, BNt, s, Z);
  return cudaGetLastError();
}

}  // namespace

cudaError_t launch_sample_dense_oz(const double* A, int64_t lda, int64_t N, const double* Om,
                                   const double* Ps, int s, double* Y, double* Z, int digits,
                                   bool shared_planes, cudaStream_t st) {
  if (s < 1 || s > 256 || N < 1 || N > (int64_t(1) << 20) || lda < N)
    return cudaErrorInvalidValue;
  int BN, BNt;
  column_tiles(s, &BN, &BNt);
  if (oz_smem_bytes(digits, BN) > kMaxNodeSmemBytes) return cudaErrorInvalidValue;
  switch (digits) {
    case 5: return launch_products<5>(A, lda, N, Om, Ps, s, Y, Z, shared_planes, st);
    case 7: return launch_products<7>(A, lda, N, Om, Ps, s, Y, Z, shared_planes, st);
    default: return cudaErrorInvalidValue;
  }
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
  if (e == cudaSuccess && clear) e = cudaMemset(status, 0, kStatusWords * sizeof(int));
  return e;
}

cudaError_t sample_oz_inject(int bits) {
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return e;
  int* status = nullptr;
  {
    std::lock_guard<std::mutex> lock(g_oz_mutex);
    if (dev < static_cast<int>(g_oz_scratch.size())) status = static_cast<int*>(g_oz_scratch[dev].ptr);
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

}  // namespace hbs
