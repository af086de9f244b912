// Double-float arithmetic for the compensated node products of the mixed precision: a value is
// an unevaluated sum hi + lo of two FP32 words with |lo| <= ulp(hi) / 2, about 48 significant
// bits in FP32's exponent range. Sums use Knuth's TwoSum and Dekker's Fast2Sum, products the
// exact FMA residual of hi * hi (Dekker 1971; Joldes, Muller and Popescu, ACM TOMS 2017, the
// "sloppy" variants). Every operation runs on the FP32 pipe, which GB300 drives at 64 times the
// FP64 rate; all roundings are explicit (__fadd_rn etc.), so the compiler can neither contract
// nor reorder them.
#pragma once

#include <cuda_runtime.h>

namespace hbs {

struct dfloat {
  float hi, lo;
};

__device__ __forceinline__ dfloat df_two_sum(float a, float b) {
  const float s = __fadd_rn(a, b);
  const float bb = __fsub_rn(s, a);
  const float e = __fadd_rn(__fsub_rn(a, __fsub_rn(s, bb)), __fsub_rn(b, bb));
  return {s, e};
}

__device__ __forceinline__ dfloat df_fast_two_sum(float a, float b) {   // needs |a| >= |b|
  const float s = __fadd_rn(a, b);
  return {s, __fsub_rn(b, __fsub_rn(s, a))};
}

// An FP64 value as a double-float (to ~2^-48 relative; FP32 exponent range), by integer
// operations on its bits: hi is x truncated to 24 significant bits, lo the remaining 29 bits
// truncated to 24 (|lo| < ulp(hi); 48 of x's 53 bits are kept). On GB300 every FP64 instruction, a conversion included,
// runs at 1/64 of the FP32 rate, so the common case stays off the FP64 pipe; zeros and values
// whose hi or lo would leave FP32's normal range take the FP64 conversions.
__device__ __forceinline__ dfloat df_from(double x) {
  const unsigned long long u = static_cast<unsigned long long>(__double_as_longlong(x));
  const int e = static_cast<int>((u >> 52) & 0x7ff);            // biased exponent
  if (e >= 1075 - 126 && e <= 1023 + 127) {          // 2^(e - 1075) and hi both FP32-normal
    const unsigned sign = static_cast<unsigned>(u >> 32) & 0x80000000u;
    const unsigned mhi = static_cast<unsigned>((u >> 29) & 0x7fffffu);
    const float hi = __int_as_float(static_cast<int>(sign | (static_cast<unsigned>(e - 1023 + 127) << 23) | mhi));
    // lo = rem 2^(e - 1075) for the remaining 29 bits, truncated to 24 significant bits: the
    // leading one of rem at bit p gives the exponent, the 23 bits below it the fraction
    const unsigned rem = static_cast<unsigned>(u & 0x1fffffffu);
    unsigned lo_bits = 0;
    if (rem != 0u) {
      const int lz = __clz(static_cast<int>(rem));
      const unsigned frac = static_cast<unsigned>(
          ((static_cast<unsigned long long>(rem) << (lz + 1)) & 0xffffffffull) >> 9);
      lo_bits = sign | (static_cast<unsigned>(e + (31 - lz) - 948) << 23) | frac;
    }
    return {hi, __int_as_float(static_cast<int>(lo_bits))};
  }
  const float h = __double2float_rn(x);
  return {h, __double2float_rn(x - static_cast<double>(h))};
}

__device__ __forceinline__ double df_to(dfloat a) {
  return static_cast<double>(a.hi) + static_cast<double>(a.lo);
}

// a * b + c
__device__ __forceinline__ dfloat df_fma(dfloat a, dfloat b, dfloat c) {
  const float p = __fmul_rn(a.hi, b.hi);
  float e = __fmaf_rn(a.hi, b.hi, -p);                 // exact: a.hi b.hi = p + e
  e = __fmaf_rn(a.hi, b.lo, e);
  e = __fmaf_rn(a.lo, b.hi, e);
  const dfloat s = df_two_sum(c.hi, p);
  const float t = __fadd_rn(s.lo, __fadd_rn(c.lo, e));
  return df_fast_two_sum(s.hi, t);
}

// acc + a * b for a running sum that is not renormalised at every step: hi is updated by
// TwoSum (exactly), and its error and the product's low part are added to lo (12 FP32
// operations instead of 15). Over K steps |lo| grows to at most ~K ulp(hi), so its own roundings
// stay near 2^-48 K of the sum (the accumulated Dot2 of Ogita, Rump and Oishi, SISC 2005);
// df_norm renormalises once at the end.
__device__ __forceinline__ dfloat df_fma_acc(dfloat a, dfloat b, dfloat acc) {
  const float p = __fmul_rn(a.hi, b.hi);
  float e = __fmaf_rn(a.hi, b.hi, -p);
  e = __fmaf_rn(a.hi, b.lo, e);
  e = __fmaf_rn(a.lo, b.hi, e);
  const dfloat s = df_two_sum(acc.hi, p);
  return {s.hi, __fadd_rn(acc.lo, __fadd_rn(s.lo, e))};
}

__device__ __forceinline__ dfloat df_norm(dfloat a) { return df_fast_two_sum(a.hi, a.lo); }

__device__ __forceinline__ dfloat df_add(dfloat a, dfloat b) {
  const dfloat s = df_two_sum(a.hi, b.hi);
  const float t = __fadd_rn(s.lo, __fadd_rn(a.lo, b.lo));
  return df_fast_two_sum(s.hi, t);
}

__device__ __forceinline__ dfloat df_neg(dfloat a) { return {-a.hi, -a.lo}; }

__device__ __forceinline__ dfloat df_zero() { return {0.f, 0.f}; }

}  // namespace hbs
