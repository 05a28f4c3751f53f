// Arithmetic on unevaluated sums of two floats ("float pairs": the value h + l with
// |l| <= ulp(h) / 2), run on the FP32 and integer pipes.
//
// On GB300 an FP64 warp instruction occupies the FP64 pipe for 16 cycles, so an
// FP64 multiply-add per matrix entry or per pair bounds a sweep well below the HBM
// roofline.  A float pair carries 48 significand bits: a double rounded to a pair
// (hi = RN(x), lo = RN(x - hi)) is within 2^-48 |x|, and products and sums of pairs
// built from the error-free transformations below keep errors of that order
// relative to the magnitudes involved, on a pipe 64 times faster (down to 2^-126 in
// magnitude; below, the floats' subnormal spacing 2^-149 bounds the absolute error).
//
// Error-free transformations, restated from their published definitions:
//  * two_sum: Knuth's TwoSum (The Art of Computer Programming, vol. 2, 4.2.2):
//    s + e = a + b exactly, for any a, b;
//  * fast_two_sum: Dekker's Fast2Sum (1971): the same when |a| >= |b| (or a = 0);
//  * two_prod: Dekker's TwoProduct in its FMA form: p + e = a b exactly.
// The _rn intrinsics keep the compiler from contracting or reordering them.
#pragma once

#include "afc_internal.h"

namespace afc {

__device__ __forceinline__ void two_sum(float a, float b, float& s, float& e) {
  s = __fadd_rn(a, b);
  const float bb = __fsub_rn(s, a);
  e = __fadd_rn(__fsub_rn(a, __fsub_rn(s, bb)), __fsub_rn(b, bb));
}

__device__ __forceinline__ void fast_two_sum(float a, float b, float& s, float& e) {
  s = __fadd_rn(a, b);
  e = __fsub_rn(b, __fsub_rn(s, a));
}

__device__ __forceinline__ void two_prod(float a, float b, float& p, float& e) {
  p = __fmul_rn(a, b);
  e = __fmaf_rn(a, b, -p);
}

// Lexicographic order of normalised pairs, which is the order of their values
// (for h1 > h2, h1 + l1 >= h2 + l2 since |l| <= ulp(h) / 2).
__device__ __forceinline__ bool pair_gt(float ah, float al, float bh, float bl) {
  return ah > bh || (ah == bh && al > bl);
}

// (sh, sl) = a - b, normalised.
__device__ __forceinline__ void pair_sub(float ah, float al, float bh, float bl, float& sh, float& sl) {
  float s, e;
  two_sum(ah, -bh, s, e);
  e = __fadd_rn(e, __fsub_rn(al, bl));
  two_sum(s, e, sh, sl);
}

// (ph, pl) = a * b (unnormalised: |pl| <= ~2^-23 |ph|): the exact product of the
// high parts plus the cross terms; the product of the low parts (2^-48 relative) is
// dropped.
__device__ __forceinline__ void pair_mul(float ah, float al, float bh, float bl, float& ph, float& pl) {
  float e;
  two_prod(ah, bh, ph, e);
  pl = __fmaf_rn(ah, bl, __fmaf_rn(al, bh, e));
}

// Doubles of magnitude 2^127 or more, Inf and NaN, beyond the range of float pairs:
// kept out of line so that its FP64 instructions issue only for the warps that need
// them.
static __device__ __noinline__ float2 split_pair_fp64(double x) {
  const float h = __double2float_rn(x);
  return make_float2(h, __double2float_rn(x - (double)h));
}

// hi = RN(x), lo = RN(x - hi) (round to nearest, ties to even) on the integer pipe, for
// |x| < 2^127.  With e the biased exponent of x, the low 29 bits of its
// significand are what the float drops; rounding adds one unit to the kept bits (a
// carry may move into the exponent), and x - hi = r * 2^(e - 1075) with r = dropped
// bits - carry * 2^29, an integer of at most 29 bits.  Where that value is a normal
// float or a multiple of 2^-149 (e >= 926), it is rounded once, by the conversion of r
// to float, and scaled exactly (by 2^(e - 1075), or by 2^-100 * 2^(e - 975) so that
// every factor is a normal float).  Otherwise it is subnormal and not a multiple of
// 2^-149: r is shifted to units of 2^-149 and rounded in integers, as is x itself when
// |x| < 2^-126.  |x| >= 2^127 (and Inf, NaN) take split_pair_fp64.
__device__ __forceinline__ float2 split_pair(double x) {
  const unsigned long long b = (unsigned long long)__double_as_longlong(x);
  const unsigned sign = (unsigned)(b >> 32) & 0x80000000u;
  const unsigned e = (unsigned)(b >> 52) & 0x7ffu;
  if (e < 897u) {   // |x| < 2^-126: hi is subnormal (or 0) and lo = 0, as |x - hi| <= 2^-150
    unsigned q = 0;   // RN(|x| / 2^-149), 0 for |x| < 2^-151
    if (e >= 872u) {
      const unsigned sh = 926u - e;   // 30 .. 54
      const unsigned long long sig = (b & 0xfffffffffffffull) | (1ull << 52);
      const unsigned long long rb = sig & ((1ull << sh) - 1ull), half = 1ull << (sh - 1u);
      q = (unsigned)(sig >> sh);
      q += (rb > half) | ((rb == half) & (q & 1u));
    }
    return make_float2(__uint_as_float(sign | q), 0.f);
  }
  if (e > 1149u) return split_pair_fp64(x);
  const unsigned rem = (unsigned)b & 0x1fffffffu;
  unsigned t = (unsigned)(((b >> 29) & 0x3ffffffffull) - (896ull << 23));
  const unsigned up = (rem > 0x10000000u) | ((rem == 0x10000000u) & (t & 1u));
  t += up;
  const int r = (int)rem - (int)(up << 29);
  const unsigned m = r < 0 ? (unsigned)(-r) : (unsigned)r;
  bool normal = e >= 926u;   // lo = r * 2^(e - 1075) is a multiple of 2^-149, or normal
  unsigned sh = 0;
  if (!normal) {
    sh = 926u - e;                      // 1 .. 29: |lo| = m * 2^-sh units of 2^-149
    normal = (m >> sh) >= 0x800000u;    // |lo| >= 2^-126
  }
  unsigned lb;
  if (normal) {
    const bool low = e < 949u;
    const float s1 = low ? 7.888609052210118e-31f : 1.f;                  // 2^-100
    const float s2 = __uint_as_float((low ? e - 848u : e - 948u) << 23);  // 2^(e - 975) or 2^(e - 1075)
    lb = __float_as_uint(__fmul_rn(__fmul_rn(__int2float_rn(r), s1), s2));
  } else {
    unsigned q = m >> sh;
    const unsigned rb = m & ((1u << sh) - 1u), half = 1u << (sh - 1u);
    q += (rb > half) | ((rb == half) & (q & 1u));
    lb = q | (r < 0 ? 0x80000000u : 0u);   // the bit pattern of q * 2^-149 (q <= 2^23)
  }
  return make_float2(__uint_as_float(sign | t), __uint_as_float(lb ^ sign));
}

}  // namespace afc
