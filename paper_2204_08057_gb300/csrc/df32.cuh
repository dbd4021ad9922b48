// Double-float arithmetic on the FP32 pipe: a value is carried as the unevaluated sum h + l of
// two floats (about 48 significant bits).  On this GPU the FP64 unit runs at about 1/64 of the
// FP32 rate, so the true residual b - G X of the refinement loop, which needs more than FP32
// precision, is formed from FP32 operations only.
//
// Error-free transformations used (no FP64 operation anywhere):
// * TwoSum (Knuth, TAOCP vol. 2, 4.2.2): s = fl(a + b) and e with s + e = a + b exactly.
// * The FMA form of Dekker's product (Dekker 1971): p = fl(a b) and e = fma(a, b, -p) with
//   p + e = a b exactly.
// The intrinsics __fadd_rn / __fmul_rn keep the compiler from contracting these steps into
// FMAs, which would break the exactness.
// A sum of products is accumulated as Ogita, Rump and Oishi's Dot2 (SIAM J. Sci. Comput.
// 2005): the leading products are summed with TwoSum into S, every rounding error (and the
// second-order cross terms of the operands' low parts) into a plain float C; the result S + C
// is as accurate as a computation in twice the working precision, followed by a rounding.
//
// An FP64 input a is split by integer operations into h (its leading 24 significant bits,
// truncated) and l (the remaining 29 bits rounded to 24), |a - h - l| <= 2^-47 |a|.  The split
// is valid for a = 0 and for 2^-60 <= |a| < 2^61; the range keeps every product of two such
// values and its rounding error in the normal FP32 range (products of the operator entries,
// checked at set-up to lie in [2^-40, 2^40], with these stay above 2^-100).  Outside it the
// caller recomputes the pixel in FP64.
#pragma once

#include <cstdint>

namespace sylv {
namespace df {

__device__ __forceinline__ void two_sum(float a, float b, float& s, float& e) {
  s = __fadd_rn(a, b);
  const float bb = __fsub_rn(s, a);
  e = __fadd_rn(__fsub_rn(a, __fsub_rn(s, bb)), __fsub_rn(b, bb));
}

// s + e = a + b exactly, given |a| >= |b| (or a = 0).
__device__ __forceinline__ void fast_two_sum(float a, float b, float& s, float& e) {
  s = __fadd_rn(a, b);
  e = __fsub_rn(b, __fsub_rn(s, a));
}

__device__ __forceinline__ void two_prod(float a, float b, float& p, float& e) {
  p = __fmul_rn(a, b);
  e = __fmaf_rn(a, b, -p);
}

// Sum of products: value s + c.
struct Acc {
  float s, c;
};

__device__ __forceinline__ Acc zero() { return Acc{0.f, 0.f}; }

// acc += (ah + al)(bh + bl), the al bl term (below 2^-46 of the product) dropped.
__device__ __forceinline__ void fma(Acc& acc, float ah, float al, float bh, float bl) {
  float p, e, s, t;
  two_prod(ah, bh, p, e);
  e = __fmaf_rn(ah, bl, e);
  e = __fmaf_rn(al, bh, e);
  two_sum(acc.s, p, s, t);
  acc.s = s;
  acc.c = __fadd_rn(acc.c, __fadd_rn(t, e));
}

// The accumulated value as a normalised pair (h = fl(value) up to one rounding of c).
__device__ __forceinline__ void norm(const Acc& a, float& h, float& l) {
  fast_two_sum(a.s, a.c, h, l);
}

// r = (bh + bl) - value of g, normalised.
__device__ __forceinline__ void sub_from(float bh, float bl, const Acc& g, float& rh, float& rl) {
  float s, t;
  two_sum(bh, -g.s, s, t);
  const float c = __fsub_rn(__fadd_rn(t, bl), g.c);
  fast_two_sum(s, c, rh, rl);
}

// ---- the same on pairs of values, with the packed FP32 instructions of sm_100+
// (add/mul/fma.rn.f32x2): lane by lane the same error-free transformations, half the
// instructions.  a - b is formed as fma(b, -1, a): the product is exact, one rounding.
__device__ __forceinline__ float2 sub2(float2 a, float2 b) {
  return __ffma2_rn(b, make_float2(-1.f, -1.f), a);
}

__device__ __forceinline__ void two_sum2(float2 a, float2 b, float2& s, float2& e) {
  s = __fadd2_rn(a, b);
  const float2 bb = sub2(s, a);
  e = __fadd2_rn(sub2(a, sub2(s, bb)), sub2(b, bb));
}

__device__ __forceinline__ void fast_two_sum2(float2 a, float2 b, float2& s, float2& e) {
  s = __fadd2_rn(a, b);
  e = sub2(b, sub2(s, a));
}

struct Acc2 {
  float2 s, c;
};

__device__ __forceinline__ Acc2 zero2() {
  return Acc2{make_float2(0.f, 0.f), make_float2(0.f, 0.f)};
}

// acc += (ah + al)(bh + bl) lane by lane (lo lo dropped)
__device__ __forceinline__ void fma2(Acc2& acc, float2 ah, float2 al, float2 bh, float2 bl) {
  const float2 p = __fmul2_rn(ah, bh);
  float2 e = __ffma2_rn(ah, bh, make_float2(-p.x, -p.y));
  e = __ffma2_rn(ah, bl, e);
  e = __ffma2_rn(al, bh, e);
  float2 s, t;
  two_sum2(acc.s, p, s, t);
  acc.s = s;
  acc.c = __fadd2_rn(acc.c, __fadd2_rn(t, e));
}

__device__ __forceinline__ void norm2(const Acc2& a, float2& h, float2& l) {
  fast_two_sum2(a.s, a.c, h, l);
}

__device__ __forceinline__ void sub_from2(float2 bh, float2 bl, const Acc2& g, float2& rh,
                                          float2& rl) {
  float2 s, t;
  two_sum2(bh, make_float2(-g.s.x, -g.s.y), s, t);
  const float2 c = sub2(__fadd2_rn(t, bl), g.c);
  fast_two_sum2(s, c, rh, rl);
}

// Splits an FP64 value into h + l (see the header); returns false outside the valid range
// (h, l are then meaningless).
__device__ __forceinline__ bool split(double a, float& h, float& l) {
  const unsigned long long u = (unsigned long long)__double_as_longlong(a);
  const unsigned hi = (unsigned)(u >> 32), lo = (unsigned)u;
  const unsigned sgn = hi & 0x80000000u;
  const unsigned e = (hi >> 20) & 0x7FFu;                     // biased exponent (bias 1023)
  const unsigned frac23 = ((hi & 0xFFFFFu) << 3) | (lo >> 29);  // leading 23 fraction bits
  const unsigned rest = lo & 0x1FFFFFFFu;                     // the other 29
  // h: exponent rebiased to 127; l: rest * 2^(e - 1075) (the scale built from its exponent)
  h = __uint_as_float(sgn | ((e - 896u) << 23) | frac23);
  const float scale = __uint_as_float((e - 948u) << 23);
  l = __uint_as_float(__float_as_uint(__fmul_rn(__uint2float_rn(rest), scale)) | sgn);
  if ((u << 1) == 0ull) {   // +-0
    h = __uint_as_float(sgn);
    l = 0.f;
    return true;
  }
  return (e - 963u) <= 120u;   // 2^-60 <= |a| < 2^61
}

}  // namespace df
}  // namespace sylv
