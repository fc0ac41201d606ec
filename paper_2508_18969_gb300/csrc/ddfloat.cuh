// Double-float arithmetic: a value is the unevaluated sum hi + lo of two FP32 numbers
// (about 48 significant bits). Built from the error-free transformations of Knuth (TwoSum,
// TAOCP vol. 2) and Dekker (1971; the product error through a fused multiply-add). It moves
// the O(n^2) mixing sums of the equation of state from the FP64 pipe -- 1/64 of the FP32 rate
// on this GPU -- to the FP32 pipes at ~1e-14 relative accuracy.
//
// All operations use the _rn intrinsics so the compiler cannot contract or reorder them
// (a contracted a*b+c inside TwoSum would break the error bookkeeping).
#pragma once

#include <cuda_runtime.h>

namespace dfgb {

struct f2 {
  float h, l;
};

__device__ __forceinline__ f2 f2_make(float h, float l) { return f2{h, l}; }

// Conversions between FP64 and FP32 done with integer operations: on this GPU the
// F2F conversions run on the FP64 pipe, which is the scarce one. Values outside the ranges
// handled by the bit manipulation (very small or very large magnitudes, inf, NaN) take the
// ordinary conversion instructions.

// Exact FP32 -> FP64 (zeros included; subnormals, inf and NaN take the conversion instruction).
__device__ __forceinline__ double f_to_d(float f) {
  const unsigned u = __float_as_uint(f);
  const unsigned e = (u >> 23) & 0xFFu;
  if ((u & 0x7FFFFFFFu) == 0u) return __hiloint2double((int)(u & 0x80000000u), 0);
  if (e == 0u || e == 255u) return (double)f;
  const unsigned hi = (u & 0x80000000u) | ((e + 896u) << 20) | ((u & 0x7FFFFFu) >> 3);
  return __hiloint2double((int)hi, (int)(u << 29));
}

// Classification of FP64 values on their bits (integer pipes).
__device__ __forceinline__ bool d_finite(double x) {
  return ((__double2hiint(x) >> 20) & 0x7FF) != 0x7FF;
}
// x > 0 (false for zeros, negative values and NaN with the sign set).
__device__ __forceinline__ bool d_pos(double x) { return __double_as_longlong(x) > 0; }
// x >= c for a positive finite threshold c (false for negative x and NaN with the sign set;
// a positive NaN compares true, so test d_finite as well).
__device__ __forceinline__ bool d_ge_pos(double x, double c) {
  return __double_as_longlong(x) >= __double_as_longlong(c);
}

// FP64 -> FP32 by truncation of the significand (relative error < 2^-23); used for seeds and
// for inputs whose FP32 rounding error is irrelevant.
__device__ __forceinline__ float d_to_f_trunc(double x) {
  const unsigned hi32 = (unsigned)__double2hiint(x);
  const int e = (int)((hi32 >> 20) & 0x7FFu);
  if (e < 897 || e > 1150) return __double2float_rn(x);
  const unsigned lo32 = (unsigned)__double2loint(x);
  return __uint_as_float((hi32 & 0x80000000u) | ((unsigned)(e - 896) << 23) |
                         ((hi32 & 0xFFFFFu) << 3) | (lo32 >> 29));
}

// Split of an FP64 number into hi + lo: hi is x with its significand cut to 24 bits (exact),
// lo the remaining 29 bits rounded to 24 (x == hi + lo to ~2^-53 relative).
__device__ __forceinline__ f2 f2_from(double x) {
  const unsigned hi32 = (unsigned)__double2hiint(x);
  const unsigned lo32 = (unsigned)__double2loint(x);
  const int e = (int)((hi32 >> 20) & 0x7FFu);
  if (e >= 897 && e <= 1100) {
    const unsigned sign = hi32 & 0x80000000u;
    const unsigned hb = sign | ((unsigned)(e - 896) << 23) | ((hi32 & 0xFFFFFu) << 3) | (lo32 >> 29);
    // remainder r * 2^(e - 1075), formed as r * 2^-64 * 2^(e - 1011) to stay in range
    float l = __fmul_rn(__fmul_rn(__uint2float_rn(lo32 & 0x1FFFFFFFu), 5.421010862427522e-20f),
                        __int_as_float((e - 884) << 23));
    l = __uint_as_float(__float_as_uint(l) | sign);
    return f2{__uint_as_float(hb), l};
  }
  if (((hi32 & 0x7FFFFFFFu) | lo32) == 0u) return f2{__uint_as_float(hi32 & 0x80000000u), 0.0f};
  const float h = __double2float_rn(x);
  return f2{h, __double2float_rn(x - (double)h)};
}

__device__ __forceinline__ double f2_to(f2 a) { return f_to_d(a.h) + f_to_d(a.l); }

// f2 -> FP64 with integer operations only, for a normalised pair (|lo| <= ulp(hi) / 2, as
// f2_norm leaves it): the exact sum of the two significands is formed in a 64-bit integer
// and cut to 53 bits (truncation: relative error below 2^-52). Other pairs (zeros, subnormal,
// inf, NaN, or a low part out of range) take f2_to.
__device__ __forceinline__ double f2_to_int(f2 a) {
  const unsigned uh = __float_as_uint(a.h), ul = __float_as_uint(a.l);
  const int eh = (int)((uh >> 23) & 0xFFu), el = (int)((ul >> 23) & 0xFFu);
  if ((ul & 0x7FFFFFFFu) == 0u) return f_to_d(a.h);
  const int sh = 39 + el - eh;                 // scale of lo's significand against hi's << 39
  if (eh == 0 || eh == 255 || el == 0 || el == 255 || sh > 15) return f2_to(a);
  const unsigned long long mh = (unsigned long long)((uh & 0x7FFFFFu) | 0x800000u);
  const unsigned long long ml = (unsigned long long)((ul & 0x7FFFFFu) | 0x800000u);
  const unsigned long long tl = sh >= 0 ? (ml << sh) : (sh > -40 ? (ml >> -sh) : 0ull);
  unsigned long long S = mh << 39;
  S = (((uh ^ ul) & 0x80000000u) == 0u) ? S + tl : S - tl;   // S in [2^61, 2^64)
  const int pos = 63 - __clzll((long long)S);                 // leading bit, 61..63
  const unsigned long long mant = (S >> (pos - 52)) & ((1ull << 52) - 1ull);
  const unsigned e = (unsigned)(eh - 127 + pos - 62 + 1023);
  return __hiloint2double((int)((uh & 0x80000000u) | (e << 20) | (unsigned)(mant >> 32)),
                          (int)(unsigned)mant);
}

// TwoSum (Knuth): s + e == a + b exactly.
__device__ __forceinline__ void two_sum(float a, float b, float& s, float& e) {
  s = __fadd_rn(a, b);
  const float bb = __fsub_rn(s, a);
  e = __fadd_rn(__fsub_rn(a, __fsub_rn(s, bb)), __fsub_rn(b, bb));
}

// FastTwoSum (Dekker), valid for |a| >= |b|.
__device__ __forceinline__ f2 f2_norm(float a, float b) {
  const float s = __fadd_rn(a, b);
  return f2{s, __fsub_rn(b, __fsub_rn(s, a))};
}

__device__ __forceinline__ f2 f2_add(f2 a, f2 b) {
  float s, e;
  two_sum(a.h, b.h, s, e);
  e = __fadd_rn(e, __fadd_rn(a.l, b.l));
  return f2_norm(s, e);
}

// Product hi part and its error: a*b == p + e (Dekker, via fma), lo parts to first order.
__device__ __forceinline__ void f2_prod(f2 a, f2 b, float& p, float& e) {
  p = __fmul_rn(a.h, b.h);
  e = __fmaf_rn(a.h, b.h, -p);
  e = __fmaf_rn(a.h, b.l, e);
  e = __fmaf_rn(a.l, b.h, e);
}

__device__ __forceinline__ f2 f2_mul(f2 a, f2 b) {
  float p, e;
  f2_prod(a, b, p, e);
  return f2_norm(p, e);
}

__device__ __forceinline__ f2 f2_scale2(f2 a) { return f2{2.0f * a.h, 2.0f * a.l}; }

// a * b for an FP32 b.
__device__ __forceinline__ f2 f2_mulf(f2 a, float b) {
  const float p = __fmul_rn(a.h, b);
  float e = __fmaf_rn(a.h, b, -p);
  e = __fmaf_rn(a.l, b, e);
  return f2_norm(p, e);
}

// 1 / a: FP32 reciprocal of the high part and one Newton step in double-float,
// r = r0 + r0 (1 - a r0) (relative error ~2^-46 for a normal a).
__device__ __forceinline__ f2 f2_rcp(f2 a) {
  const float r0 = __frcp_rn(a.h);
  float p, e;
  f2_prod(a, f2{r0, 0.0f}, p, e);          // a r0 = p + e, close to 1
  const float res = __fadd_rn(__fsub_rn(1.0f, p), -e);  // 1 - a r0, exact to ~2^-48
  return f2_norm(r0, __fmul_rn(r0, res));
}

// Accumulator with a lazily kept low part: s += p + e.
__device__ __forceinline__ void acc_add(f2& s, float p, float e) {
  float t, err;
  two_sum(s.h, p, t, err);
  s.h = t;
  s.l = __fadd_rn(s.l, __fadd_rn(e, err));
}

__device__ __forceinline__ void acc_add(f2& s, f2 a) { acc_add(s, a.h, a.l); }

// s += a * b
__device__ __forceinline__ void acc_fma(f2& s, f2 a, f2 b) {
  float p, e;
  f2_prod(a, b, p, e);
  acc_add(s, p, e);
}

__device__ __forceinline__ f2 f2_fin(f2 s) { return f2_norm(s.h, s.l); }

// Double-float constant from an FP64 value (hi = fl32(x), lo = fl32(x - hi)).
__host__ __device__ constexpr f2 f2_const(double x) {
  return f2{(float)x, (float)(x - (double)(float)x)};
}

__device__ __forceinline__ f2 f2_neg(f2 a) { return f2{-a.h, -a.l}; }
__device__ __forceinline__ f2 f2_sub(f2 a, f2 b) { return f2_add(a, f2_neg(b)); }
__device__ __forceinline__ f2 f2_addf(f2 a, float b) {
  float s, e;
  two_sum(a.h, b, s, e);
  return f2_norm(s, __fadd_rn(e, a.l));
}

// a * b + c in one pass: the product's error term and both low parts join the TwoSum error.
__device__ __forceinline__ f2 f2_fma(f2 a, f2 b, f2 c) {
  float p, e, s, t;
  f2_prod(a, b, p, e);
  two_sum(p, c.h, s, t);
  return f2_norm(s, __fadd_rn(t, __fadd_rn(e, c.l)));
}

// a > b by the sign of the double-float difference. Comparing high parts first would need
// both pairs in one canonical form, and f2_from's high part is truncated (its low part can
// reach a whole ulp) while arithmetic results are rounded to nearest.
__device__ __forceinline__ bool f2_gt(f2 a, f2 b) {
  float s, e;
  two_sum(a.h, -b.h, s, e);
  e = __fadd_rn(e, __fsub_rn(a.l, b.l));
  return __fadd_rn(s, e) > 0.0f;   // rounding keeps the sign of a nonzero s + e
}
__device__ __forceinline__ bool f2_lt(f2 a, f2 b) { return f2_gt(b, a); }

// sqrt(a) for a positive normal a: t0 = a.h r with r = rsqrt_32(a.h), then one Newton step
// t = t0 + (a - t0^2) r / 2, the residual formed exactly (t0^2 by a product error, a.h - t0^2
// by Sterbenz) and rounded once (relative error ~2^-46).
__device__ __forceinline__ f2 f2_sqrt_pos(f2 a) {
  const float r = rsqrtf(a.h);
  const float t0 = __fmul_rn(a.h, r);
  const float p = __fmul_rn(t0, t0);
  const float pe = __fmaf_rn(t0, t0, -p);
  const float res = __fadd_rn(__fsub_rn(a.h, p), __fsub_rn(a.l, pe));
  return f2_norm(t0, __fmul_rn(res, __fmul_rn(0.5f, r)));
}

// s += a * b into an accumulator offset by a power of two sigma: h starts at sigma, and every
// partial sum and every product are bounded by B <= sigma (terms of one sign: h stays in
// [sigma, 2 sigma]) or by B <= sigma / 4 (terms of both signs: h stays within sigma / 4 of
// sigma). Then s = fl(a.h b.h + h) and h lie within a factor of two of each other, so h - s
// is exact (Sterbenz) and fma(a.h, b.h, h - s) is the rounding error of the first FMA, itself
// rounded once (below ulp(sigma) 2^-25). l collects it with the cross terms a.h b.l + a.l b.h;
// the sum is (h - sigma) + l, where h - sigma is exact too. Six FP32 operations per term
// against twelve for a product error plus TwoSum.
__device__ __forceinline__ void acc_off_fma(float& h, float& l, f2 a, f2 b) {
  const float s = __fmaf_rn(a.h, b.h, h);
  const float r = __fmaf_rn(a.h, b.h, __fsub_rn(h, s));
  l = __fadd_rn(l, r);
  l = __fmaf_rn(a.h, b.l, l);
  l = __fmaf_rn(a.l, b.h, l);
  h = s;
}

// Moves the part of l on h's grid into h (both steps exact: t - h by Sterbenz, the remainder
// because it is l less its rounding onto that grid), so that l stays small and its own FP32
// rounding stays far below ulp(h). The value (h - sigma) + l is unchanged.
__device__ __forceinline__ void acc_renorm(float& h, float& l) {
  const float t = __fadd_rn(h, l);
  l = __fsub_rn(l, __fsub_rn(t, h));
  h = t;
}

// Smallest power of two >= x for a finite x >= 0 (the smallest normal for subnormal x).
__device__ __forceinline__ float pow2_up(float x) {
  return __uint_as_float((__float_as_uint(x) + 0x007FFFFFu) & 0xFF800000u);
}

}  // namespace dfgb
