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

// Exact split of an FP64 number into hi + lo (lo carries the next 24 bits).
__device__ __forceinline__ f2 f2_from(double x) {
  const float h = __double2float_rn(x);
  const float l = __double2float_rn(x - (double)h);
  return f2{h, l};
}

__device__ __forceinline__ double f2_to(f2 a) { return (double)a.h + (double)a.l; }

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

}  // namespace dfgb
