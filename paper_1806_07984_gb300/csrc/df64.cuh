// Double-float ("df64") arithmetic: a value is the unevaluated sum hi + lo of
// two FP32 numbers with |lo| <= ulp(hi) / 2, about 48 significant bits.
// Built from error-free transformations: TwoSum (Knuth, TAOCP vol. 2),
// TwoProduct by fused multiply-add, and the double-double add / multiply /
// divide of Hida, Li and Bailey ("Algorithms for quad-double precision
// floating point arithmetic", ARITH 2001), specialised to pairs of floats.
//
// On GB300 the FP32 pipes issue about 62 times as many operations as the FP64
// pipe, so a ~15-operation double-float multiply-add is still several times
// faster than one FP64 FMA.
#pragma once
#include <cuda_runtime.h>

namespace ader {
// The type and its functions live in their own namespace so that they are
// found only by argument-dependent lookup and never hide the FP64/FP32 math
// functions (fma, isfinite) for built-in types.
namespace dfp {

struct df64 {
  float hi, lo;
  df64() = default;
  __host__ __device__ constexpr df64(float h, float l) : hi(h), lo(l) {}
  __device__ __forceinline__ df64(double x) {
    hi = __double2float_rn(x);
    lo = __double2float_rn(x - double(hi));
  }
  __device__ __forceinline__ df64(int x) : df64(double(x)) {}
  __device__ __forceinline__ explicit operator double() const { return double(hi) + double(lo); }
};

// s + e = a + b exactly (Knuth's TwoSum)
__device__ __forceinline__ df64 df_two_sum(float a, float b) {
  const float s = a + b;
  const float bb = s - a;
  const float e = (a - (s - bb)) + (b - bb);
  return df64(s, e);
}

// s + e = a + b exactly when |a| >= |b| (Dekker's FastTwoSum)
__device__ __forceinline__ df64 df_quick_two_sum(float a, float b) {
  const float s = a + b;
  const float e = b - (s - a);
  return df64(s, e);
}

__device__ __forceinline__ df64 operator-(df64 a) { return df64(-a.hi, -a.lo); }

// accurate sum (both parts carried through TwoSum)
__device__ __forceinline__ df64 operator+(df64 a, df64 b) {
  df64 s = df_two_sum(a.hi, b.hi);
  const df64 t = df_two_sum(a.lo, b.lo);
  s = df_quick_two_sum(s.hi, s.lo + t.hi);
  return df_quick_two_sum(s.hi, s.lo + t.lo);
}

__device__ __forceinline__ df64 operator-(df64 a, df64 b) { return a + (-b); }

// product: TwoProduct of the high parts plus the cross terms
__device__ __forceinline__ df64 operator*(df64 a, df64 b) {
  const float p = a.hi * b.hi;
  float e = fmaf(a.hi, b.hi, -p);
  e = fmaf(a.hi, b.lo, e);
  e = fmaf(a.lo, b.hi, e);
  return df_quick_two_sum(p, e);
}

// a * b + c
__device__ __forceinline__ df64 fma(df64 a, df64 b, df64 c) {
  const float p = a.hi * b.hi;
  float e = fmaf(a.hi, b.hi, -p);
  e = fmaf(a.hi, b.lo, e);
  e = fmaf(a.lo, b.hi, e);
  const df64 s = df_two_sum(p, c.hi);
  return df_quick_two_sum(s.hi, s.lo + (e + c.lo));
}

// Accumulating a * b + c without renormalising: the rounding error of the
// high-part sum (TwoSum) and of the product (TwoProduct and the cross terms)
// are added to the low part, which may grow to a few units in the last place
// of the high part; `settle` restores the canonical pair.  This is the
// compensated dot product of Ogita, Rump and Oishi ("Accurate sum and dot
// product", SIAM J. Sci. Comput. 26, 2005) applied to double-float operands:
// 12 FP32 operations per term instead of 15.
__device__ __forceinline__ df64 fma_acc(df64 a, df64 b, df64 c) {
  const float p = a.hi * b.hi;
  float e = fmaf(a.hi, b.hi, -p);
  e = fmaf(a.hi, b.lo, e);
  e = fmaf(a.lo, b.hi, e);
  const df64 s = df_two_sum(c.hi, p);
  return df64(s.hi, c.lo + (s.lo + e));
}

__device__ __forceinline__ df64 settle(df64 a) { return df_two_sum(a.hi, a.lo); }

// quotient: FP32 estimate, one correction with the df64 residual
__device__ __forceinline__ df64 operator/(df64 a, df64 b) {
  const float q1 = a.hi / b.hi;
  const df64 r = a - b * df64(q1, 0.0f);
  const float q2 = r.hi / b.hi;
  return df_quick_two_sum(q1, q2);
}

__device__ __forceinline__ bool isfinite(df64 a) { return ::isfinite(a.hi) && ::isfinite(a.lo); }

}  // namespace dfp
using dfp::df64;
}  // namespace ader
