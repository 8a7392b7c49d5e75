// Float-float ("double-float") arithmetic on the FP32 pipe.
//
// A value is the unevaluated sum hi + lo of two floats with |lo| <= ulp(hi)
// (normalised) or a few ulp (the accumulators below).  The building blocks are
// the error-free transformations of Knuth (TwoSum), Dekker (Fast2Sum) and the
// FMA-based exact product (TwoProd: a b - fl(a b) is one fma), combined as in
// Dekker (1971) and the double-double literature (Hida, Li & Bailey 2001;
// Joldes, Muller & Popescu 2017): the sum of two float-floats with one TwoSum
// on the high parts ("sloppy" addition) and the product with one TwoProd plus
// the two cross terms.  The relative error of each operation is a few times
// 2^-48, with the exponent range of FP32.  Every operation uses the explicit
// round-to-nearest intrinsics so that the compiler cannot contract or reorder
// the error terms.
//
// The type serves the flux, SAT and viscous kernels in the ES_FP64X precision
// mode: state, entropy sums and the relaxation solve stay in FP64.
#pragma once
#include <cuda_runtime.h>

namespace es {

// the FP32/FP64 math functions stay visible next to the float-float overloads below
using ::fabs;
using ::fmax;
using ::log;

struct __align__(8) ff {
  float hi, lo;
  ff() = default;
  __host__ __device__ constexpr ff(float h, float l) : hi(h), lo(l) {}
  // split of a double: hi = fl32(d), lo = fl32(d - hi) (exact difference in FP64)
  __host__ __device__ explicit ff(double d) : hi(float(d)), lo(float(d - double(float(d)))) {}
  __host__ __device__ explicit ff(int i) : hi(float(i)), lo(0.0f) {}
  __host__ __device__ explicit operator double() const { return double(hi) + double(lo); }
};

// s + e = a + b exactly (Knuth's TwoSum, 6 operations, no condition on a, b)
__device__ __forceinline__ ff two_sum(float a, float b) {
  const float s = __fadd_rn(a, b);
  const float bb = __fsub_rn(s, a);
  const float e = __fadd_rn(__fsub_rn(a, __fsub_rn(s, bb)), __fsub_rn(b, bb));
  return ff(s, e);
}

// s + e = a + b exactly when |a| >= |b| or a == 0 (Dekker's Fast2Sum, 3 operations)
__device__ __forceinline__ ff fast_two_sum(float a, float b) {
  const float s = __fadd_rn(a, b);
  const float e = __fsub_rn(b, __fsub_rn(s, a));
  return ff(s, e);
}

__device__ __forceinline__ ff ff_norm(ff x) { return fast_two_sum(x.hi, x.lo); }

__device__ __forceinline__ ff operator+(ff x, ff y) {
  const ff s = two_sum(x.hi, y.hi);
  return fast_two_sum(s.hi, __fadd_rn(s.lo, __fadd_rn(x.lo, y.lo)));
}
__device__ __forceinline__ ff operator-(ff x) { return ff(-x.hi, -x.lo); }
__device__ __forceinline__ ff operator-(ff x, ff y) { return x + (-y); }

__device__ __forceinline__ ff operator*(ff x, ff y) {
  const float p = __fmul_rn(x.hi, y.hi);
  float e = __fmaf_rn(x.hi, y.hi, -p);
  e = __fmaf_rn(x.hi, y.lo, e);
  e = __fmaf_rn(x.lo, y.hi, e);
  return fast_two_sum(p, e);
}

__device__ __forceinline__ ff& operator+=(ff& x, ff y) { return x = x + y; }
__device__ __forceinline__ ff& operator-=(ff& x, ff y) { return x = x - y; }
__device__ __forceinline__ ff& operator*=(ff& x, ff y) { return x = x * y; }

// comparisons on the value (hi decides unless equal)
__device__ __forceinline__ bool operator<(ff x, ff y) { return x.hi < y.hi || (x.hi == y.hi && x.lo < y.lo); }
__device__ __forceinline__ bool operator>(ff x, ff y) { return y < x; }

__device__ __forceinline__ ff fabs(ff x) { return x.hi < 0.0f ? -x : x; }
__device__ __forceinline__ ff fmax(ff x, ff y) { return x < y ? y : x; }

// acc += a b with the product's rounding error kept (TwoProd) and the sum's error
// carried in acc.lo (TwoSum on the high parts, no renormalisation: acc.lo grows by
// at most an ulp of acc.hi per call and is absorbed by the next normalising use).
__device__ __forceinline__ void ff_fma_acc(ff& acc, ff a, ff b) {
  const float p = __fmul_rn(a.hi, b.hi);
  float e = __fmaf_rn(a.hi, b.hi, -p);
  e = __fmaf_rn(a.hi, b.lo, e);
  e = __fmaf_rn(a.lo, b.hi, e);
  const ff s = two_sum(acc.hi, p);
  acc.hi = s.hi;
  acc.lo = __fadd_rn(acc.lo, __fadd_rn(s.lo, e));
}

// 1/x: the FP32 hardware approximation r (rcp.approx.ftz.f32, about one ulp)
// refined with the residual t = 1 - x r (two fmas, the second with x.lo) by the
// second-order step r (1 + t + t^2): the truncation r t^3 is far below 2^-48 and
// the result carries the rounding of t and of the correction, ~2^-46 relative.
__device__ __forceinline__ ff ff_rcp(ff x) {
  float r;
  asm("rcp.approx.ftz.f32 %0, %1;" : "=f"(r) : "f"(x.hi));
  float t = __fmaf_rn(-x.hi, r, 1.0f);
  t = __fmaf_rn(-x.lo, r, t);
  // second-order term keeps the result at float-float precision: r (1 + t + t^2)
  const float c = __fmul_rn(r, __fmaf_rn(t, t, t));
  return fast_two_sum(r, c);
}

// logarithm through FP64 (used only off the hot path: entropy variables for the
// entropy-rate output and the log-mean's rare branch)
__device__ __forceinline__ ff log(ff x) { return ff(::log(double(x))); }

}  // namespace es
