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

struct ff;
__device__ __forceinline__ ff ff_from_double(double d);
__device__ __forceinline__ double ff_to_double(float hi, float lo);

struct __align__(8) ff {
  float hi, lo;
  ff() = default;
  __host__ __device__ constexpr ff(float h, float l) : hi(h), lo(l) {}
  // split of a double (device: on the integer pipe, see ff_from_double;
  // host: hi = fl32(d), lo = fl32(d - hi))
  __host__ __device__ explicit ff(double d);
  __host__ __device__ explicit ff(int i) : hi(float(i)), lo(0.0f) {}
  __host__ __device__ explicit operator double() const;
};

// float -> double by placing the bits (exact; no FP64 instruction).  Zero keeps its
// sign; subnormal, infinite and NaN inputs take the conversion instruction.
__device__ __forceinline__ double f32_to_f64_bits(float f) {
  const unsigned u = __float_as_uint(f);
  const unsigned e = (u >> 23) & 0xFFu;
  if (e - 1u < 254u) {
    const unsigned hi32 = (u & 0x80000000u) | ((e + 896u) << 20) | ((u & 0x7FFFFFu) >> 3);
    return __hiloint2double(int(hi32), int(u << 29));
  }
  if ((u << 1) == 0u) return __hiloint2double(int(u & 0x80000000u), 0);
  return double(f);
}

// double -> float-float on the integer and FP32 pipes: hi = d with its significand
// truncated to 24 bits (exact in FP32), lo = the remaining 29 significand bits rounded
// to 24 (one FP32 rounding): |hi + lo - d| <= 2^-48 |d|.  The fast path covers
// 2^-74 <= |d| < 2^127 and zero; other magnitudes use the FP64 conversions.
__device__ __forceinline__ ff ff_from_double(double d) {
  const unsigned h = unsigned(__double_as_longlong(d) >> 32);
  const unsigned l = unsigned(__double_as_longlong(d));
  const unsigned e = (h >> 20) & 0x7FFu;
  const unsigned sign = h & 0x80000000u;
  if (e - 949u < 202u) {
    const float hi = __uint_as_float(sign | ((e - 896u) << 23) | ((h & 0xFFFFFu) << 3) | (l >> 29));
    // m29 = 2^6 a + b, a < 2^23, b < 2^6: both exact as floats (magic-number conversion),
    // one fma rounds 64 a + b to 24 bits, the power-of-two scale 2^(e - 1075) is exact
    const unsigned m29 = l & 0x1FFFFFFFu;
    const float a = __fsub_rn(__uint_as_float(0x4B000000u | (m29 >> 6)), 8388608.0f);
    const float b = __fsub_rn(__uint_as_float(0x4B000000u | (m29 & 63u)), 8388608.0f);
    const float m = __fmaf_rn(a, 64.0f, b);
    const float scale = __uint_as_float(sign | ((e - 948u) << 23));
    return ff(hi, __fmul_rn(m, scale));
  }
  if (((h << 1) | l) == 0u) return ff(__uint_as_float(sign), 0.0f);
  const float hi = __double2float_rn(d);
  return ff(hi, __double2float_rn(d - double(hi)));
}

// float-float -> double: both parts placed exactly, one FP64 addition rounds the sum
__device__ __forceinline__ double ff_to_double(float hi, float lo) {
  return f32_to_f64_bits(hi) + f32_to_f64_bits(lo);
}

__host__ __device__ inline ff::ff(double d) {
#ifdef __CUDA_ARCH__
  *this = ff_from_double(d);
#else
  hi = float(d);
  lo = float(d - double(hi));
#endif
}

__host__ __device__ inline ff::operator double() const {
#ifdef __CUDA_ARCH__
  return ff_to_double(hi, lo);
#else
  return double(hi) + double(lo);
#endif
}

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
