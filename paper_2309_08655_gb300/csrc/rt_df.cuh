// Double-float scalar: FP64-class arithmetic on the FP32 pipe.
//
// A value is the unevaluated sum hi + lo of two floats with |lo| <= ulp(hi)/2
// (about 48 significant bits).  On this GPU an FP64 instruction, and every
// conversion between FP32 and FP64, issues at 1/64 of the FP32 rate, while a
// double-float product or sum costs 6-10 FP32 instructions: the integrator
// instantiated on this type (rt_trace_df.cu) does the FP64 integrator's
// arithmetic to a few units of 2^-47 at several times its rate.
//
// Built from the error-free transformations TwoSum (Knuth, TAOCP vol. 2,
// 4.2.2: s + e = a + b exactly), Fast2Sum (Dekker 1971, the same for
// |a| >= |b|) and TwoProd by one fused multiply-add (p + e = a b exactly).
// Sums take the short form (one TwoSum, the low parts added, renormalised):
// its error is a few units of 2^-47 of the larger operand, the analogue of
// FP64 rounding on the operands.  The rounded operations of the
// transformations are written as the non-contractible intrinsics, and nothing
// is compiled with fast-math, so the compiler neither fuses, reassociates nor
// drops the compensating terms.
#pragma once
#include <cuda_runtime.h>
#include <math.h>

#include "rt_device.cuh"

namespace rtk {

struct DF {
  float hi, lo;
  DF() = default;
  RT_HD constexpr DF(float h, float l) : hi(h), lo(l) {}
  RT_HD constexpr DF(int i) : hi((float)i), lo(0.0f) {}
  // rounding of a double (exact for the 48 leading bits); constexpr so that
  // constants fold at compile time
  RT_HD constexpr explicit DF(double d) : hi((float)d), lo((float)(d - (double)(float)d)) {}
};

// Rounded FP32 operations the compiler may not fuse into a multiply-add: a
// contraction of a product with the sum that follows would make the rounding
// error computed from them wrong.
RT_HD __forceinline__ float rn_add(float a, float b) {
#ifdef __CUDA_ARCH__
  return __fadd_rn(a, b);
#else
  return a + b;
#endif
}
RT_HD __forceinline__ float rn_sub(float a, float b) {
#ifdef __CUDA_ARCH__
  return __fsub_rn(a, b);
#else
  return a - b;
#endif
}
RT_HD __forceinline__ float rn_mul(float a, float b) {
#ifdef __CUDA_ARCH__
  return __fmul_rn(a, b);
#else
  return a * b;
#endif
}

RT_HD __forceinline__ DF df_fast_sum(float a, float b) {   // |a| >= |b| (or a == 0)
  const float s = rn_add(a, b);
  return DF(s, rn_sub(b, rn_sub(s, a)));
}
RT_HD __forceinline__ DF df_two_sum(float a, float b) {
  const float s = rn_add(a, b);
  const float bb = rn_sub(s, a);
  return DF(s, rn_add(rn_sub(a, rn_sub(s, bb)), rn_sub(b, bb)));
}
RT_HD __forceinline__ DF df_two_prod(float a, float b) {
  const float p = rn_mul(a, b);
  return DF(p, fmaf(a, b, -p));
}

RT_HD __forceinline__ DF operator+(DF a, DF b) {
  const DF s = df_two_sum(a.hi, b.hi);
  return df_fast_sum(s.hi, s.lo + (a.lo + b.lo));
}
RT_HD __forceinline__ DF operator+(DF a, float b) {
  const DF s = df_two_sum(a.hi, b);
  return df_fast_sum(s.hi, s.lo + a.lo);
}
RT_HD __forceinline__ DF operator-(DF a) { return DF(-a.hi, -a.lo); }
RT_HD __forceinline__ DF operator-(DF a, DF b) { return a + (-b); }
RT_HD __forceinline__ DF operator*(DF a, DF b) {
  const float p = rn_mul(a.hi, b.hi);
  return df_fast_sum(p, fmaf(a.hi, b.lo, fmaf(a.lo, b.hi, fmaf(a.hi, b.hi, -p))));
}
RT_HD __forceinline__ DF operator*(DF a, float b) {
  const float p = rn_mul(a.hi, b);
  return df_fast_sum(p, fmaf(a.lo, b, fmaf(a.hi, b, -p)));
}
RT_HD __forceinline__ DF operator*(float b, DF a) { return a * b; }
RT_HD __forceinline__ DF& operator+=(DF& a, DF b) {
  a = a + b;
  return a;
}
RT_HD __forceinline__ DF& operator-=(DF& a, DF b) {
  a = a - b;
  return a;
}
RT_HD __forceinline__ bool operator<(DF a, DF b) {
  return a.hi < b.hi || (a.hi == b.hi && a.lo < b.lo);
}
RT_HD __forceinline__ bool operator>(DF a, DF b) { return b < a; }
RT_HD __forceinline__ bool operator<=(DF a, DF b) { return !(b < a); }
RT_HD __forceinline__ bool operator>=(DF a, DF b) { return !(a < b); }
RT_HD __forceinline__ bool operator==(DF a, DF b) { return a.hi == b.hi && a.lo == b.lo; }
RT_HD __forceinline__ bool operator!=(DF a, DF b) { return !(a == b); }

// hi is the rounding of hi + lo to FP32
RT_HD __forceinline__ float df_f(DF a) { return a.hi; }
RT_HD __forceinline__ double df_d(DF a) { return (double)a.hi + (double)a.lo; }
RT_HD __forceinline__ DF df_of(double d) {
  const float h = (float)d;
  return DF(h, (float)(d - (double)h));
}

RT_HD __forceinline__ bool df_le(DF a, DF b) { return !(b < a); }
RT_HD __forceinline__ DF df_abs(DF a) { return (a.hi < 0.0f) ? -a : a; }
RT_HD __forceinline__ DF df_max(DF a, DF b) { return (a < b) ? b : a; }

// a / b: the FP32 quotient q corrected by the remainder a - q b formed in
// double-float, q + (a - q b) / b.
RT_HD __forceinline__ DF df_div(DF a, DF b) {
  const float q = a.hi / b.hi;
  const DF r = a - b * q;
  return df_fast_sum(q, r.hi / b.hi);
}

// sqrt(x): the FP32 root y corrected by the remainder, y + (x - y^2) / (2 y).
RT_HD __forceinline__ DF df_sqrt(DF x) {
  if (!(x.hi > 0.0f)) return DF(0.0f, 0.0f);
  const float y = sqrtf(x.hi);
  const DF r = x - df_two_prod(y, y);
  return df_fast_sum(y, r.hi * 0.5f / y);
}
RT_HD __forceinline__ DF operator/(DF a, DF b) { return df_div(a, b); }
RT_HD __forceinline__ DF rt_sqrt(DF x) { return df_sqrt(x); }

// x^(-1/5) for x in [1e-6, 1e6] (the step-size controller's power): the FP32
// estimate y corrected by the series of (1 - r)^(-1/5) in the residual
// r = 1 - x y^5 formed in double-float, y (1 + r/5 + 3 r^2/25).
RT_HD __forceinline__ DF df_pow_m1_5(DF x) {
  const float y = exp2f(-0.2f * log2f(x.hi));
  const DF y2 = df_two_prod(y, y);
  const DF t = x * ((y2 * y2) * y);
  const float r = (1.0f - t.hi) - t.lo;
  return df_fast_sum(y, y * (r * fmaf(0.12f, r, 0.2f)));
}

// 1/sqrt(x): the FP32 estimate y (within 2 ulp) corrected by the series of
// (1 - r)^(-1/2) in the residual r = 1 - x y^2 formed in double-float,
// y (1 + r/2 + 3 r^2/8): the truncation is O(r^3) ~ 2^-66, the result good to
// the double-float rounding.
RT_HD __forceinline__ DF rt_rsqrt(DF x) {
#ifdef __CUDA_ARCH__
  const float y = rsqrtf(x.hi);
#else
  const float y = 1.0f / sqrtf(x.hi);
#endif
  const DF xy2 = x * df_two_prod(y, y);
  const float r = (1.0f - xy2.hi) - xy2.lo;     // 1 - xy2.hi is exact (Sterbenz)
  return df_fast_sum(y, 0.5f * y * r * fmaf(0.75f, r, 1.0f));
}

}  // namespace rtk
