// Forward-mode dual numbers with N tangent directions, for device code.
//
// The adjoint of the integrator needs products of the right-hand side's
// Jacobian with vectors.  Instantiating the analytic right-hand side
// (ham_rhs) with Dual<N> gives J u for a seeded direction u, and the
// derivatives with respect to the star constants it reads, exactly (to
// rounding), without a second hand derivation of the Hessian of H.
#pragma once
#include <cuda_runtime.h>

#include "rt_device.cuh"

namespace rtk {

template <int N>
struct Dual {
  double v;
  double d[N];
  RT_HD Dual() : v(0.0) {
#pragma unroll
    for (int i = 0; i < N; ++i) d[i] = 0.0;
  }
  RT_HD Dual(double x) : v(x) {  // NOLINT: implicit constants
#pragma unroll
    for (int i = 0; i < N; ++i) d[i] = 0.0;
  }
  RT_HD static Dual var(double x, int k) {
    Dual r(x);
    r.d[k] = 1.0;
    return r;
  }
};

template <int N>
RT_HD __forceinline__ Dual<N> operator+(const Dual<N>& a, const Dual<N>& b) {
  Dual<N> r;
  r.v = a.v + b.v;
#pragma unroll
  for (int i = 0; i < N; ++i) r.d[i] = a.d[i] + b.d[i];
  return r;
}
template <int N>
RT_HD __forceinline__ Dual<N> operator-(const Dual<N>& a, const Dual<N>& b) {
  Dual<N> r;
  r.v = a.v - b.v;
#pragma unroll
  for (int i = 0; i < N; ++i) r.d[i] = a.d[i] - b.d[i];
  return r;
}
template <int N>
RT_HD __forceinline__ Dual<N> operator-(const Dual<N>& a) {
  Dual<N> r;
  r.v = -a.v;
#pragma unroll
  for (int i = 0; i < N; ++i) r.d[i] = -a.d[i];
  return r;
}
template <int N>
RT_HD __forceinline__ Dual<N> operator*(const Dual<N>& a, const Dual<N>& b) {
  Dual<N> r;
  r.v = a.v * b.v;
#pragma unroll
  for (int i = 0; i < N; ++i) r.d[i] = a.d[i] * b.v + a.v * b.d[i];
  return r;
}
template <int N>
RT_HD __forceinline__ Dual<N> operator/(const Dual<N>& a, const Dual<N>& b) {
  Dual<N> r;
  const double ib = 1.0 / b.v;
  r.v = a.v / b.v;   // the value rounds exactly as in double arithmetic
#pragma unroll
  for (int i = 0; i < N; ++i) r.d[i] = (a.d[i] - r.v * b.d[i]) * ib;
  return r;
}
template <int N>
RT_HD __forceinline__ Dual<N>& operator+=(Dual<N>& a, const Dual<N>& b) {
  a = a + b;
  return a;
}
template <int N>
RT_HD __forceinline__ Dual<N>& operator-=(Dual<N>& a, const Dual<N>& b) {
  a = a - b;
  return a;
}
template <int N>
RT_HD __forceinline__ Dual<N>& operator*=(Dual<N>& a, const Dual<N>& b) {
  a = a * b;
  return a;
}
template <int N>
RT_HD __forceinline__ bool operator<(const Dual<N>& a, const Dual<N>& b) { return a.v < b.v; }
template <int N>
RT_HD __forceinline__ bool operator>(const Dual<N>& a, const Dual<N>& b) { return a.v > b.v; }

// chain rule for a scalar function with value fv and derivative df at a.v
template <int N>
RT_HD __forceinline__ Dual<N> chain(const Dual<N>& a, double fv, double df) {
  Dual<N> r;
  r.v = fv;
#pragma unroll
  for (int i = 0; i < N; ++i) r.d[i] = df * a.d[i];
  return r;
}

template <int N>
RT_HD __forceinline__ Dual<N> rt_sqrt(const Dual<N>& a) {
  const double s = sqrt(a.v);
  return chain(a, s, 0.5 / s);
}
template <int N>
RT_HD __forceinline__ Dual<N> rt_rsqrt(const Dual<N>& a) {
  const double q = 1.0 / sqrt(a.v);
  return chain(a, q, -0.5 * q * q * q);
}
template <int N>
RT_HD __forceinline__ Dual<N> rt_rcp(const Dual<N>& a) {
  const double q = 1.0 / a.v;
  return chain(a, q, -q * q);
}
template <int N>
RT_HD __forceinline__ Dual<N> dabs(const Dual<N>& a) {
  return a.v < 0.0 ? -a : a;
}
template <int N>
RT_HD __forceinline__ Dual<N> dsin(const Dual<N>& a) {
  return chain(a, sin(a.v), cos(a.v));
}
template <int N>
RT_HD __forceinline__ Dual<N> dcos(const Dual<N>& a) {
  return chain(a, cos(a.v), -sin(a.v));
}
template <int N>
RT_HD __forceinline__ Dual<N> dexp(const Dual<N>& a) {
  const double e = exp(a.v);
  return chain(a, e, e);
}

}  // namespace rtk
