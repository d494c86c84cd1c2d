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

// Dual<N, T>: value and N tangent components in the scalar type T (double, or
// float for the single-precision reverse sweep).
template <int N, class T = double>
struct Dual {
  T v;
  T d[N];
  RT_HD Dual() : v(T(0)) {
#pragma unroll
    for (int i = 0; i < N; ++i) d[i] = T(0);
  }
  RT_HD Dual(T x) : v(x) {  // NOLINT: implicit constants
#pragma unroll
    for (int i = 0; i < N; ++i) d[i] = T(0);
  }
  RT_HD static Dual var(T x, int k) {
    Dual r(x);
    r.d[k] = T(1);
    return r;
  }
};

template <int N, class T>
RT_HD __forceinline__ Dual<N, T> operator+(const Dual<N, T>& a, const Dual<N, T>& b) {
  Dual<N, T> r;
  r.v = a.v + b.v;
#pragma unroll
  for (int i = 0; i < N; ++i) r.d[i] = a.d[i] + b.d[i];
  return r;
}
template <int N, class T>
RT_HD __forceinline__ Dual<N, T> operator-(const Dual<N, T>& a, const Dual<N, T>& b) {
  Dual<N, T> r;
  r.v = a.v - b.v;
#pragma unroll
  for (int i = 0; i < N; ++i) r.d[i] = a.d[i] - b.d[i];
  return r;
}
template <int N, class T>
RT_HD __forceinline__ Dual<N, T> operator-(const Dual<N, T>& a) {
  Dual<N, T> r;
  r.v = -a.v;
#pragma unroll
  for (int i = 0; i < N; ++i) r.d[i] = -a.d[i];
  return r;
}
template <int N, class T>
RT_HD __forceinline__ Dual<N, T> operator*(const Dual<N, T>& a, const Dual<N, T>& b) {
  Dual<N, T> r;
  r.v = a.v * b.v;
#pragma unroll
  for (int i = 0; i < N; ++i) r.d[i] = a.d[i] * b.v + a.v * b.d[i];
  return r;
}
template <int N, class T>
RT_HD __forceinline__ Dual<N, T> operator/(const Dual<N, T>& a, const Dual<N, T>& b) {
  Dual<N, T> r;
  const T ib = T(1) / b.v;
  r.v = a.v / b.v;   // the value rounds exactly as in plain arithmetic
#pragma unroll
  for (int i = 0; i < N; ++i) r.d[i] = (a.d[i] - r.v * b.d[i]) * ib;
  return r;
}
template <int N, class T>
RT_HD __forceinline__ Dual<N, T>& operator+=(Dual<N, T>& a, const Dual<N, T>& b) {
  a = a + b;
  return a;
}
template <int N, class T>
RT_HD __forceinline__ Dual<N, T>& operator-=(Dual<N, T>& a, const Dual<N, T>& b) {
  a = a - b;
  return a;
}
template <int N, class T>
RT_HD __forceinline__ Dual<N, T>& operator*=(Dual<N, T>& a, const Dual<N, T>& b) {
  a = a * b;
  return a;
}
template <int N, class T>
RT_HD __forceinline__ bool operator<(const Dual<N, T>& a, const Dual<N, T>& b) {
  return a.v < b.v;
}
template <int N, class T>
RT_HD __forceinline__ bool operator>(const Dual<N, T>& a, const Dual<N, T>& b) {
  return a.v > b.v;
}

// chain rule for a scalar function with value fv and derivative df at a.v
template <int N, class T>
RT_HD __forceinline__ Dual<N, T> chain(const Dual<N, T>& a, T fv, T df) {
  Dual<N, T> r;
  r.v = fv;
#pragma unroll
  for (int i = 0; i < N; ++i) r.d[i] = df * a.d[i];
  return r;
}

template <int N, class T>
RT_HD __forceinline__ Dual<N, T> rt_sqrt(const Dual<N, T>& a) {
  const T s = rt_sqrt(a.v);
  return chain(a, s, T(0.5) / s);
}
template <int N, class T>
RT_HD __forceinline__ Dual<N, T> rt_rsqrt(const Dual<N, T>& a) {
  const T q = T(1) / rt_sqrt(a.v);
  return chain(a, q, T(-0.5) * q * q * q);
}
template <int N, class T>
RT_HD __forceinline__ Dual<N, T> rt_rcp(const Dual<N, T>& a) {
  const T q = T(1) / a.v;
  return chain(a, q, -q * q);
}
template <int N, class T>
RT_HD __forceinline__ Dual<N, T> dabs(const Dual<N, T>& a) {
  return a.v < T(0) ? -a : a;
}
template <int N, class T>
RT_HD __forceinline__ Dual<N, T> dsin(const Dual<N, T>& a) {
  return chain(a, T(sin(a.v)), T(cos(a.v)));
}
template <int N, class T>
RT_HD __forceinline__ Dual<N, T> dcos(const Dual<N, T>& a) {
  return chain(a, T(cos(a.v)), T(-sin(a.v)));
}
template <int N, class T>
RT_HD __forceinline__ Dual<N, T> dexp(const Dual<N, T>& a) {
  const T e = exp(a.v);
  return chain(a, e, e);
}

}  // namespace rtk
