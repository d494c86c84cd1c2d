// Oracle (test infrastructure only; never linked into the product path).
//
// Forward-mode dual numbers.  The oracle obtains every derivative of the
// Hamiltonian (Hamilton's equations, Eq. Hamilton, Sec. 2) and of the
// resonance function (the Jacobian of the delta function, Eq. IntegralTrick,
// Sec. 3) by differentiating the plain formula automatically, so it shares no
// hand-derived gradient with the CUDA path.
#pragma once
#include <cmath>

namespace orc {

using std::fabs;
using std::sqrt;
using std::sin;
using std::cos;

template <int N>
struct Dual {
  double v;
  double d[N];
  Dual() : v(0.0) { for (int i = 0; i < N; ++i) d[i] = 0.0; }
  Dual(double x) : v(x) { for (int i = 0; i < N; ++i) d[i] = 0.0; }  // NOLINT
  static Dual var(double x, int i) { Dual r(x); r.d[i] = 1.0; return r; }
};

template <int N> inline Dual<N> operator+(const Dual<N>& a, const Dual<N>& b) {
  Dual<N> r; r.v = a.v + b.v; for (int i = 0; i < N; ++i) r.d[i] = a.d[i] + b.d[i]; return r;
}
template <int N> inline Dual<N> operator-(const Dual<N>& a, const Dual<N>& b) {
  Dual<N> r; r.v = a.v - b.v; for (int i = 0; i < N; ++i) r.d[i] = a.d[i] - b.d[i]; return r;
}
template <int N> inline Dual<N> operator-(const Dual<N>& a) {
  Dual<N> r; r.v = -a.v; for (int i = 0; i < N; ++i) r.d[i] = -a.d[i]; return r;
}
template <int N> inline Dual<N> operator*(const Dual<N>& a, const Dual<N>& b) {
  Dual<N> r; r.v = a.v * b.v;
  for (int i = 0; i < N; ++i) r.d[i] = a.d[i] * b.v + a.v * b.d[i];
  return r;
}
template <int N> inline Dual<N> operator/(const Dual<N>& a, const Dual<N>& b) {
  Dual<N> r; r.v = a.v / b.v;
  for (int i = 0; i < N; ++i) r.d[i] = (a.d[i] * b.v - a.v * b.d[i]) / (b.v * b.v);
  return r;
}
template <int N> inline Dual<N> operator+(const Dual<N>& a, double b) { return a + Dual<N>(b); }
template <int N> inline Dual<N> operator+(double a, const Dual<N>& b) { return Dual<N>(a) + b; }
template <int N> inline Dual<N> operator-(const Dual<N>& a, double b) { return a - Dual<N>(b); }
template <int N> inline Dual<N> operator-(double a, const Dual<N>& b) { return Dual<N>(a) - b; }
template <int N> inline Dual<N> operator*(const Dual<N>& a, double b) { return a * Dual<N>(b); }
template <int N> inline Dual<N> operator*(double a, const Dual<N>& b) { return Dual<N>(a) * b; }
template <int N> inline Dual<N> operator/(const Dual<N>& a, double b) { return a / Dual<N>(b); }
template <int N> inline Dual<N> operator/(double a, const Dual<N>& b) { return Dual<N>(a) / b; }

template <int N> inline Dual<N> sqrt(const Dual<N>& a) {
  Dual<N> r; r.v = std::sqrt(a.v);
  for (int i = 0; i < N; ++i) r.d[i] = a.d[i] / (2.0 * r.v);
  return r;
}
// |a|: derivative sign(a) * a' (the kink at a = 0 is a set of measure zero).
template <int N> inline Dual<N> fabs(const Dual<N>& a) {
  return a.v < 0.0 ? -a : a;
}

// sin and cos (the rotation phase of a rotating magnetic axis, Eq. GJDensity).
template <int N> inline Dual<N> sin(const Dual<N>& a) {
  Dual<N> r; r.v = std::sin(a.v);
  const double c = std::cos(a.v);
  for (int i = 0; i < N; ++i) r.d[i] = c * a.d[i];
  return r;
}
template <int N> inline Dual<N> cos(const Dual<N>& a) {
  Dual<N> r; r.v = std::cos(a.v);
  const double sn = std::sin(a.v);
  for (int i = 0; i < N; ++i) r.d[i] = -sn * a.d[i];
  return r;
}

inline double value(double x) { return x; }
template <int N> inline double value(const Dual<N>& x) { return x.v; }

}  // namespace orc
