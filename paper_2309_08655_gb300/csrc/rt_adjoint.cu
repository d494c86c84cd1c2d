// Reverse-mode (adjoint) gradient of a smooth line-flux functional through
// sampling and the FP64 integrator.
//
// Functional (a reading: the paper differentiates nothing; the functional is
// the line flux toward an observer, smoothed on the sphere):
//   F = sum_i w_i K(khat_i . o),  K(mu) = C exp(kappa (mu - 1)),
//   C = kappa / (2 pi (1 - exp(-2 kappa)))   (von Mises-Fisher, unit mass),
// over ESCAPED rays, khat_i the static orthonormal-frame momentum direction at
// the escape point r = r_out, o = (sin i, 0, cos i).  Parameters p = (m_a
// [eV], B0 [G], theta_m [rad], M [Msun], R [km], i [rad]).
//
// dF/dp = sum_i [ K dw_i/dp + w_i K' dmu_i/dp ], where mu_i depends on p through
// the initial state y0(p) and the constants q = (r_s/R, omega_p^2 coefficient,
// magnetic axis m) of the ray equations.  Per ray:
//  * y0, w and their p-derivatives come from the sampling code instantiated
//    with 5-tangent dual numbers (the root's derivative by the implicit
//    function theorem);
//  * the trajectory is replayed from checkpoints stored every CK accepted
//    steps, each segment re-integrated (bitwise the same steps) and swept
//    backwards step by step: the discrete adjoint of a Dormand-Prince step at
//    its accepted step size, with J^T v of the right-hand side f = Omega grad H
//    obtained from one forward-mode product, J^T v = Omega J (Omega v), and the
//    q-derivatives from the same dual evaluation (q = r_s, the omega_p^2
//    coefficient, and the magnetic axis along dm/dtheta_m: four tangents);
//  * where the Goldreich-Julian branch switches on the null cone c(x) = 0
//    (the right-hand side jumps there), the saltation matrix
//    S = I + (f_new - f_old) grad c^T / (grad c . f_old) is applied, together
//    with the shift of the crossing with the magnetic axis;
//  * the escape point is the continuous extension at the theta* where
//    |x| = r_out, differentiated with theta* implicit.
#include <cuda_runtime.h>
#include <stdint.h>

#include "rt_df.cuh"
#include "rt_dual.cuh"
#include "rt_integrator.cuh"
#include "rt_internal.h"
#include "rt_sample_core.cuh"

namespace rtk {

// dual-number overloads used by the sampling core (argument-dependent lookup)
template <int N>
__device__ __forceinline__ double val(const Dual<N>& x) {
  return x.v;
}
template <int N>
__device__ __forceinline__ Dual<N> tabs(const Dual<N>& x) {
  return dabs(x);
}
template <int N>
__device__ __forceinline__ Dual<N> root_of(double r, const Dual<N>& G, double dGdr) {
  Dual<N> o(r);
#pragma unroll
  for (int k = 0; k < N; ++k) o.d[k] = -G.d[k] / dGdr;
  return o;
}

// 1/sqrt of a double-float dual: the value by the series-corrected
// double-float rsqrt, the derivative -q^3 / 2.
template <int N>
__device__ __forceinline__ Dual<N, DF> rt_rsqrt(const Dual<N, DF>& a) {
  const DF q = rt_rsqrt(a.v);
  return chain(a, q, DF(-0.5) * (q * q) * q);
}

__device__ __forceinline__ double dval(double x) { return x; }
__device__ __forceinline__ double dval(float x) { return (double)x; }
__device__ __forceinline__ double dval(DF x) { return df_d(x); }

namespace {

using sampling::SampConst;
using sampling::SampOut;
using sampling::sample_core;

typedef Dual<6> D6;

// A segment record's stage derivatives start here (SEGREC, rt_internal.h): the
// reverse sweep reads them back instead of re-forming the stages.
constexpr int SEG_K = 10;
enum { FL_FLIP_BEFORE = 1, FL_FLIP_AFTER = 2, FL_ESCAPE = 4 };

struct AdjParams {
  SampConst<Dual<NSAMP_TANGENTS>> sc;
  SampConst<double> scv;
  double R_km, ma_eV, rs_prop, cp, plasma_a, cos_tm, sin_tm;
  int dispersion, plasma;
  double drsp_dM, drsp_dR, dcp_dma, dcp_dB0;
  double incl, kappa, knorm;
  double rtol, atol, r_out, r_capture;
  int max_steps;
  int64_t n;
  const double* u;
  const int64_t* ck_off;
  double* ck;
  double* seg;
  double* F_ray;
  double* G_ray;
  uint8_t* status;
  int32_t* flags;
  int64_t* counters;
  unsigned long long* queue;
  const int64_t* tape_off;
  double* tape;
  double* head;
  const int64_t* order;
};

// Right-hand side in the sweep's precision T.
template <class T>
__device__ __forceinline__ void rhs_t(const RayConst<T>& c, const T* y, T* f) {
  ham_rhs<T>(c, y[0], y[1], y[2], y[3], y[4], y[5], f[0], f[1], f[2], f[3], f[4], f[5]);
}

// The ray's constants in the sweep's precision.
template <class T>
__device__ __forceinline__ RayConst<T> cast_const(const RayConst<double>& c) {
  RayConst<T> o;
  o.rs = T(c.rs);
  o.cp = T(c.cp);
  o.pa = T(c.pa);
  o.W2 = T(c.W2);
  o.iW2 = T(c.iW2);
  o.m0 = T(c.m0);
  o.m1 = T(c.m1);
  o.m2 = T(c.m2);
  o.sig = T(c.sig);
  o.disp = c.disp;
  o.plasma = c.plasma;
  return o;
}

// Constants q of the ray equations that the parameters move: r_s / R, the
// omega_p^2 coefficient, and the misalignment theta_m, which moves the
// magnetic axis m along dm/dtheta_m (the ray's rotation phase is fixed).
constexpr int NQ = 3;
enum { Q_RS = 0, Q_CP, Q_THM };

// J^T v and v . df/dq at y, from one dual evaluation in the scalar type T
// with 1 + NQ tangents: the direction Omega v, and q (m along dm).
template <class T>
__device__ __noinline__ void rhs_vjp(const RayConst<T>& c, const T* dm, const T* y, const T* v,
                                     T* out, T* qbar) {
  typedef Dual<1 + NQ, T> DT;
  RayConst<DT> cd;
  cd.rs = DT::var(c.rs, 1 + Q_RS);
  cd.cp = DT::var(c.cp, 1 + Q_CP);
  cd.pa = DT(c.pa);
  cd.W2 = DT(c.W2);
  cd.iW2 = DT(c.iW2);
  cd.m0 = DT(c.m0);
  cd.m1 = DT(c.m1);
  cd.m2 = DT(c.m2);
  cd.m0.d[1 + Q_THM] = dm[0];
  cd.m1.d[1 + Q_THM] = dm[1];
  cd.m2.d[1 + Q_THM] = dm[2];
  cd.sig = DT(c.sig);
  cd.disp = c.disp;
  cd.plasma = c.plasma;
  // u = Omega v = (v_k, -v_x)
  DT yd[6];
#pragma unroll
  for (int j = 0; j < 3; ++j) {
    yd[j] = DT(y[j]);
    yd[j].d[0] = v[3 + j];
    yd[3 + j] = DT(y[3 + j]);
    yd[3 + j].d[0] = -v[j];
  }
  DT f[6];
  ham_rhs<DT>(cd, yd[0], yd[1], yd[2], yd[3], yd[4], yd[5], f[0], f[1], f[2], f[3], f[4], f[5]);
  // J^T v = Omega (J u) = ((Ju)_k, -(Ju)_x)
#pragma unroll
  for (int j = 0; j < 3; ++j) {
    out[j] = f[3 + j].d[0];
    out[3 + j] = -f[j].d[0];
  }
#pragma unroll
  for (int m = 1; m <= NQ; ++m) {
    T s = T(0);
#pragma unroll
    for (int j = 0; j < 6; ++j) s += v[j] * f[j].d[m];
    qbar[m - 1] += s;
  }
}

// Dual number of the mixed sweep: the value and the state-direction tangent in
// FP64 (the tangent that carries the adjoint along the trajectory, where
// rounding errors compound), an FP32 copy of the value from its own FP32
// evaluation, and the NQ parameter tangents in FP32 (their products with the
// adjoint only add up over the steps).  A product costs 3 FP64 operations
// instead of the 9 of a four-tangent FP64 dual.
struct HDual {
  double v, d;
  float vf;
  float q[NQ];
  HDual() = default;
  __device__ HDual(int i) : v((double)i), d(0.0), vf((float)i) {  // NOLINT: constants
#pragma unroll
    for (int k = 0; k < NQ; ++k) q[k] = 0.0f;
  }
  __device__ explicit HDual(double x) : v(x), d(0.0), vf((float)x) {
#pragma unroll
    for (int k = 0; k < NQ; ++k) q[k] = 0.0f;
  }
};
__device__ __forceinline__ HDual operator+(const HDual& a, const HDual& b) {
  HDual r;
  r.v = a.v + b.v;
  r.d = a.d + b.d;
  r.vf = a.vf + b.vf;
#pragma unroll
  for (int k = 0; k < NQ; ++k) r.q[k] = a.q[k] + b.q[k];
  return r;
}
__device__ __forceinline__ HDual operator-(const HDual& a, const HDual& b) {
  HDual r;
  r.v = a.v - b.v;
  r.d = a.d - b.d;
  r.vf = a.vf - b.vf;
#pragma unroll
  for (int k = 0; k < NQ; ++k) r.q[k] = a.q[k] - b.q[k];
  return r;
}
__device__ __forceinline__ HDual operator-(const HDual& a) {
  HDual r;
  r.v = -a.v;
  r.d = -a.d;
  r.vf = -a.vf;
#pragma unroll
  for (int k = 0; k < NQ; ++k) r.q[k] = -a.q[k];
  return r;
}
__device__ __forceinline__ HDual operator*(const HDual& a, const HDual& b) {
  HDual r;
  r.v = a.v * b.v;
  r.d = a.d * b.v + a.v * b.d;
  r.vf = a.vf * b.vf;
#pragma unroll
  for (int k = 0; k < NQ; ++k) r.q[k] = a.q[k] * b.vf + a.vf * b.q[k];
  return r;
}
__device__ __forceinline__ HDual& operator+=(HDual& a, const HDual& b) {
  a = a + b;
  return a;
}
__device__ __forceinline__ HDual& operator-=(HDual& a, const HDual& b) {
  a = a - b;
  return a;
}
__device__ __forceinline__ bool operator<(const HDual& a, const HDual& b) { return a.v < b.v; }
__device__ __forceinline__ bool operator>(const HDual& a, const HDual& b) { return a.v > b.v; }
__device__ __forceinline__ HDual rt_rsqrt(const HDual& a) {
  HDual r;
  r.v = ::rtk::rt_rsqrt(a.v);
  r.d = -0.5 * r.v * r.v * r.v * a.d;
  r.vf = rsqrtf(a.vf);
  const float cf = -0.5f * r.vf * r.vf * r.vf;
#pragma unroll
  for (int k = 0; k < NQ; ++k) r.q[k] = cf * a.q[k];
  return r;
}
__device__ __forceinline__ HDual rt_sqrt(const HDual& a) {
  HDual r;
  r.v = sqrt(a.v);
  r.d = 0.5 / r.v * a.d;
  r.vf = sqrtf(a.vf);
  const float cf = 0.5f / r.vf;
#pragma unroll
  for (int k = 0; k < NQ; ++k) r.q[k] = cf * a.q[k];
  return r;
}

// rhs_vjp for the mixed sweep (HDual): J^T v in FP64, v . df/dq from the FP32
// parameter tangents (summed in FP32 per stage, accumulated in FP64).
__device__ __noinline__ void rhs_vjp_h(const RayConst<double>& c, const double* dm,
                                       const double* y, const double* v, double* out,
                                       double* qbar) {
  RayConst<HDual> cd;
  cd.rs = HDual(c.rs);
  cd.rs.q[Q_RS] = 1.0f;
  cd.cp = HDual(c.cp);
  cd.cp.q[Q_CP] = 1.0f;
  cd.pa = HDual(c.pa);
  cd.W2 = HDual(c.W2);
  cd.iW2 = HDual(c.iW2);
  cd.m0 = HDual(c.m0);
  cd.m1 = HDual(c.m1);
  cd.m2 = HDual(c.m2);
  cd.m0.q[Q_THM] = (float)dm[0];
  cd.m1.q[Q_THM] = (float)dm[1];
  cd.m2.q[Q_THM] = (float)dm[2];
  cd.sig = HDual(c.sig);
  cd.disp = c.disp;
  cd.plasma = c.plasma;
  HDual yd[6];
#pragma unroll
  for (int j = 0; j < 3; ++j) {
    yd[j] = HDual(y[j]);
    yd[j].d = v[3 + j];
    yd[3 + j] = HDual(y[3 + j]);
    yd[3 + j].d = -v[j];
  }
  HDual f[6];
  ham_rhs<HDual>(cd, yd[0], yd[1], yd[2], yd[3], yd[4], yd[5], f[0], f[1], f[2], f[3], f[4],
                 f[5]);
#pragma unroll
  for (int j = 0; j < 3; ++j) {
    out[j] = f[3 + j].d;
    out[3 + j] = -f[j].d;
  }
  float vf[6];
#pragma unroll
  for (int j = 0; j < 6; ++j) vf[j] = (float)v[j];
#pragma unroll
  for (int m = 0; m < NQ; ++m) {
    float s = 0.0f;
#pragma unroll
    for (int j = 0; j < 6; ++j) s += vf[j] * f[j].q[m];
    qbar[m] += (double)s;
  }
}

// The Jacobian product of the sweep: four-tangent duals in T, or (HYB, T =
// double) the mixed HDual.
template <bool HYB, class T>
__device__ __forceinline__ void vjp(const RayConst<T>& c, const T* dm, const T* y, const T* v,
                                    T* out, T* qbar) {
  if constexpr (HYB)
    rhs_vjp_h(c, dm, y, v, out, qbar);
  else
    rhs_vjp(c, dm, y, v, out, qbar);
}

// Adjoint of a branch switch at y from sig_old to -sig_old:
// ybar <- S^T ybar, and the crossing's dependence on the magnetic axis.
template <class T>
__device__ void saltation(RayConst<T> c, const T* dm, const T* y, T sig_old, T* ybar, T* qbar) {
  T fo[6], fn[6];
  c.sig = sig_old;
  rhs_t(c, y, fo);
  c.sig = -sig_old;
  rhs_t(c, y, fn);
  // c(x) = 3 z (m.x) - m_z |x|^2 (the sign of Omega . B)
  const T mx = c.m0 * y[0] + c.m1 * y[1] + c.m2 * y[2];
  const T gc0 = T(3) * y[2] * c.m0 - T(2) * c.m2 * y[0];
  const T gc1 = T(3) * y[2] * c.m1 - T(2) * c.m2 * y[1];
  const T gc2 = T(3) * mx + T(3) * y[2] * c.m2 - T(2) * c.m2 * y[2];
  const T den = gc0 * fo[0] + gc1 * fo[1] + gc2 * fo[2];
  if (den == T(0)) return;
  T num = T(0);
#pragma unroll
  for (int j = 0; j < 6; ++j) num += (fn[j] - fo[j]) * ybar[j];
  const T s = num / den;
  ybar[0] += s * gc0;
  ybar[1] += s * gc1;
  ybar[2] += s * gc2;
  // the crossing moves with the axis: dc/dm . dm/dtheta_m
  const T r2 = y[0] * y[0] + y[1] * y[1] + y[2] * y[2];
  qbar[Q_THM] += s * (T(3) * y[2] * y[0] * dm[0] + T(3) * y[2] * y[1] * dm[1] +
                      (T(3) * y[2] * y[2] - r2) * dm[2]);
}

// Discrete adjoint of one accepted Dormand-Prince step from y with step h, in
// the scalar type T (double: the FP64 sweep, or with HYB the mixed sweep whose
// Jacobian products take FP32 parameter tangents; DF: the double-float
// sweep), from the step's FP64 record (its seven stage derivatives K, as the
// replay formed them).
// ybar: in, the adjoint at the step's end (unused when escape); out, at y.
// Escape: the step ends at the theta* of the continuous extension where
// |x| = r_out, and ybar_e is the adjoint there.
template <class T, bool HYB = false>
__device__ void step_adjoint(const RayConst<T>& c, const T* dm, const T* y, T h,
                             const double* Krec, bool escape, T r_out, const T* ybar_e, T* ybar,
                             T* qbar) {
  const T b1 = T(DP::b1), b3 = T(DP::b3), b4 = T(DP::b4), b5 = T(DP::b5), b6 = T(DP::b6);
  T K[7][6], t[6];
#pragma unroll
  for (int s = 0; s < 7; ++s)
#pragma unroll
    for (int i = 0; i < 6; ++i) K[s][i] = T(Krec[6 * s + i]);
  T kb[7][6], ynb[6], yb[6];
#pragma unroll
  for (int s = 0; s < 7; ++s)
#pragma unroll
    for (int i = 0; i < 6; ++i) kb[s][i] = T(0);
  if (escape) {
    const T d1 = T(DP::d1), d3 = T(DP::d3), d4 = T(DP::d4), d5 = T(DP::d5), d6 = T(DP::d6),
            d7 = T(DP::d7);
    T yn[6], r2v[6], r3[6], r4[6], r5[6];
#pragma unroll
    for (int i = 0; i < 6; ++i) {
      yn[i] = y[i] + h * (b1 * K[0][i] + b3 * K[2][i] + b4 * K[3][i] + b5 * K[4][i] +
                          b6 * K[5][i]);
      r2v[i] = yn[i] - y[i];
      r3[i] = h * K[0][i] - r2v[i];
      r4[i] = r2v[i] - h * K[6][i] - r3[i];
      r5[i] = h * (d1 * K[0][i] + d3 * K[2][i] + d4 * K[3][i] + d5 * K[4][i] + d6 * K[5][i] +
                   d7 * K[6][i]);
    }
    // the same bisection as the forward step
    T lo = T(0), hi = T(1);
    for (int it = 0; it < 200; ++it) {
      const T mid = T(0.5) * (lo + hi);
      if (mid <= lo || mid >= hi) break;
      T xd[3];
#pragma unroll
      for (int i = 0; i < 3; ++i)
        xd[i] = y[i] + mid * (r2v[i] + (T(1) - mid) * (r3[i] + mid * (r4[i] + (T(1) - mid) *
                                                                             r5[i])));
      const T rd2 = xd[0] * xd[0] + xd[1] * xd[1] + xd[2] * xd[2];
      if (rd2 < r_out * r_out) lo = mid; else hi = mid;
    }
    const T th = T(0.5) * (lo + hi);
    const T al = th, be = th * (T(1) - th), ga = th * th * (T(1) - th),
            de = th * th * (T(1) - th) * (T(1) - th);
    const T dal = T(1), dbe = T(1) - T(2) * th, dga = T(2) * th - T(3) * th * th,
            dde = T(2) * th * (T(1) - th) * (T(1) - th) - T(2) * th * th * (T(1) - th);
    T xe[3], dD[6];
#pragma unroll
    for (int i = 0; i < 6; ++i) {
      dD[i] = dal * r2v[i] + dbe * r3[i] + dga * r4[i] + dde * r5[i];
      if (i < 3) xe[i] = y[i] + al * r2v[i] + be * r3[i] + ga * r4[i] + de * r5[i];
    }
    T s = T(0), cth = T(0);
#pragma unroll
    for (int i = 0; i < 6; ++i) s += ybar_e[i] * dD[i];
#pragma unroll
    for (int i = 0; i < 3; ++i) cth += T(2) * xe[i] * dD[i];
    T yt[6];
#pragma unroll
    for (int i = 0; i < 6; ++i) yt[i] = ybar_e[i] - ((i < 3) ? (s / cth) * T(2) * xe[i] : T(0));
    T r2b[6], r3b[6], r4b[6], r5b[6];
#pragma unroll
    for (int i = 0; i < 6; ++i) {
      r2b[i] = al * yt[i];
      r3b[i] = be * yt[i];
      r4b[i] = ga * yt[i];
      r5b[i] = de * yt[i];
      yb[i] = yt[i];
      kb[0][i] += h * d1 * r5b[i];
      kb[2][i] += h * d3 * r5b[i];
      kb[3][i] += h * d4 * r5b[i];
      kb[4][i] += h * d5 * r5b[i];
      kb[5][i] += h * d6 * r5b[i];
      kb[6][i] += h * d7 * r5b[i];
      r2b[i] += r4b[i];
      kb[6][i] -= h * r4b[i];
      r3b[i] -= r4b[i];
      kb[0][i] += h * r3b[i];
      r2b[i] -= r3b[i];
      ynb[i] = r2b[i];
      yb[i] -= r2b[i];
    }
    vjp<HYB>(c, dm, yn, kb[6], t, qbar);
#pragma unroll
    for (int i = 0; i < 6; ++i) ynb[i] += t[i];
  } else {
#pragma unroll
    for (int i = 0; i < 6; ++i) {
      ynb[i] = ybar[i];
      yb[i] = T(0);
    }
  }
  // yn = y + h sum b_j k_j
#pragma unroll
  for (int i = 0; i < 6; ++i) {
    yb[i] += ynb[i];
    kb[0][i] += h * b1 * ynb[i];
    kb[2][i] += h * b3 * ynb[i];
    kb[3][i] += h * b4 * ynb[i];
    kb[4][i] += h * b5 * ynb[i];
    kb[5][i] += h * b6 * ynb[i];
  }
  // stages, last to first: k_s = f(Y_s), Y_s = y + h sum_j a_sj k_j (Y_s formed
  // when its stage is reached, from the K held in registers)
  const T A[6][5] = {{T(0), T(0), T(0), T(0), T(0)},
                     {T(DP::a21), T(0), T(0), T(0), T(0)},
                     {T(DP::a31), T(DP::a32), T(0), T(0), T(0)},
                     {T(DP::a41), T(DP::a42), T(DP::a43), T(0), T(0)},
                     {T(DP::a51), T(DP::a52), T(DP::a53), T(DP::a54), T(0)},
                     {T(DP::a61), T(DP::a62), T(DP::a63), T(DP::a64), T(DP::a65)}};
#pragma unroll
  for (int s = 5; s >= 0; --s) {
    T Ys[6], Yb[6];
#pragma unroll
    for (int i = 0; i < 6; ++i) {
      T acc = T(0);
#pragma unroll
      for (int j = 0; j < s; ++j) acc += A[s][j] * K[j][i];
      Ys[i] = (s == 0) ? y[i] : y[i] + h * acc;
    }
    vjp<HYB>(c, dm, Ys, kb[s], Yb, qbar);
#pragma unroll
    for (int i = 0; i < 6; ++i) {
      yb[i] += Yb[i];
#pragma unroll
      for (int j = 0; j < s; ++j) kb[j][i] += h * A[s][j] * Yb[i];
    }
  }
#pragma unroll
  for (int i = 0; i < 6; ++i) ybar[i] = yb[i];
}

// K(mu) at a scaled state, in the operation order of flux_kernel_value.
__device__ double flux_K(const double* x, const double* k, double rs, double si, double ci,
                         double kappa, double knorm) {
  const double r = sqrt(x[0] * x[0] + x[1] * x[1] + x[2] * x[2]);
  double n[3];
#pragma unroll
  for (int j = 0; j < 3; ++j) n[j] = x[j] / r;
  const double A = 1.0 - rs / r;
  const double kn = n[0] * k[0] + n[1] * k[1] + n[2] * k[2];
  const double cr = (sqrt(A) - 1.0) * kn;
  double ko[3];
#pragma unroll
  for (int j = 0; j < 3; ++j) ko[j] = k[j] + cr * n[j];
  const double kk = 1.0 / sqrt(ko[0] * ko[0] + ko[1] * ko[1] + ko[2] * ko[2]);
  const double mu = (ko[0] * si + ko[2] * ci) * kk;
  return knorm * exp(kappa * (mu - 1.0));
}

// The functional's integrand at the escape point and its gradient with
// respect to the state and r_s (w and the observer direction held fixed).
__device__ double flux_kernel_value(const AdjParams& P, const double* y, double w, double* ybar,
                                    double* rsbar, double* dmu_dincl, double* Kout) {
  typedef Dual<7> D7;
  D7 x[3], k[3];
#pragma unroll
  for (int j = 0; j < 3; ++j) {
    x[j] = D7::var(y[j], j);
    k[j] = D7::var(y[3 + j], 3 + j);
  }
  const D7 rs = D7::var(P.rs_prop, 6);
  const D7 r = rt_sqrt(x[0] * x[0] + x[1] * x[1] + x[2] * x[2]);
  D7 n[3];
#pragma unroll
  for (int j = 0; j < 3; ++j) n[j] = x[j] / r;
  const D7 A = D7(1.0) - rs / r;
  const D7 kn = n[0] * k[0] + n[1] * k[1] + n[2] * k[2];
  const D7 cr = (rt_sqrt(A) - D7(1.0)) * kn;
  D7 ko[3];
#pragma unroll
  for (int j = 0; j < 3; ++j) ko[j] = k[j] + cr * n[j];
  const D7 kk = rt_rsqrt(ko[0] * ko[0] + ko[1] * ko[1] + ko[2] * ko[2]);
  double si, ci;
  sincos(P.incl, &si, &ci);
  const D7 mu = (ko[0] * D7(si) + ko[2] * D7(ci)) * kk;
  const double K = P.knorm * exp(P.kappa * (mu.v - 1.0));
  *Kout = K;
  const double g = w * K * P.kappa;
#pragma unroll
  for (int j = 0; j < 6; ++j) ybar[j] = g * mu.d[j];
  *rsbar = g * mu.d[6];
  *dmu_dincl = (ko[0].v * ci - ko[2].v * si) * kk.v;
  return w * K;
}

__device__ void store_ck(double* ck, const Lane& L) {
#pragma unroll
  for (int j = 0; j < 6; ++j) ck[j] = L.y[j];
  ck[6] = L.h;
  ck[7] = L.h_resume;
  ck[8] = L.c.sig;
  ck[9] = L.last_rej ? 1.0 : 0.0;
  ck[10] = L.switching ? 1.0 : 0.0;
  ck[11] = (double)L.na;
  ck[12] = (double)L.nr;
}

__device__ void load_ck(const double* ck, Lane& L) {
#pragma unroll
  for (int j = 0; j < 6; ++j) L.y[j] = ck[j];
  L.h = ck[6];
  L.h_resume = ck[7];
  L.c.sig = ck[8];
  L.last_rej = ck[9] != 0.0;
  L.switching = ck[10] != 0.0;
  L.na = (int)ck[11];
  L.nr = (int)ck[12];
  rhs64(L.c, L.y, L.f0);
}

// Records every accepted step of a segment replay, with its stages.
struct RecHook {
  double* seg;
  int nrec, cap;
  bool pend_flip;
  __device__ void on_accept(const Lane& L, const double* y, const double*, const double* k1,
                            const double* k2, const double* k3, const double* k4,
                            const double* k5, const double* k6, const double* k7, double h) {
    if (nrec < cap) {
      double* r = seg + (int64_t)nrec * SEGREC;
#pragma unroll
      for (int j = 0; j < 6; ++j) r[j] = y[j];
      r[6] = h;
      r[7] = L.c.sig;
      r[8] = pend_flip ? (double)FL_FLIP_BEFORE : 0.0;
      double* K = r + SEG_K;
#pragma unroll
      for (int j = 0; j < 6; ++j) {
        K[j] = k1[j];
        K[6 + j] = k2[j];
        K[12 + j] = k3[j];
        K[18 + j] = k4[j];
        K[24 + j] = k5[j];
        K[30 + j] = k6[j];
        K[36 + j] = k7[j];
      }
    }
    pend_flip = false;
    ++nrec;
  }
};

// The trace parameters of the replays (those of the forward run).
__device__ __forceinline__ TraceParams replay_params(const AdjParams& P) {
  TraceParams tp;
  tp.rtol = P.rtol;
  tp.atol = P.atol;
  tp.r_out = P.r_out;
  tp.lambda_max = 0.0;
  tp.r_capture = P.r_capture;
  tp.max_steps = P.max_steps;
  tp.ts = nullptr;
  tp.park = nullptr;
  return tp;
}

// Samples ray i with its parameter tangents (so) and its plain values (sv,
// exactly as the sampling kernel computes them) and sets up the lane exactly
// as the forward trace loads it from the state.  false: no conversion point;
// the ray's outputs are zeroed.
__device__ bool begin_ray(const AdjParams& P, int64_t i, SampOut<Dual<NSAMP_TANGENTS>>& so,
                          SampOut<double>& sv, Lane& L, double& cps, double& sps) {
  const int64_t n = P.n;
  double u[6];
#pragma unroll
  for (int j = 0; j < 6; ++j) u[j] = P.u[j * n + i];
  sample_core(P.sc, u, (double)n, so);
  sample_core(P.scv, u, (double)n, sv);
  P.flags[i] = 0;
  if (!sv.ok || !so.ok) {
    P.F_ray[i] = 0.0;
    for (int k = 0; k < NPARAMS; ++k) P.G_ray[k * n + i] = 0.0;
    P.status[i] = RAY_NO_ROOT;
    return false;
  }
  const double iR = 1.0 / P.R_km, im = 1.0 / P.ma_eV;
#pragma unroll
  for (int j = 0; j < 3; ++j) {
    L.y[j] = (sv.x[j] * P.R_km) * iR;
    L.y[3 + j] = (sv.k[j] * P.ma_eV) * im;
  }
  const double om = 1.0 + sv.delta;
  sincos(sv.psi, &sps, &cps);
  L.R_km = P.R_km;
  L.ma_eV = P.ma_eV;
  L.c.rs = P.rs_prop;
  L.c.cp = P.cp;
  L.c.pa = P.plasma_a;
  L.c.W2 = om * om;
  L.c.iW2 = 1.0 / (om * om);
  L.c.m0 = P.sin_tm * cps;
  L.c.m1 = P.sin_tm * sps;
  L.c.m2 = P.cos_tm;
  L.c.disp = P.dispersion;
  L.c.plasma = P.plasma;
  L.c.sig = gj_side<double>(L.c.m0, L.c.m1, L.c.m2, L.y[0], L.y[1], L.y[2]);
  L.switching = false;
  L.h_resume = 0.0;
  rhs64(L.c, L.y, L.f0);
  L.h = initial_step(L.c, L.y, L.f0, P.rtol, P.atol, 1e30);
  L.lam = 0.0;
  L.na = 0;
  L.nr = 0;
  L.last_rej = false;
  return true;
}

// T: precision of the reverse sweep (the forward replay is FP64 either way).
// Checkpointed recompute: one replay storing a checkpoint every CK accepted
// steps, then segment by segment (last first) a replay of the segment that
// records its steps and the reverse sweep over them.
template <class T, bool HYB = false>
__device__ void adjoint_ray(const AdjParams& P, int64_t i, double* seg, long long* steps) {
  const int64_t n = P.n;
  SampOut<Dual<NSAMP_TANGENTS>> so;
  SampOut<double> sv;
  Lane L;
  double sps, cps;
  if (!begin_ray(P, i, so, sv, L, cps, sps)) return;
  double G[NPARAMS];
  TraceParams tp = replay_params(P);
  // forward replay with a checkpoint every CK accepted steps
  const int64_t c0 = P.ck_off[i];
  const int64_t cmax = P.ck_off[i + 1] - c0;
  double* ck = P.ck + c0 * CKREC;
  int64_t nck = 0;
  if (nck < cmax) store_ck(ck, L);
  ++nck;
  NoHook nh;
  int st;
  for (;;) {
    const int na0 = L.na;
    st = advance(tp, L, nh);
    if (st >= 0) break;
    if (L.na != na0 && L.na % CK == 0) {
      if (nck < cmax) store_ck(ck + nck * CKREC, L);
      ++nck;
    }
  }
  const int na_final = L.na;
  *steps += na_final + L.nr;
  P.status[i] = (uint8_t)st;
  if (nck > cmax) {
    P.flags[i] = 1;   // more steps than the forward pass: no gradient
    if (P.counters) atomicAdd((unsigned long long*)&P.counters[CTR_PROMOTED], 1ull);
    P.F_ray[i] = 0.0;
    for (int k = 0; k < NPARAMS; ++k) P.G_ray[k * n + i] = 0.0;
    return;
  }
  if (st != RAY_ESCAPED) {
    P.F_ray[i] = 0.0;
    for (int k = 0; k < NPARAMS; ++k) P.G_ray[k * n + i] = 0.0;
    return;
  }
  // functional at the escape point
  double ybar[6], qbar[NQ] = {0, 0, 0}, rsb, dmu_di;
  const double w = sv.w;
  double Kv;
  const double Fi = flux_kernel_value(P, L.y, w, ybar, &rsb, &dmu_di, &Kv);
  qbar[Q_RS] += rsb;
  const double dmdth[3] = {P.cos_tm * cps, P.cos_tm * sps, -P.sin_tm};
  T yb[6], ye[6], qb[NQ], dm[3];
#pragma unroll
  for (int j = 0; j < 6; ++j) {
    yb[j] = T(ybar[j]);
    ye[j] = yb[j];
  }
#pragma unroll
  for (int k = 0; k < NQ; ++k) qb[k] = T(qbar[k]);
#pragma unroll
  for (int j = 0; j < 3; ++j) dm[j] = T(dmdth[j]);
  // reverse sweep over the segments
  const int last_seg = (na_final - 1) / CK;
  for (int sgi = last_seg; sgi >= 0; --sgi) {
    load_ck(ck + (int64_t)sgi * CKREC, L);
    const int end_na = (sgi == last_seg) ? na_final : (sgi + 1) * CK;
    RecHook rh;
    rh.seg = seg;
    rh.nrec = 0;
    rh.cap = CK;
    rh.pend_flip = false;
    int st2 = -1;
    while (L.na < end_na) {
      const int na0 = L.na;
      const double sig0 = L.c.sig;
      st2 = advance(tp, L, rh);
      if (L.na == na0) {
        if (L.c.sig != sig0) rh.pend_flip = true;   // switched at the current point
      } else if (st2 < 0 && L.c.sig != sig0 && rh.nrec <= CK) {
        seg[(int64_t)(rh.nrec - 1) * SEGREC + 8] += (double)FL_FLIP_AFTER;
      }
      if (st2 >= 0) break;
    }
    if (st2 >= 0 && rh.nrec >= 1 && rh.nrec <= CK)
      seg[(int64_t)(rh.nrec - 1) * SEGREC + 8] += (double)FL_ESCAPE;
    const int nrec = rh.nrec < CK ? rh.nrec : CK;
    for (int j = nrec - 1; j >= 0; --j) {
      const double* r = seg + (int64_t)j * SEGREC;
      const int fl = (int)r[8];
      RayConst<T> cj = cast_const<T>(L.c);
      cj.sig = T(r[7]);
      T y[6];
#pragma unroll
      for (int q = 0; q < 6; ++q) y[q] = T(r[q]);
      if (fl & FL_FLIP_AFTER) {
        // the branch switched at the end of this step: undo at y_{n+1}
        T yn[6];
        // y_{n+1} is the next record's start, or the next checkpoint's state
        if (j + 1 < nrec) {
#pragma unroll
          for (int q = 0; q < 6; ++q) yn[q] = T(seg[(int64_t)(j + 1) * SEGREC + q]);
        } else {
          const double* nx = ck + (int64_t)(sgi + 1) * CKREC;
#pragma unroll
          for (int q = 0; q < 6; ++q) yn[q] = T(nx[q]);
        }
        saltation(cj, dm, yn, T(r[7]), yb, qb);
      }
      step_adjoint<T, HYB>(cj, dm, y, T(r[6]), r + SEG_K, (fl & FL_ESCAPE) != 0, T(P.r_out),
                           ye, yb, qb);
      if (fl & FL_FLIP_BEFORE) saltation(cj, dm, y, T(-r[7]), yb, qb);
    }
  }
#pragma unroll
  for (int j = 0; j < 6; ++j) ybar[j] = dval(yb[j]);
#pragma unroll
  for (int k = 0; k < NQ; ++k) qbar[k] = dval(qb[k]);
  // assemble dF/dp for this ray
#pragma unroll
  for (int k = 0; k < NSAMP_TANGENTS; ++k) {
    double g = Kv * so.w.d[k];
#pragma unroll
    for (int j = 0; j < 3; ++j) g += ybar[j] * so.x[j].d[k] + ybar[3 + j] * so.k[j].d[k];
    G[k] = g;
  }
  G[PAR_MA] += qbar[Q_CP] * P.dcp_dma;
  G[PAR_B0] += qbar[Q_CP] * P.dcp_dB0;
  G[PAR_THM] += qbar[Q_THM];
  G[PAR_M] += qbar[Q_RS] * P.drsp_dM;
  G[PAR_R] += qbar[Q_RS] * P.drsp_dR;
  G[PAR_INCL] = w * Kv * P.kappa * dmu_di;
  P.F_ray[i] = Fi;
  for (int k = 0; k < NPARAMS; ++k) P.G_ray[k * n + i] = G[k];
}

template <class T, bool HYB = false>
__global__ void __launch_bounds__(64) adjoint_kernel(AdjParams P) {
  const int64_t tid = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  double* seg = P.seg + tid * (int64_t)CK * SEGREC;
  long long steps = 0, rays = 0;
  for (;;) {
    const int64_t i = (int64_t)atomicAdd(P.queue, 1ull);
    if (i >= P.n) break;
    adjoint_ray<T, HYB>(P, i, seg, &steps);
    ++rays;
  }
  if (P.counters) {
    atomicAdd((unsigned long long*)&P.counters[CTR_ACC], (unsigned long long)steps);
    atomicAdd((unsigned long long*)&P.counters[CTR_RAYS], (unsigned long long)rays);
  }
}

// ---------------------------------------------------------------------------
// Full step tape: every accepted step of every ray is held in device memory at
// once (SEGREC doubles a step), so that each ray is replayed once.  Two
// persistent kernels claiming the rays longest first from a global queue: the
// tape kernel replays them in FP64, one attempt per iteration, a warp claiming
// new rays once TAPE_REFILL of its lanes are free, and records every accepted
// step; the sweep kernel walks each ray's records backwards, one step per
// iteration, a lane claiming its next ray as soon as it is free, so that the
// lanes of a warp run the same step adjoint.

constexpr int TAPE_BLOCK = 128;
constexpr int SWEEP_BLOCK = 128;
// a warp of the replay claims new rays once this many of its lanes are free
// (the FP64 forward kernels' default)
constexpr int TAPE_REFILL = 8;

// Samples ray i with its tangents and writes its head record: tangents, dm,
// the ray's constants, the initial state and the weight (one thread per ray,
// ahead of the replay, so that the replay's lanes do not wait on one
// another's dual-number sampling).
__global__ void __launch_bounds__(128) adjoint_sample_kernel(AdjParams P) {
  const int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (i >= P.n) return;
  SampOut<Dual<NSAMP_TANGENTS>> so;
  SampOut<double> sv;
  Lane L;
  double cps, sps;
  double* hd = P.head + i * HEADREC;
  if (!begin_ray(P, i, so, sv, L, cps, sps)) {
    hd[HD_NREC] = -1.0;
    return;
  }
  hd[HD_NREC] = 0.0;
#pragma unroll
  for (int k = 0; k < NSAMP_TANGENTS; ++k) {
#pragma unroll
    for (int j = 0; j < 3; ++j) {
      hd[HD_TAN + 7 * k + j] = so.x[j].d[k];
      hd[HD_TAN + 7 * k + 3 + j] = so.k[j].d[k];
    }
    hd[HD_TAN + 7 * k + 6] = so.w.d[k];
  }
  hd[HD_DM + 0] = P.cos_tm * cps;
  hd[HD_DM + 1] = P.cos_tm * sps;
  hd[HD_DM + 2] = -P.sin_tm;
  hd[HD_W2] = L.c.W2;
  hd[HD_IW2] = L.c.iW2;
  hd[HD_M + 0] = L.c.m0;
  hd[HD_M + 1] = L.c.m1;
  hd[HD_M + 2] = L.c.m2;
#pragma unroll
  for (int j = 0; j < 6; ++j) hd[HD_Y0 + j] = L.y[j];
  hd[HD_W] = sv.w;
}

// The lane of ray i from its head record, exactly as begin_ray leaves it.
__device__ __forceinline__ void tape_load(const AdjParams& P, const double* hd, Lane& L) {
#pragma unroll
  for (int j = 0; j < 6; ++j) L.y[j] = hd[HD_Y0 + j];
  L.R_km = P.R_km;
  L.ma_eV = P.ma_eV;
  L.c.rs = P.rs_prop;
  L.c.cp = P.cp;
  L.c.pa = P.plasma_a;
  L.c.W2 = hd[HD_W2];
  L.c.iW2 = hd[HD_IW2];
  L.c.m0 = hd[HD_M + 0];
  L.c.m1 = hd[HD_M + 1];
  L.c.m2 = hd[HD_M + 2];
  L.c.disp = P.dispersion;
  L.c.plasma = P.plasma;
  L.c.sig = gj_side<double>(L.c.m0, L.c.m1, L.c.m2, L.y[0], L.y[1], L.y[2]);
  L.switching = false;
  L.h_resume = 0.0;
  rhs64(L.c, L.y, L.f0);
  L.h = initial_step(L.c, L.y, L.f0, P.rtol, P.atol, 1e30);
  L.lam = 0.0;
  L.na = 0;
  L.nr = 0;
  L.last_rej = false;
}

// The end of ray i's replay: status, the escape flag and the final state on
// the tape, the functional and its seed adjoint in the head record.
__device__ __noinline__ void tape_finish(const AdjParams& P, int64_t i, const Lane& L,
                                         const RecHook& rh, double w, int st) {
  const int64_t n = P.n;
  double* hd = P.head + i * HEADREC;
  P.status[i] = (uint8_t)st;
  const bool left_out = rh.nrec > rh.cap;
  if (left_out || st != RAY_ESCAPED) {
    if (left_out) {
      P.flags[i] = 1;   // more steps than the forward pass: no gradient
      if (P.counters) atomicAdd((unsigned long long*)&P.counters[CTR_PROMOTED], 1ull);
    }
    hd[HD_NREC] = -1.0;
    P.F_ray[i] = 0.0;
    for (int k = 0; k < NPARAMS; ++k) P.G_ray[k * n + i] = 0.0;
    return;
  }
  if (rh.nrec >= 1) rh.seg[(int64_t)(rh.nrec - 1) * SEGREC + 8] += (double)FL_ESCAPE;
#pragma unroll
  for (int j = 0; j < 6; ++j) rh.seg[(int64_t)rh.nrec * SEGREC + j] = L.y[j];
  double ybar[6], rsb, dmu_di, Kv;
  const double Fi = flux_kernel_value(P, L.y, w, ybar, &rsb, &dmu_di, &Kv);
#pragma unroll
  for (int j = 0; j < 6; ++j) hd[HD_YBAR + j] = ybar[j];
  hd[HD_RSBAR] = rsb;
  hd[HD_K] = Kv;
  hd[HD_NREC] = (double)rh.nrec;
  P.F_ray[i] = Fi;
  P.G_ray[PAR_INCL * n + i] = w * Kv * P.kappa * dmu_di;
}

__global__ void __launch_bounds__(TAPE_BLOCK) adjoint_tape_kernel(AdjParams P) {
  constexpr unsigned FULL = 0xffffffffu;
  const TraceParams tp = replay_params(P);
  Lane L;
  RecHook rh;
  rh.seg = nullptr;
  rh.nrec = rh.cap = 0;
  rh.pend_flip = false;
  double w = 0.0;
  int64_t item = -1;
  ClaimChunk ch;
  long long steps = 0, rays = 0;
  for (;;) {
    claim_items(P.queue, P.n, TAPE_REFILL, 1, item, ch, [&](int64_t e) -> int64_t {
      const int64_t i = P.order[e];
      ++rays;
      const double* hd = P.head + i * HEADREC;
      if (hd[HD_NREC] < 0.0) return -1;   // no conversion point
      tape_load(P, hd, L);
      w = hd[HD_W];
      rh.seg = P.tape + P.tape_off[i] * SEGREC;
      rh.cap = (int)(P.tape_off[i + 1] - P.tape_off[i] - 1);
      rh.nrec = 0;
      rh.pend_flip = false;
      return i;
    });
    if (__ballot_sync(FULL, item != -2) == 0) break;
    if (item >= 0) {
      const int na0 = L.na;
      const double sig0 = L.c.sig;
      const int st = advance(tp, L, rh);
      if (L.na == na0) {
        if (L.c.sig != sig0) rh.pend_flip = true;   // switched at the current point
      } else if (st < 0 && L.c.sig != sig0 && rh.nrec <= rh.cap) {
        rh.seg[(int64_t)(rh.nrec - 1) * SEGREC + 8] += (double)FL_FLIP_AFTER;
      }
      if (st >= 0) {
        tape_finish(P, item, L, rh, w, st);
        steps += L.na + L.nr;
        item = -1;
      }
    }
  }
  if (P.counters) {
    atomicAdd((unsigned long long*)&P.counters[CTR_ACC], (unsigned long long)steps);
    atomicAdd((unsigned long long*)&P.counters[CTR_RAYS], (unsigned long long)rays);
  }
}

// dF/dp of ray i from the adjoint at its initial state and the q-adjoints.
template <class T>
__device__ __noinline__ void sweep_finish(const AdjParams& P, int64_t i, const T* yb,
                                          const T* qb) {
  const int64_t n = P.n;
  const double* hd = P.head + i * HEADREC;
  double ybar[6], qbar[NQ], G[NSAMP_TANGENTS];
#pragma unroll
  for (int j = 0; j < 6; ++j) ybar[j] = dval(yb[j]);
#pragma unroll
  for (int k = 0; k < NQ; ++k) qbar[k] = dval(qb[k]);
  const double Kv = hd[HD_K];
#pragma unroll
  for (int k = 0; k < NSAMP_TANGENTS; ++k) {
    const double* tk = hd + HD_TAN + 7 * k;
    double g = Kv * tk[6];
#pragma unroll
    for (int j = 0; j < 3; ++j) g += ybar[j] * tk[j] + ybar[3 + j] * tk[3 + j];
    G[k] = g;
  }
  G[PAR_MA] += qbar[Q_CP] * P.dcp_dma;
  G[PAR_B0] += qbar[Q_CP] * P.dcp_dB0;
  G[PAR_THM] += qbar[Q_THM];
  G[PAR_M] += qbar[Q_RS] * P.drsp_dM;
  G[PAR_R] += qbar[Q_RS] * P.drsp_dR;
#pragma unroll
  for (int k = 0; k < NSAMP_TANGENTS; ++k) P.G_ray[k * n + i] = G[k];
}

template <class T, bool HYB = false>
__global__ void __launch_bounds__(SWEEP_BLOCK) adjoint_sweep_kernel(AdjParams P) {
  constexpr unsigned FULL = 0xffffffffu;
  int64_t item = -1;
  ClaimChunk ch;
  int j = -1;
  const double* base = nullptr;
  T yb[6], ye[6], qb[NQ], dm[3];
  RayConst<T> c;
  c.rs = T(P.rs_prop);
  c.cp = T(P.cp);
  c.pa = T(P.plasma_a);
  c.disp = P.dispersion;
  c.plasma = P.plasma;
  for (;;) {
    claim_items(P.queue, P.n, 1, 1, item, ch, [&](int64_t e) -> int64_t {
      const int64_t i = P.order[e];
      const double* hd = P.head + i * HEADREC;
      const int nrec = (int)hd[HD_NREC];
      if (nrec < 0) return -1;
#pragma unroll
      for (int q = 0; q < 6; ++q) {
        yb[q] = T(hd[HD_YBAR + q]);
        ye[q] = yb[q];
      }
      qb[Q_RS] = T(hd[HD_RSBAR]);
      qb[Q_CP] = T(0);
      qb[Q_THM] = T(0);
#pragma unroll
      for (int q = 0; q < 3; ++q) dm[q] = T(hd[HD_DM + q]);
      c.W2 = T(hd[HD_W2]);
      c.iW2 = T(hd[HD_IW2]);
      c.m0 = T(hd[HD_M + 0]);
      c.m1 = T(hd[HD_M + 1]);
      c.m2 = T(hd[HD_M + 2]);
      base = P.tape + P.tape_off[i] * SEGREC;
      j = nrec - 1;
      return i;
    });
    if (__ballot_sync(FULL, item != -2) == 0) break;
    if (item >= 0) {
      if (j >= 0) {
        const double* r = base + (int64_t)j * SEGREC;
        const int fl = (int)r[8];
        RayConst<T> cj = c;
        cj.sig = T(r[7]);
        T y[6];
#pragma unroll
        for (int q = 0; q < 6; ++q) y[q] = T(r[q]);
        if (fl & FL_FLIP_AFTER) {
          // the branch switched at the end of this step: undo at y_{n+1}, the
          // next record's start (or the ray's final state)
          T yn[6];
#pragma unroll
          for (int q = 0; q < 6; ++q) yn[q] = T(r[SEGREC + q]);
          saltation(cj, dm, yn, T(r[7]), yb, qb);
        }
        step_adjoint<T, HYB>(cj, dm, y, T(r[6]), r + SEG_K, (fl & FL_ESCAPE) != 0, T(P.r_out),
                             ye, yb, qb);
        if (fl & FL_FLIP_BEFORE) saltation(cj, dm, y, T(-r[7]), yb, qb);
        --j;
      }
      if (j < 0) {
        sweep_finish(P, item, yb, qb);
        item = -1;
      }
    }
  }
}

// Longest-first order of the rays by their forward step counts: 32 buckets
// of floor(log2(nacc + 1)), counted, scanned and scattered (the order within
// a bucket is that of the atomics; no result depends on it).
__device__ __forceinline__ int len_bucket(int32_t na) {
  return __clz((unsigned)(na > 0 ? na : 0) + 1u);
}

__global__ void order_count_kernel(const int32_t* nacc, int64_t n, unsigned long long* bucket) {
  __shared__ unsigned int cnt[32];
  if (threadIdx.x < 32) cnt[threadIdx.x] = 0u;
  __syncthreads();
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n;
       i += (int64_t)gridDim.x * blockDim.x)
    atomicAdd(&cnt[len_bucket(nacc[i])], 1u);
  __syncthreads();
  if (threadIdx.x < 32 && cnt[threadIdx.x])
    atomicAdd(&bucket[threadIdx.x], (unsigned long long)cnt[threadIdx.x]);
}

__global__ void order_scan_kernel(unsigned long long* bucket) {
  if (threadIdx.x != 0 || blockIdx.x != 0) return;
  unsigned long long acc = 0;
  for (int b = 0; b < 32; ++b) {
    const unsigned long long v = bucket[b];
    bucket[b] = acc;
    acc += v;
  }
}

__global__ void order_scatter_kernel(const int32_t* nacc, int64_t n, unsigned long long* bucket,
                                     int64_t* order) {
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n;
       i += (int64_t)gridDim.x * blockDim.x) {
    const unsigned long long pos = atomicAdd(&bucket[len_bucket(nacc[i])], 1ull);
    order[pos] = i;
  }
}

// Tape offsets: an exclusive prefix sum of tape_slots(nacc) (one block; fixed
// order).
__global__ void tape_offsets_kernel(const int32_t* nacc, int64_t n, int64_t* off) {
  __shared__ int64_t part[1024];
  const int t = threadIdx.x, T = blockDim.x;
  const int64_t chunk = (n + T - 1) / T;
  const int64_t b = (int64_t)t * chunk, e = (b + chunk < n) ? b + chunk : n;
  int64_t s = 0;
  for (int64_t i = b; i < e; ++i) s += tape_slots(nacc[i]);
  part[t] = s;
  __syncthreads();
  if (t == 0) {
    int64_t acc = 0;
    for (int q = 0; q < T; ++q) {
      const int64_t v = part[q];
      part[q] = acc;
      acc += v;
    }
    off[n] = acc;
  }
  __syncthreads();
  int64_t acc = part[t];
  for (int64_t i = b; i < e; ++i) {
    off[i] = acc;
    acc += tape_slots(nacc[i]);
  }
}

// The functional over already traced rays: F_ray[i] = w_i K(mu_i).
__global__ void flux_value_kernel(const StarDev* sd, int64_t n, const double* state,
                                  const double* weight, const uint8_t* status, double incl,
                                  double kappa, double knorm, double* F_ray) {
  const StarDev& s = *sd;
  double si, ci;
  sincos(incl, &si, &ci);
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n;
       i += (int64_t)gridDim.x * blockDim.x) {
    if (status[i] != RAY_ESCAPED) {
      F_ray[i] = 0.0;
      continue;
    }
    const double iR = 1.0 / s.R_km, im = 1.0 / s.ma_eV;
    double x[3], k[3];
#pragma unroll
    for (int j = 0; j < 3; ++j) {
      x[j] = state[j * n + i] * iR;
      k[j] = state[(3 + j) * n + i] * im;
    }
    F_ray[i] = weight[i] * flux_K(x, k, s.rs_prop, si, ci, kappa, knorm);
  }
}

// Deterministic sums of rows of an (nrow x n) array: one block per row, each
// thread a strided partial sum in a fixed order, then a fixed-shape tree.
__global__ void row_sums_kernel(const double* a, int64_t n, double* out) {
  __shared__ double sh[256];
  const int row = blockIdx.x;
  double s = 0.0;
  for (int64_t i = threadIdx.x; i < n; i += blockDim.x) s += a[row * n + i];
  sh[threadIdx.x] = s;
  __syncthreads();
  for (int w = blockDim.x / 2; w > 0; w >>= 1) {
    if ((int)threadIdx.x < w) sh[threadIdx.x] += sh[threadIdx.x + w];
    __syncthreads();
  }
  if (threadIdx.x == 0) out[row] = sh[0];
}

// Checkpoint counts per ray from the forward step counts, and their exclusive
// prefix sum (one block; fixed order).
__global__ void ck_offsets_kernel(const int32_t* nacc, int64_t n, int64_t* off) {
  __shared__ int64_t part[1024];
  const int t = threadIdx.x, T = blockDim.x;
  const int64_t chunk = (n + T - 1) / T;
  const int64_t b = (int64_t)t * chunk, e = (b + chunk < n) ? b + chunk : n;
  int64_t s = 0;
  for (int64_t i = b; i < e; ++i) s += (int64_t)(nacc[i] / CK) + 2;
  part[t] = s;
  __syncthreads();
  if (t == 0) {
    int64_t acc = 0;
    for (int q = 0; q < T; ++q) {
      const int64_t v = part[q];
      part[q] = acc;
      acc += v;
    }
    off[n] = acc;
  }
  __syncthreads();
  int64_t acc = part[t];
  for (int64_t i = b; i < e; ++i) {
    off[i] = acc;
    acc += (int64_t)(nacc[i] / CK) + 2;
  }
}

}  // namespace

cudaError_t launch_flux_value(const StarDev* d_star, int64_t n, const double* state,
                              const double* weight, const uint8_t* status, double incl,
                              double kappa, double knorm, double* F_ray, double* F_total,
                              cudaStream_t stream) {
  if (n <= 0) return cudaSuccess;
  int dev = 0, nsm = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return e;
  e = cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev);
  if (e != cudaSuccess) return e;
  int64_t grid = (n + 255) / 256;
  if (grid > (int64_t)nsm * 8) grid = (int64_t)nsm * 8;
  flux_value_kernel<<<(unsigned)grid, 256, 0, stream>>>(d_star, n, state, weight, status, incl,
                                                        kappa, knorm, F_ray);
  e = cudaGetLastError();
  if (e != cudaSuccess) return e;
  row_sums_kernel<<<1, 256, 0, stream>>>(F_ray, n, F_total);
  return cudaGetLastError();
}

cudaError_t launch_ck_offsets(const int32_t* nacc, int64_t n, int64_t* off, cudaStream_t stream) {
  ck_offsets_kernel<<<1, 1024, 0, stream>>>(nacc, n, off);
  return cudaGetLastError();
}

cudaError_t adjoint_grid(int prec, int* grid, int* block) {
  int dev = 0, nsm = 0, occ = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return e;
  e = cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev);
  if (e != cudaSuccess) return e;
  *block = 64;
  e = (prec == PREC_MIXED)
          ? cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, adjoint_kernel<double, true>,
                                                          *block, 0)
      : (prec == PREC_DF)
          ? cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, adjoint_kernel<DF>, *block, 0)
          : cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, adjoint_kernel<double>, *block, 0);
  if (e != cudaSuccess) return e;
  *grid = nsm * (occ > 0 ? occ : 1);
  return cudaSuccess;
}

static AdjParams adj_params(const AdjLaunch& a) {
  AdjParams P;
  P.sc = a.sc;
  {
    const auto& d = a.sc;
    SampConst<double>& v = P.scv;
    v.rs = d.rs.v;
    v.cp = d.cp.v;
    v.sin_tm = d.sin_tm.v;
    v.cos_tm = d.cos_tm.v;
    v.B0_eV2 = d.B0_eV2.v;
    v.R_eV = d.R_eV.v;
    v.n_inf = d.n_inf.v;
    v.ma_eV = d.ma_eV.v;
    v.v0 = d.v0;
    v.psi_fixed = d.psi_fixed;
    v.plasma_a = d.plasma_a;
    v.rlc = d.rlc;
    v.g_eV = d.g_eV;
    v.w_unit = d.w_unit;
    v.disp = d.disp;
    v.plasma = d.plasma;
    v.fa_model = d.fa_model;
    v.phase_mode = d.phase_mode;
    v.weight_mode = d.weight_mode;
    v.per_cm3 = d.per_cm3;
  }
  P.R_km = a.star->R_km;
  P.ma_eV = a.star->ma_eV;
  P.rs_prop = a.star->rs_prop;
  P.cp = a.star->cp;
  P.plasma_a = a.star->plasma_a;
  P.cos_tm = a.star->cos_tm;
  P.sin_tm = a.star->sin_tm;
  P.dispersion = a.star->dispersion;
  P.plasma = a.star->plasma;
  P.drsp_dM = a.drsp_dM;
  P.drsp_dR = a.drsp_dR;
  P.dcp_dma = a.dcp_dma;
  P.dcp_dB0 = a.dcp_dB0;
  P.incl = a.incl;
  P.kappa = a.kappa;
  P.knorm = a.knorm;
  P.rtol = a.rtol;
  P.atol = a.atol;
  P.r_out = a.r_out;
  P.r_capture = a.r_capture;
  P.max_steps = a.max_steps;
  P.n = a.n;
  P.u = a.u;
  P.ck_off = a.ck_off;
  P.ck = a.ck;
  P.seg = a.seg;
  P.F_ray = a.F_ray;
  P.G_ray = a.G_ray;
  P.status = a.status;
  P.flags = a.flags;
  P.counters = a.counters;
  P.queue = a.queue;
  P.tape_off = a.tape_off;
  P.tape = a.tape;
  P.head = a.head;
  P.order = a.order;
  return P;
}

// dF/dp and F: deterministic sums of the per-ray terms.
static cudaError_t launch_sums(const AdjLaunch& a, cudaStream_t stream) {
  row_sums_kernel<<<NPARAMS, 256, 0, stream>>>(a.G_ray, a.n, a.grad);
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return e;
  row_sums_kernel<<<1, 256, 0, stream>>>(a.F_ray, a.n, a.F);
  return cudaGetLastError();
}

cudaError_t launch_adjoint(const AdjLaunch& a, cudaStream_t stream) {
  const AdjParams P = adj_params(a);
  cudaError_t e = cudaMemsetAsync(a.queue, 0, sizeof(unsigned long long), stream);
  if (e != cudaSuccess) return e;
  if (a.prec == PREC_MIXED)
    adjoint_kernel<double, true><<<a.grid, a.block, 0, stream>>>(P);
  else if (a.prec == PREC_DF)
    adjoint_kernel<DF><<<a.grid, a.block, 0, stream>>>(P);
  else
    adjoint_kernel<double><<<a.grid, a.block, 0, stream>>>(P);
  e = cudaGetLastError();
  if (e != cudaSuccess) return e;
  return launch_sums(a, stream);
}

cudaError_t launch_tape_offsets(const int32_t* nacc, int64_t n, int64_t* off,
                                cudaStream_t stream) {
  tape_offsets_kernel<<<1, 1024, 0, stream>>>(nacc, n, off);
  return cudaGetLastError();
}

// One resident grid of a persistent kernel: every SM times its occupancy.
template <class K>
static cudaError_t persistent_grid(K kernel, int block, int* grid) {
  int dev = 0, nsm = 0, occ = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return e;
  e = cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev);
  if (e != cudaSuccess) return e;
  e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, kernel, block, 0);
  if (e != cudaSuccess) return e;
  *grid = nsm * (occ > 0 ? occ : 1);
  return cudaSuccess;
}

template <class T, bool HYB = false>
static cudaError_t launch_sweep(const AdjParams& P, cudaStream_t stream) {
  int grid = 0;
  cudaError_t e = persistent_grid(adjoint_sweep_kernel<T, HYB>, SWEEP_BLOCK, &grid);
  if (e != cudaSuccess) return e;
  adjoint_sweep_kernel<T, HYB><<<grid, SWEEP_BLOCK, 0, stream>>>(P);
  return cudaGetLastError();
}

cudaError_t launch_adjoint_tape(const AdjLaunch& a, cudaStream_t stream) {
  const AdjParams P = adj_params(a);
  int dev = 0, nsm = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return e;
  e = cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev);
  if (e != cudaSuccess) return e;
  // longest first
  int64_t og = (a.n + 255) / 256;
  if (og > (int64_t)nsm * 4) og = (int64_t)nsm * 4;
  if ((e = cudaMemsetAsync(a.bucket, 0, 32 * sizeof(unsigned long long), stream)) != cudaSuccess)
    return e;
  order_count_kernel<<<(unsigned)og, 256, 0, stream>>>(a.nacc, a.n, a.bucket);
  order_scan_kernel<<<1, 32, 0, stream>>>(a.bucket);
  order_scatter_kernel<<<(unsigned)og, 256, 0, stream>>>(a.nacc, a.n, a.bucket, a.order);
  if ((e = cudaGetLastError()) != cudaSuccess) return e;
  // sampling with tangents, one thread per ray
  adjoint_sample_kernel<<<(unsigned)((a.n + 127) / 128), 128, 0, stream>>>(P);
  if ((e = cudaGetLastError()) != cudaSuccess) return e;
  // the replay onto the tape
  int grid = 0;
  if ((e = persistent_grid(adjoint_tape_kernel, TAPE_BLOCK, &grid)) != cudaSuccess) return e;
  if ((e = cudaMemsetAsync(a.queue, 0, sizeof(unsigned long long), stream)) != cudaSuccess)
    return e;
  adjoint_tape_kernel<<<grid, TAPE_BLOCK, 0, stream>>>(P);
  if ((e = cudaGetLastError()) != cudaSuccess) return e;
  // the reverse sweep
  if ((e = cudaMemsetAsync(a.queue, 0, sizeof(unsigned long long), stream)) != cudaSuccess)
    return e;
  if (a.prec == PREC_MIXED)
    e = launch_sweep<double, true>(P, stream);
  else if (a.prec == PREC_DF)
    e = launch_sweep<DF>(P, stream);
  else
    e = launch_sweep<double>(P, stream);
  if (e != cudaSuccess) return e;
  return launch_sums(a, stream);
}

}  // namespace rtk
