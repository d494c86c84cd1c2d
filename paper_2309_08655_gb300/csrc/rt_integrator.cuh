// The FP64 Dormand-Prince 5(4) integrator of Hamilton's equations (Eq.
// Hamilton) shared by the forward, backward and adjoint kernels: the lane
// state of one ray, the step-size controller, and one step attempt with the
// null-cone branch switching, the step-reach bound and the escape event.
#pragma once
#include <cuda_runtime.h>
#include <stdint.h>

#include "rt_device.cuh"
#include "rt_internal.h"

namespace rtk {
namespace {

constexpr unsigned FULL = 0xffffffffu;

__device__ __forceinline__ void rhs64(const RayConst<double>& c, const double* y, double* f) {
  ham_rhs<double>(c, y[0], y[1], y[2], y[3], y[4], y[5], f[0], f[1], f[2], f[3], f[4], f[5]);
}

// err^(-1/5) to within an ulp or two: a single-precision estimate refined by
// two Newton steps on y^-5 = err, y <- y (6 - err y^5) / 5 (quadratic
// convergence: 1e-7, 1e-14, rounding).  Used where the result is clamped to
// [0.2, 5] after the factor 0.9, i.e. for err in [1.9e-4, 1.9e3].
__device__ __forceinline__ double pow_m1_5(double err) {
  double y = (double)exp2f(-0.2f * log2f((float)err));
#pragma unroll
  for (int it = 0; it < 2; ++it) {
    const double y2 = y * y;
    y = y * (1.2 - 0.2 * err * (y2 * y2 * y));
  }
  return y;
}

__device__ __forceinline__ double step_factor(double err, bool accepted, bool last_rej) {
  // outside [1e-6, 1e6] the clamp below decides: 0.9 err^-0.2 > 5 or < 0.2
  double fac = (err > 1e6) ? 0.0 : (err >= 1e-6) ? 0.9 * pow_m1_5(err) : 5.0;
  fac = fmin(5.0, fmax(0.2, fac));
  if (!accepted || last_rej) fac = fmin(fac, 1.0);
  return fac;
}

// Hairer's two-evaluation initial step (order 5).
__device__ double initial_step(const RayConst<double>& c, const double* y0, const double* f0,
                               double rtol, double atol, double hmax) {
  double dnf = 0.0, dny = 0.0;
#pragma unroll
  for (int i = 0; i < 6; ++i) {
    const double sk = atol + rtol * fabs(y0[i]);
    dnf += (f0[i] / sk) * (f0[i] / sk);
    dny += (y0[i] / sk) * (y0[i] / sk);
  }
  double h = (dnf <= 1e-10 || dny <= 1e-10) ? 1e-6 : sqrt(dny / dnf) * 0.01;
  h = fmin(h, hmax);
  double y1[6], f1[6];
#pragma unroll
  for (int i = 0; i < 6; ++i) y1[i] = y0[i] + h * f0[i];
  rhs64(c, y1, f1);
  double der2 = 0.0;
#pragma unroll
  for (int i = 0; i < 6; ++i) {
    const double sk = atol + rtol * fabs(y0[i]);
    der2 += ((f1[i] - f0[i]) / sk) * ((f1[i] - f0[i]) / sk);
  }
  der2 = sqrt(der2) / h;
  const double der12 = fmax(fabs(der2), sqrt(dnf));
  const double h1 = (der12 <= 1e-15) ? fmax(1e-6, h * 1e-3) : pow(0.01 / der12, 0.2);
  return fmin(fmin(100.0 * h, h1), hmax);
}

struct Lane {
  RayConst<double> c;
  double y[6], f0[6];
  double h, lam;
  int na, nr;
  bool last_rej;
  bool switching;      // the current attempt ends just past a null-cone crossing
  double h_resume;     // step size to resume with after that crossing
  double R_km, ma_eV;
};

// The Goldreich-Julian density |2 Omega . B / e| has a kink on the null cone
// Omega . B = 0 (Eq. GJDensity): dk/dlambda jumps there, which an embedded
// error estimate cannot resolve inside a step.  Each step integrates the
// smooth continuation of the side it starts on (c.sig); when an accepted step
// ends on the other side, the crossing is located on the continuous extension,
// the step is redone to end just past it, and the side is switched there.
constexpr double SWITCH_MIN_FRACTION = 1e-6;
constexpr double SWITCH_OVERSHOOT = 1e-10;

// Squared angular distance of ray i's start point from the Goldreich-Julian
// null cone F = 3 n_z (m.n) - m_z = 0, (F / |grad_n F|)^2 (the gradient on
// the unit sphere); 1e300 for the other plasmas.  Rays guided along the cone for
// thousands of steps start within 1e-2 rad of it.
__device__ __forceinline__ double cone_dist2(const StarDev& s, const double* state, int64_t n,
                                             int64_t i) {
  if (s.plasma != PLASMA_GJ) return 1e300;
  const double x0 = state[i], x1 = state[n + i], x2 = state[2 * n + i];
  double sp, cpsi;
  sincos(state[7 * n + i], &sp, &cpsi);
  const double m0 = s.sin_tm * cpsi, m1 = s.sin_tm * sp, m2 = s.cos_tm;
  const double ir = rsqrt(x0 * x0 + x1 * x1 + x2 * x2);
  const double n0 = x0 * ir, n1 = x1 * ir, n2 = x2 * ir;
  const double mu = m0 * n0 + m1 * n1 + m2 * n2;
  const double F = 3.0 * n2 * mu - m2;
  // grad_n F = 3 (mu e_z + n_z m) minus its radial part 6 mu n_z n
  const double c = 6.0 * mu * n2;
  const double g0 = 3.0 * n2 * m0 - c * n0, g1 = 3.0 * n2 * m1 - c * n1,
               g2 = 3.0 * (mu + n2 * m2) - c * n2;
  return (F * F) / (g0 * g0 + g1 * g1 + g2 * g2);
}

// Cost-ordered claims and finished rays.  A ray finished in one pass has had
// its state overwritten, and the cost bucket of its new state may match a
// later pass.  Stores therefore write the state, fence, then the status
// (status_after_state), and a claim that read the state for the bucket
// re-reads the status after a fence (status_still): a claim that saw any of
// the new state sees the ray finished.
__device__ __forceinline__ void status_after_state(const TraceParams& p, int64_t i, int st) {
  __threadfence();
  p.status[i] = (uint8_t)st;
}
__device__ __forceinline__ bool status_still(const TraceParams& p, int64_t i, int want) {
  __threadfence();
  return *(volatile const uint8_t*)(p.status + i) == want;
}

// Cost bucket for the cost-ordered claim (TraceParams::order): 0 for a start
// within 1e-3 rad of the null cone, 1 within 1e-2 rad, 2 otherwise.
__device__ __forceinline__ int cost_bucket(const StarDev& s, const double* state, int64_t n,
                                           int64_t i) {
  const double d2 = cone_dist2(s, state, n, i);
  return (d2 < 1e-6) ? 0 : (d2 < 1e-4) ? 1 : 2;
}

// Observer of accepted steps (forward tracing needs none).
struct NoHook {
  __device__ __forceinline__ void on_accept(const Lane&, const double*, const double*,
                                            const double*, const double*, const double*,
                                            const double*, const double*, const double*,
                                            const double*, double) {}
};

// The last th in [0, 1] on the non-negative side of side_val, given
// side_val(0) = flo >= 0 > fhi = side_val(1): Illinois (regula falsi that
// halves the retained end's value), with a bisection step whenever the
// bracket did not halve over two steps, run to the last representable th.
// Returns lo (side_val >= 0); *hi_out the first th past it.
// T is the type of th and of the values (double, or float in the mixed
// kernel); [lo, hi] the starting bracket.
template <class S, class T>
__device__ __forceinline__ T last_nonneg(const S& side_val, T flo, T fhi, T* hi_out, T lo = T(0),
                                         T hi = T(1)) {
  int last = 0;
  T width = hi - lo;
  for (int it = 0; it < 200; ++it) {
    T mid = (lo * fhi - hi * flo) / (fhi - flo);
    if ((it & 1) && hi - lo > T(0.5) * width) mid = T(0.5) * (lo + hi);
    if (!(mid > lo && mid < hi)) mid = T(0.5) * (lo + hi);
    if (mid <= lo || mid >= hi) break;
    if (it & 1) width = hi - lo;
    const T fm = side_val(mid);
    if (fm >= T(0)) {
      lo = mid;
      flo = fm;
      if (last > 0) fhi *= T(0.5);
      last = 1;
    } else {
      hi = mid;
      fhi = fm;
      if (last < 0) flo *= T(0.5);
      last = -1;
    }
  }
  *hi_out = hi;
  return lo;
}

// Plain Illinois on the bracket [lo, hi] (side(lo) = flo >= 0 > fhi =
// side(hi)), updated in place, until it is at most tol x hi wide, stops
// shrinking, or maxit evaluations were spent.  Superlinear for a simple root;
// no bisection steps (the caller finishes with last_nonneg if needed).
template <class S, class T>
__device__ __forceinline__ void illinois(const S& side, T& lo, T& hi, T& flo, T& fhi, T tol,
                                         int maxit) {
  int last = 0;
  for (int it = 0; it < maxit && hi - lo > tol * hi; ++it) {
    T mid = (lo * fhi - hi * flo) / (fhi - flo);
    if (!(mid > lo && mid < hi)) mid = T(0.5) * (lo + hi);
    if (mid <= lo || mid >= hi) break;
    const T fm = side(mid);
    if (fm >= T(0)) {
      lo = mid;
      flo = fm;
      if (last > 0) fhi *= T(0.5);
      last = 1;
    } else {
      hi = mid;
      fhi = fm;
      if (last < 0) flo *= T(0.5);
      last = -1;
    }
  }
}

// Event location on the continuous extension: the last th in [0, 1] on the
// non-negative side of a function given in FP64 (f64) and, to FP32 rounding,
// by a cheap FP32 model (f32), with f64(0) = flo >= 0 > fhi = f64(1).  The FP32
// model's root (plain Illinois to 2^-22 relative) is widened by SEED_WIDEN on
// each side; FP64 values at the two ends confirm that the root lies inside
// (else the part of [0, 1] left or right of it holds one), and FP64 Illinois
// narrows that bracket to SEED_TOL64 relative, far below the 1e-10 relative
// overshoot of a switch and below the rounding of an escape point.  About six
// FP64 evaluations where bisection-guarded Illinois from [0, 1] to the last
// bit takes twenty or more.  Returns lo; *hi_out the end past it.
constexpr float SEED_TOL32 = 0x1p-22f;
constexpr double SEED_WIDEN = 0x1p-16;
constexpr double SEED_TOL64 = 0x1p-44;
template <class S64, class S32>
__device__ __forceinline__ double last_nonneg_seeded(const S64& f64, const S32& f32, double flo,
                                                     double fhi, double* hi_out) {
  float l = 0.0f, u = 1.0f, fl = (float)flo, fu = (float)fhi;
  if (!(fl >= 0.0f)) fl = 0.0f;
  if (!(fu < 0.0f)) fu = -1e-30f;
  illinois(f32, l, u, fl, fu, SEED_TOL32, 40);
  double lo = 0.0, hi = 1.0;
  const double a = fmax(0.0, (double)l - SEED_WIDEN), b = fmin(1.0, (double)u + SEED_WIDEN);
  const double fa = (a > 0.0) ? f64(a) : flo;
  if (fa < 0.0) {
    hi = a;                                        // the root lies left of the FP32 bracket
    fhi = fa;
  } else {
    lo = a;
    flo = fa;
    const double fb = (b < 1.0) ? f64(b) : fhi;
    if (fb >= 0.0) {
      lo = b;                                      // right of it
      flo = fb;
    } else {
      hi = b;
      fhi = fb;
    }
  }
  illinois(f64, lo, hi, flo, fhi, SEED_TOL64, 40);
  if (hi - lo > SEED_TOL64 * hi) return last_nonneg(f64, flo, fhi, hi_out, lo, hi);
  *hi_out = hi;
  return lo;
}

// FP32 model of the null-cone side function sig F(x(th)), F = 3 z (m.x) -
// m_z |x|^2, along the continuous extension x(th) = y + d(th), d(th) =
// th (r2 + (1 - th) (r3 + th (r4 + (1 - th) r5))): F(y + d) = F0 + gF.d +
// 3 d_z (m.d) - m_z |d|^2 with F0 = F(y) from FP64 and gF = grad F(y).
struct ConeModel32 {
  float sg, F0, m0, m1, m2, gF[3], r2[3], r3[3], r4[3], r5[3];
  // y, R2..R5: the first three (position) components
  template <class T>
  __device__ __forceinline__ void init(float sig, float F0f, float cm0, float cm1, float cm2,
                                       const T* y, const T* R2, const T* R3, const T* R4,
                                       const T* R5) {
    sg = sig;
    F0 = F0f;
    m0 = cm0;
    m1 = cm1;
    m2 = cm2;
    const float y0 = (float)y[0], y1 = (float)y[1], y2 = (float)y[2];
    const float mx = m0 * y0 + m1 * y1 + m2 * y2;
    gF[0] = 3.0f * y2 * m0 - 2.0f * m2 * y0;
    gF[1] = 3.0f * y2 * m1 - 2.0f * m2 * y1;
    gF[2] = 3.0f * mx + 3.0f * y2 * m2 - 2.0f * m2 * y2;
#pragma unroll
    for (int i = 0; i < 3; ++i) {
      r2[i] = (float)R2[i];
      r3[i] = (float)R3[i];
      r4[i] = (float)R4[i];
      r5[i] = (float)R5[i];
    }
  }
  __device__ __forceinline__ float operator()(float th) const {
    float d[3];
#pragma unroll
    for (int i = 0; i < 3; ++i)
      d[i] = th * (r2[i] + (1.0f - th) * (r3[i] + th * (r4[i] + (1.0f - th) * r5[i])));
    const float md = m0 * d[0] + m1 * d[1] + m2 * d[2];
    const float dd = d[0] * d[0] + d[1] * d[1] + d[2] * d[2];
    return sg * (F0 + (gF[0] * d[0] + gF[1] * d[1] + gF[2] * d[2]) + (3.0f * d[2] * md - m2 * dd));
  }
};

// FP32 model of r_out^2 - |x(th)|^2 on the same extension: c0 - 2 y.d - |d|^2,
// c0 = r_out^2 - |y|^2 from FP64.
struct EscapeModel32 {
  float c0, y[3], r2[3], r3[3], r4[3], r5[3];
  template <class T>
  __device__ __forceinline__ void init(float c0f, const T* yd, const T* R2, const T* R3,
                                       const T* R4, const T* R5) {
    c0 = c0f;
#pragma unroll
    for (int i = 0; i < 3; ++i) {
      y[i] = (float)yd[i];
      r2[i] = (float)R2[i];
      r3[i] = (float)R3[i];
      r4[i] = (float)R4[i];
      r5[i] = (float)R5[i];
    }
  }
  __device__ __forceinline__ float operator()(float th) const {
    float d[3];
#pragma unroll
    for (int i = 0; i < 3; ++i)
      d[i] = th * (r2[i] + (1.0f - th) * (r3[i] + th * (r4[i] + (1.0f - th) * r5[i])));
    return c0 - (2.0f * (y[0] * d[0] + y[1] * d[1] + y[2] * d[2]) +
                 (d[0] * d[0] + d[1] * d[1] + d[2] * d[2]));
  }
};

// One attempted Dormand-Prince step.  Returns -1 to continue, else the final
// ray status.  hook.on_accept sees every accepted step (start, end, stages).
template <class Hook>
__device__ int advance(const TraceParams& p, Lane& L, Hook& hook) {
  if (L.na >= p.max_steps || L.na + L.nr >= 4 * p.max_steps) return RAY_MAXSTEPS;
  bool clipped = false;
  double h = L.h;
  {
    // displacement of one step at most STEP_REACH x the distance to the centre
    const double v2 = L.f0[0] * L.f0[0] + L.f0[1] * L.f0[1] + L.f0[2] * L.f0[2];
    const double r2 = L.y[0] * L.y[0] + L.y[1] * L.y[1] + L.y[2] * L.y[2];
    if (h * h * v2 > STEP_REACH * STEP_REACH * r2) h = STEP_REACH * sqrt(r2 / v2);
  }
  if (p.lambda_max > 0.0 && L.lam + h >= p.lambda_max) {
    h = p.lambda_max - L.lam;
    clipped = true;
  }
  const double* y = L.y;
  const double* k1 = L.f0;
  double t[6], k2[6], k3[6], k4[6], k5[6], k6[6], k7[6], yn[6];
#pragma unroll
  for (int i = 0; i < 6; ++i) t[i] = y[i] + h * (DP::a21 * k1[i]);
  rhs64(L.c, t, k2);
#pragma unroll
  for (int i = 0; i < 6; ++i) t[i] = y[i] + h * (DP::a31 * k1[i] + DP::a32 * k2[i]);
  rhs64(L.c, t, k3);
#pragma unroll
  for (int i = 0; i < 6; ++i)
    t[i] = y[i] + h * (DP::a41 * k1[i] + DP::a42 * k2[i] + DP::a43 * k3[i]);
  rhs64(L.c, t, k4);
#pragma unroll
  for (int i = 0; i < 6; ++i)
    t[i] = y[i] + h * (DP::a51 * k1[i] + DP::a52 * k2[i] + DP::a53 * k3[i] + DP::a54 * k4[i]);
  rhs64(L.c, t, k5);
#pragma unroll
  for (int i = 0; i < 6; ++i)
    t[i] = y[i] + h * (DP::a61 * k1[i] + DP::a62 * k2[i] + DP::a63 * k3[i] + DP::a64 * k4[i] +
                       DP::a65 * k5[i]);
  rhs64(L.c, t, k6);
#pragma unroll
  for (int i = 0; i < 6; ++i)
    yn[i] = y[i] + h * (DP::b1 * k1[i] + DP::b3 * k3[i] + DP::b4 * k4[i] + DP::b5 * k5[i] +
                        DP::b6 * k6[i]);
  rhs64(L.c, yn, k7);
  double s = 0.0;
#pragma unroll
  for (int i = 0; i < 6; ++i) {
    const double e = h * (DP::e1 * k1[i] + DP::e3 * k3[i] + DP::e4 * k4[i] + DP::e5 * k5[i] +
                          DP::e6 * k6[i] + DP::e7 * k7[i]);
    const double sc = p.atol + p.rtol * fmax(fabs(y[i]), fabs(yn[i]));
    s += (e / sc) * (e / sc);
  }
  const double en = sqrt(s / 6.0);
  if (!isfinite(en)) {
    ++L.nr;
    L.h = h * 0.2;
    L.last_rej = true;
    return (L.h < 1e-12) ? RAY_NAN : -1;
  }
  const bool gj = (L.c.plasma == PLASMA_GJ);
  if (en <= 1.0 && gj && !L.switching &&
      L.c.sig * gj_side<double>(L.c.m0, L.c.m1, L.c.m2, yn[0], yn[1], yn[2]) < 0.0) {
    // the step crossed the null cone: largest th with the start side on the
    // continuous extension (bisection), then redo the step to end just past it
    double r3[3], r4[3], r5[3], r2[3];
#pragma unroll
    for (int i = 0; i < 3; ++i) {
      r2[i] = yn[i] - y[i];
      r3[i] = h * k1[i] - r2[i];
      r4[i] = r2[i] - h * k7[i] - r3[i];
      r5[i] = h * (DP::d1 * k1[i] + DP::d3 * k3[i] + DP::d4 * k4[i] + DP::d5 * k5[i] +
                   DP::d6 * k6[i] + DP::d7 * k7[i]);
    }
    // largest th with the start side on the continuous extension: Illinois
    // (regula falsi with halving) on s(th) = sig (3 z (m.x) - m_z |x|^2), whose
    // sign is the side, bracketed on [0, 1]; a bisection step whenever the
    // bracket did not halve, to the last representable th
    const double sgn = L.c.sig;
    auto side_val = [&](double th) {
      double xd[3];
#pragma unroll
      for (int i = 0; i < 3; ++i)
        xd[i] = y[i] + th * (r2[i] + (1.0 - th) * (r3[i] + th * (r4[i] + (1.0 - th) * r5[i])));
      const double mx = L.c.m0 * xd[0] + L.c.m1 * xd[1] + L.c.m2 * xd[2];
      const double rr = xd[0] * xd[0] + xd[1] * xd[1] + xd[2] * xd[2];
      return sgn * (3.0 * xd[2] * mx - L.c.m2 * rr);
    };
    double flo = side_val(0.0), fhi = side_val(1.0);
    if (!(flo >= 0.0)) flo = 0.0;                  // the start is on its own side
    if (!(fhi < 0.0)) fhi = -1e-300;
    double hi;
    const double lo = last_nonneg(side_val, flo, fhi, &hi);
    ++L.nr;
    if (lo < SWITCH_MIN_FRACTION) {
      L.c.sig = -L.c.sig;             // already at the cone: switch here
      rhs64(L.c, L.y, L.f0);
      L.h = h;
    } else {
      L.h_resume = h;
      L.h = h * lo * (1.0 + SWITCH_OVERSHOOT);
      L.switching = true;
    }
    return -1;
  }
  if (en <= 1.0) {
    ++L.na;
    hook.on_accept(L, y, yn, k1, k2, k3, k4, k5, k6, k7, h);
    const double rnew2 = yn[0] * yn[0] + yn[1] * yn[1] + yn[2] * yn[2];
    if (rnew2 >= p.r_out * p.r_out) {
      // locate |x(th)| = r_out on the continuous extension
      double r3[6], r4[6], r5[6];
#pragma unroll
      for (int i = 0; i < 6; ++i) {
        const double r2 = yn[i] - y[i];
        r3[i] = h * k1[i] - r2;
        r4[i] = r2 - h * k7[i] - r3[i];
        r5[i] = h * (DP::d1 * k1[i] + DP::d3 * k3[i] + DP::d4 * k4[i] + DP::d5 * k5[i] +
                     DP::d6 * k6[i] + DP::d7 * k7[i]);
        t[i] = r2;
      }
      // r_out^2 - |x(th)|^2 changes sign on [0, 1]: Illinois to the last
      // representable th (the root to rounding, in ~10 evaluations)
      const double ro2 = p.r_out * p.r_out;
      auto inside = [&](double th) {
        double xd[3];
#pragma unroll
        for (int i = 0; i < 3; ++i)
          xd[i] = y[i] + th * (t[i] + (1.0 - th) * (r3[i] + th * (r4[i] + (1.0 - th) * r5[i])));
        return ro2 - (xd[0] * xd[0] + xd[1] * xd[1] + xd[2] * xd[2]);
      };
      double flo = ro2 - (y[0] * y[0] + y[1] * y[1] + y[2] * y[2]);
      if (!(flo >= 0.0)) flo = 0.0;
      double fhi = ro2 - rnew2;
      if (!(fhi < 0.0)) fhi = -1e-300;
      double hi;
      const double lo = last_nonneg(inside, flo, fhi, &hi);
      const double th = 0.5 * (lo + hi);
#pragma unroll
      for (int i = 0; i < 6; ++i)
        yn[i] = y[i] + th * (t[i] + (1.0 - th) * (r3[i] + th * (r4[i] + (1.0 - th) * r5[i])));
#pragma unroll
      for (int i = 0; i < 6; ++i) L.y[i] = yn[i];
      L.lam += th * h;
      return RAY_ESCAPED;
    }
#pragma unroll
    for (int i = 0; i < 6; ++i) {
      L.y[i] = yn[i];
      L.f0[i] = k7[i];
    }
    L.lam += h;
    if (rnew2 <= p.r_capture * p.r_capture) return RAY_CAPTURED;
    if (clipped) return RAY_LAMBDA_END;
    if (gj && L.c.sig * gj_side<double>(L.c.m0, L.c.m1, L.c.m2, L.y[0], L.y[1], L.y[2]) < 0.0) {
      L.c.sig = -L.c.sig;             // past the cone: continue on the other side
      rhs64(L.c, L.y, L.f0);
    }
    if (L.switching) {
      L.h = L.h_resume;
      L.switching = false;
    } else {
      L.h = h * step_factor(en, true, L.last_rej);
    }
    L.last_rej = false;
    return -1;
  }
  ++L.nr;
  L.h = h * step_factor(en, false, L.last_rej);
  L.last_rej = true;
  return (L.h < 1e-12) ? RAY_STIFF : -1;
}

}  // namespace
}  // namespace rtk
