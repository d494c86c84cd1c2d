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
template <class S>
__device__ __forceinline__ double last_nonneg(const S& side_val, double flo, double fhi,
                                              double* hi_out) {
  double lo = 0.0, hi = 1.0;
  int last = 0;
  double width = 1.0;
  for (int it = 0; it < 200; ++it) {
    double mid = (lo * fhi - hi * flo) / (fhi - flo);
    if ((it & 1) && hi - lo > 0.5 * width) mid = 0.5 * (lo + hi);
    if (!(mid > lo && mid < hi)) mid = 0.5 * (lo + hi);
    if (mid <= lo || mid >= hi) break;
    if (it & 1) width = hi - lo;
    const double fm = side_val(mid);
    if (fm >= 0.0) {
      lo = mid;
      flo = fm;
      if (last > 0) fhi *= 0.5;
      last = 1;
    } else {
      hi = mid;
      fhi = fm;
      if (last < 0) flo *= 0.5;
      last = -1;
    }
  }
  *hi_out = hi;
  return lo;
}

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
