// Forward tracing in double-float (RT_PREC_DF): the FP64 integrator of
// rt_integrator.cuh -- the same Hamiltonian right-hand side (ham_rhs,
// instantiated on the double-float scalar of rt_df.cuh), the same
// Dormand-Prince 5(4) step with its embedded error estimate, step-size
// controller, step reach, Goldreich-Julian null-cone switch and escape
// location on the continuous extension -- with every arithmetic operation on
// the FP32 pipe.  Accuracy is FP64-class (a few units of 2^-47 per operation
// against 2^-53); no operation of an attempted step touches the FP64 pipe.
// One lane per ray in a persistent kernel with the warp-ballot work queue
// (claim_items), index- or cost-ordered; no tail mode is needed: a lone ray's
// attempt is a chain of FP32 instructions with instruction-level parallelism
// across its six components.
#include <cuda_runtime.h>
#include <stdint.h>

#include "rt_df.cuh"
#include "rt_device.cuh"
#include "rt_integrator.cuh"
#include "rt_internal.h"

namespace rtk {

namespace {

// Dormand-Prince coefficients rounded to double-float (48 bits: the method's
// order conditions hold to that precision)
struct DPD {
  static constexpr DF a21 = DF(DP::a21);
  static constexpr DF a31 = DF(DP::a31), a32 = DF(DP::a32);
  static constexpr DF a41 = DF(DP::a41), a42 = DF(DP::a42), a43 = DF(DP::a43);
  static constexpr DF a51 = DF(DP::a51), a52 = DF(DP::a52), a53 = DF(DP::a53),
                      a54 = DF(DP::a54);
  static constexpr DF a61 = DF(DP::a61), a62 = DF(DP::a62), a63 = DF(DP::a63),
                      a64 = DF(DP::a64), a65 = DF(DP::a65);
  static constexpr DF b1 = DF(DP::b1), b3 = DF(DP::b3), b4 = DF(DP::b4), b5 = DF(DP::b5),
                      b6 = DF(DP::b6);
  static constexpr DF e1 = DF(DP::e1), e3 = DF(DP::e3), e4 = DF(DP::e4), e5 = DF(DP::e5),
                      e6 = DF(DP::e6), e7 = DF(DP::e7);
  static constexpr DF d1 = DF(DP::d1), d3 = DF(DP::d3), d4 = DF(DP::d4), d5 = DF(DP::d5),
                      d6 = DF(DP::d6), d7 = DF(DP::d7);
};

constexpr float SWITCH_MIN_FRACTION_D = (float)SWITCH_MIN_FRACTION;
// the event search: the FP32 model's root widened by SEED_WIDEN_D (relative),
// then Illinois in double-float th to SEED_TOL_D relative (the rounding of
// the double-float side function near a root, ~2^-47 |x|^2 / |dF/dth|, sets
// the floor; far below the 1e-10 relative overshoot of a switch)
constexpr float SEED_WIDEN_D = 0x1p-16f;
constexpr float SEED_TOL_D = 0x1p-40f;

// Butcher rows in double-float: row s (1..5) combines stages 0..s-1 into the
// input of stage s, row 6 is the 5th-order update (b_2 = 0); the error
// weights e_j and the continuous extension's d_j (index j = stage - 1).
__constant__ DF c_A[7][6] = {
    {DF(0), DF(0), DF(0), DF(0), DF(0), DF(0)},
    {DPD::a21, DF(0), DF(0), DF(0), DF(0), DF(0)},
    {DPD::a31, DPD::a32, DF(0), DF(0), DF(0), DF(0)},
    {DPD::a41, DPD::a42, DPD::a43, DF(0), DF(0), DF(0)},
    {DPD::a51, DPD::a52, DPD::a53, DPD::a54, DF(0), DF(0)},
    {DPD::a61, DPD::a62, DPD::a63, DPD::a64, DPD::a65, DF(0)},
    {DPD::b1, DF(0), DPD::b3, DPD::b4, DPD::b5, DPD::b6}};
__constant__ DF c_E[7] = {DPD::e1, DF(0), DPD::e3, DPD::e4, DPD::e5, DPD::e6, DPD::e7};

// The right-hand side in double-float, not inlined: at ~1500 instructions a
// call, six inlined copies per attempt would overflow the instruction cache.
// The Goldreich-Julian anisotropic medium (the benchmark's) has a copy with
// the model switches fixed, free of the other media's branches.
__device__ __noinline__ void rhs_df_any(const RayConst<DF>& c, const DF* y, DF* f) {
  ham_rhs<DF>(c, y[0], y[1], y[2], y[3], y[4], y[5], f[0], f[1], f[2], f[3], f[4], f[5]);
}
__device__ __noinline__ void rhs_df_gj_aniso(const RayConst<DF>& c0, const DF* y, DF* f) {
  RayConst<DF> c = c0;
  c.plasma = PLASMA_GJ;
  c.disp = DISP_ANISO;
  ham_rhs<DF>(c, y[0], y[1], y[2], y[3], y[4], y[5], f[0], f[1], f[2], f[3], f[4], f[5]);
}
__device__ __forceinline__ void rhs_df(const RayConst<DF>& c, const DF* y, DF* f) {
  if (c.plasma == PLASMA_GJ && c.disp == DISP_ANISO)
    rhs_df_gj_aniso(c, y, f);
  else
    rhs_df_any(c, y, f);
}

// F = 3 z (m.x) - m_z |x|^2, whose sign is the side of the null cone
__device__ __forceinline__ DF cone_df(const RayConst<DF>& c, const DF* x) {
  const DF mx = c.m0 * x[0] + c.m1 * x[1] + c.m2 * x[2];
  const DF r2 = x[0] * x[0] + x[1] * x[1] + x[2] * x[2];
  return DF(3) * x[2] * mx - c.m2 * r2;
}

// The controller of step_factor() in double-float: the step sizes, and with
// them the discretisation, are the FP64 integrator's to ~1e-14 (an FP32
// controller would change every step by ~1e-7 and the end points at the level
// of the integration error).
__device__ __forceinline__ DF step_factor_df(DF err, bool accepted, bool last_rej) {
  constexpr DF c09 = DF(0.9);
  DF fac = (err.hi > 1e6f) ? DF(0) : (err.hi >= 1e-6f) ? c09 * df_pow_m1_5(err) : DF(5);
  if (fac < DF(0.2f, 0.0f)) fac = DF(0.2f, 0.0f);
  if (DF(5) < fac) fac = DF(5);
  if ((!accepted || last_rej) && DF(1) < fac) fac = DF(1);
  return fac;
}

// The scaled RMS error norm sqrt(sum ((e_i / (atol + rtol max(|y_i|, |yn_i|)))^2) / 6)
// in double-float, as the FP64 integrator forms it.
__device__ __forceinline__ DF scale_df(DF atol, DF rtol, DF a, DF b) {
  return atol + rtol * df_max(df_abs(a), df_abs(b));
}

struct LaneD {
  RayConst<DF> c;
  DF y[6], f0[6];
  DF h, h_resume;      // double-float: a redone step ends 1e-10 relative past a crossing
  int na, nr;
  bool last_rej;
  bool switching;      // the current attempt ends just past a null-cone crossing
  double R_km, ma_eV;
};

__device__ __forceinline__ int find_star_d(const TraceParams& p, int64_t i) {
  if (p.nstars <= 1) return 0;
  int lo = 0, hi = p.nstars - 1;
  while (lo < hi) {
    const int mid = (lo + hi + 1) >> 1;
    if (p.offsets[mid] <= i) lo = mid; else hi = mid - 1;
  }
  return lo;
}

// Hairer's two-evaluation initial step (order 5), as initial_step(), in
// double-float.
__device__ __forceinline__ DF initial_step_df(const RayConst<DF>& c, const DF* y0, const DF* f0,
                                              DF rtol, DF atol) {
  DF dnf(0), dny(0), sk[6];
#pragma unroll
  for (int i = 0; i < 6; ++i) {
    sk[i] = atol + rtol * df_abs(y0[i]);
    const DF a = df_div(f0[i], sk[i]), b = df_div(y0[i], sk[i]);
    dnf += a * a;
    dny += b * b;
  }
  constexpr DF c001 = DF(0.01);
  const DF h = (dnf.hi <= 1e-10f || dny.hi <= 1e-10f) ? DF(1e-6) : df_sqrt(df_div(dny, dnf)) * c001;
  DF y1[6], f1[6];
#pragma unroll
  for (int i = 0; i < 6; ++i) y1[i] = y0[i] + h * f0[i];
  rhs_df(c, y1, f1);
  DF der2(0);
#pragma unroll
  for (int i = 0; i < 6; ++i) {
    const DF d = df_div(f1[i] - f0[i], sk[i]);
    der2 += d * d;
  }
  der2 = df_div(df_sqrt(der2), h);
  const DF der12 = df_max(df_abs(der2), df_sqrt(dnf));
  // (0.01 / der12)^(1/5) = (100 der12)^(-1/5)
  DF h1;
  if (der12.hi <= 1e-15f) {
    h1 = df_max(DF(1e-6), h * 1e-3f);
  } else {
    const DF x = der12 * 100.0f;
    h1 = (x.hi >= 1e-6f && x.hi <= 1e6f) ? df_pow_m1_5(x) : DF(exp2f(-0.2f * log2f(x.hi)), 0.0f);
  }
  const DF h100 = h * 100.0f;
  return (h1 < h100) ? h1 : h100;
}

__device__ __forceinline__ void load_lane_d(const TraceParams& p, int64_t i, LaneD& L) {
  const StarDev& s = p.stars[find_star_d(p, i)];
  const int64_t n = p.n;
  L.R_km = s.R_km;
  L.ma_eV = s.ma_eV;
  const double iR = 1.0 / s.R_km, im = 1.0 / s.ma_eV;
#pragma unroll
  for (int c = 0; c < 3; ++c) {
    L.y[c] = df_of(p.state[c * n + i] * iR);
    L.y[3 + c] = df_of(p.state[(3 + c) * n + i] * im);
  }
  const double om = 1.0 + p.state[6 * n + i];
  double sp, cpsi;
  sincos(p.state[7 * n + i], &sp, &cpsi);
  L.c.rs = df_of(s.rs_prop);
  L.c.cp = df_of(s.cp);
  L.c.pa = df_of(s.plasma_a);
  L.c.W2 = df_of(om * om);
  L.c.iW2 = df_of(1.0 / (om * om));
  L.c.m0 = df_of(s.sin_tm * cpsi);
  L.c.m1 = df_of(s.sin_tm * sp);
  L.c.m2 = df_of(s.cos_tm);
  L.c.disp = s.dispersion;
  L.c.plasma = s.plasma;
  L.c.sig = (cone_df(L.c, L.y).hi < 0.0f) ? DF(-1) : DF(1);
  L.switching = false;
  L.h_resume = DF(0);
  rhs_df(L.c, L.y, L.f0);
  L.h = initial_step_df(L.c, L.y, L.f0, df_of(p.rtol), df_of(p.atol));
  L.na = 0;
  L.nr = 0;
  L.last_rej = false;
}

__device__ __forceinline__ void store_lane_d(const TraceParams& p, int64_t i, const LaneD& L, int st) {
  const int64_t n = p.n;
#pragma unroll
  for (int c = 0; c < 3; ++c) {
    p.state[c * n + i] = df_d(L.y[c]) * L.R_km;
    p.state[(3 + c) * n + i] = df_d(L.y[3 + c]) * L.ma_eV;
  }
  status_after_state(p, i, st);
  if (p.nacc) p.nacc[i] = L.na;
  if (p.nrej) p.nrej[i] = L.nr;
}

// Illinois on [lo, hi] in double-float th, FP32 values of the side function
// (side(lo) = flo >= 0 > fhi = side(hi)): th moves by the FP32 secant
// fraction of the double-float width, so it keeps its 48 bits as the bracket
// shrinks; after eight plain steps, a bisection step whenever the bracket did
// not halve over two (rounding noise of the values near the root); until the
// width is at most tol x hi, stops shrinking, or 48 evaluations were spent.
// Returns lo; *hi_out the end past it.
template <class S>
__device__ __forceinline__ DF last_nonneg_df(const S& side, DF lo, DF hi, float flo, float fhi,
                                             float tol, DF* hi_out) {
  int last = 0;
  float wprev = df_f(hi - lo);
  for (int it = 0; it < 48; ++it) {
    const DF w = hi - lo;
    const float wf = w.hi;
    if (!(wf > tol * hi.hi)) break;
    float frac = flo / (flo - fhi);
    if (it >= 8 && (it & 1) && wf > 0.5f * wprev) frac = 0.5f;
    if (!(frac > 0.0f && frac < 1.0f)) frac = 0.5f;
    if (it & 1) wprev = wf;
    const DF mid = lo + w * frac;
    if (!(lo < mid && mid < hi)) break;
    const float fm = side(mid);
    if (fm >= 0.0f) {
      lo = mid;
      flo = fm;
      if (last > 0) fhi *= 0.5f;
      last = 1;
    } else {
      hi = mid;
      fhi = fm;
      if (last < 0) flo *= 0.5f;
      last = -1;
    }
  }
  *hi_out = hi;
  return lo;
}

// The event's th, seeded by the FP32 model of the side function (model(th),
// FP32), whose plain Illinois brackets the root to 2^-22 relative.  Where the
// double-float side function confirms that bracket (two evaluations), the
// secant through those two values gives the root to ~1e-14 (the bracket is
// a few ulp of FP32 wide: curvature ~1e-13, rounding of the values ~1e-14),
// far inside the 1e-10 relative overshoot of a switch; returned as both ends.
// Otherwise (a grazing crossing, or the model's rounding moved the root
// further) the model's root, widened by SEED_WIDEN_D on each side, is checked
// and the double-float Illinois narrows the bracket (or the part of [0, 1]
// left or right of it that holds the root).
template <class S, class M>
__device__ __forceinline__ DF last_nonneg_seeded_df(const S& side, const M& model, float flo,
                                                    float fhi, DF* hi_out) {
  float l = 0.0f, u = 1.0f, fl = flo, fu = fhi;
  illinois(model, l, u, fl, fu, SEED_TOL32, 40);
  {
    const float fa = (l > 0.0f) ? side(DF(l, 0.0f)) : flo;
    const float fb = (u < 1.0f) ? side(DF(u, 0.0f)) : fhi;
    if (fa >= 0.0f && fb < 0.0f) {
      const DF th = DF(l, 0.0f) + (DF(u, 0.0f) - DF(l, 0.0f)) * (fa / (fa - fb));
      *hi_out = th;
      return th;
    }
  }
  const float W = SEED_WIDEN_D * u + 0x1p-30f;
  const float a = fmaxf(0.0f, l - W), b = fminf(1.0f, u + W);
  DF lo(0), hi(1);
  const float fa = (a > 0.0f) ? side(DF(a, 0.0f)) : flo;
  if (fa < 0.0f) {
    hi = DF(a, 0.0f);                             // the root lies left of the FP32 bracket
    fhi = fa;
  } else {
    lo = DF(a, 0.0f);
    flo = fa;
    const float fb = (b < 1.0f) ? side(DF(b, 0.0f)) : fhi;
    if (fb >= 0.0f) {
      lo = DF(b, 0.0f);                           // right of it
      flo = fb;
    } else {
      hi = DF(b, 0.0f);
      fhi = fb;
    }
  }
  return last_nonneg_df(side, lo, hi, flo, fhi, SEED_TOL_D, hi_out);
}

// One attempted Dormand-Prince step, as advance() in rt_integrator.cuh.
// ro2 = r_out^2, rc2 = r_capture^2, tol = (rtol, atol).  Returns -1 to
// continue, else the final ray status.  (Inlined: a lane passed by reference
// to a call would live in local memory.)
__device__ __forceinline__ bool out_of_steps(const TraceParams& p, const LaneD& L) {
  return L.na >= p.max_steps || L.na + L.nr >= 4 * p.max_steps;
}

// The attempt's step: the lane's, limited to a displacement of STEP_REACH x
// the distance to the centre.
__device__ __forceinline__ DF attempt_h(const LaneD& L) {
  DF h = L.h;
  const DF v2 = L.f0[0] * L.f0[0] + L.f0[1] * L.f0[1] + L.f0[2] * L.f0[2];
  const DF r2 = L.y[0] * L.y[0] + L.y[1] * L.y[1] + L.y[2] * L.y[2];
  constexpr DF sr = DF(STEP_REACH), sr2 = DF(STEP_REACH * STEP_REACH);
  if (sr2 * r2 < h * h * v2) h = sr * df_sqrt(df_div(r2, v2));
  return h;
}

// The rest of an attempt once its stages are known (k[0..6] and the 5th-order
// end point yn): error estimate, null-cone and escape events, the decision.
__device__ __forceinline__ int finish_df(const TraceParams& p, LaneD& L, DF h, DF (*k)[6],
                                         const DF* yn, DF ro2, float rc2, DF rtol, DF atol);

__device__ __forceinline__ int advance_df(const TraceParams& p, LaneD& L, DF ro2, float rc2,
                                          DF rtol, DF atol) {
  if (out_of_steps(p, L)) return RAY_MAXSTEPS;
  const DF h = attempt_h(L);
  const DF* y = L.y;
  // stages: k[0] = f(y) (first-same-as-last), k[s] = f(y + h sum_j A[s][j]
  // k[j]) for s = 1..5, and row 6 the 5th-order update yn with k[6] = f(yn);
  // rolled loops around one right-hand side call keep the hot code small
  DF k[7][6], yn[6];
#pragma unroll
  for (int i = 0; i < 6; ++i) k[0][i] = L.f0[i];
#pragma unroll 1
  for (int st = 1; st < 7; ++st) {
#pragma unroll
    for (int i = 0; i < 6; ++i) {
      DF acc = c_A[st][0] * k[0][i];
#pragma unroll 1
      for (int j = 1; j < st; ++j) acc += c_A[st][j] * k[j][i];
      yn[i] = y[i] + h * acc;
    }
    rhs_df(L.c, yn, k[st]);
  }
  return finish_df(p, L, h, k, yn, ro2, rc2, rtol, atol);
}

__device__ __forceinline__ int finish_df(const TraceParams& p, LaneD& L, DF h, DF (*k)[6],
                                         const DF* yn, DF ro2, float rc2, DF rtol, DF atol) {
  const DF* y = L.y;
  const DF* k1 = k[0];
  const DF* k3 = k[2];
  const DF* k4 = k[3];
  const DF* k5 = k[4];
  const DF* k6 = k[5];
  const DF* k7 = k[6];
  // embedded error estimate and its scaled norm
  DF s(0);
#pragma unroll 1
  for (int i = 0; i < 6; ++i) {
    DF acc = c_E[0] * k[0][i];
#pragma unroll 1
    for (int j = 2; j < 7; ++j) acc += c_E[j] * k[j][i];
    const DF e = h * acc;
    const DF q = df_div(e, scale_df(atol, rtol, y[i], yn[i]));
    s += q * q;
  }
  constexpr DF sixth = DF(1.0 / 6.0);
  const DF en = df_sqrt(s * sixth);
  const bool ok = df_le(en, DF(1));
  if (!isfinite(en.hi)) {
    ++L.nr;
    L.h = h * 0.2f;
    L.last_rej = true;
    return (L.h.hi < 1e-12f) ? RAY_NAN : -1;
  }
  const bool gj = (L.c.plasma == PLASMA_GJ);
  float Fend = 0.0f;
  if (ok && gj) Fend = df_f(cone_df(L.c, yn));
  const float sgn = L.c.sig.hi;
  if (ok && gj && !L.switching && sgn * Fend < 0.0f) {
    // the step crossed the null cone: locate the crossing on the continuous
    // extension and redo the step to end just past it
    DF r2[3], r3[3], r4[3], r5[3];
#pragma unroll
    for (int i = 0; i < 3; ++i) {
      r2[i] = yn[i] - y[i];
      r3[i] = h * k1[i] - r2[i];
      r4[i] = r2[i] - h * k7[i] - r3[i];
      r5[i] = h * (DPD::d1 * k1[i] + DPD::d3 * k3[i] + DPD::d4 * k4[i] + DPD::d5 * k5[i] +
                   DPD::d6 * k6[i] + DPD::d7 * k7[i]);
    }
    auto side = [&](DF th) -> float {
      const DF u = DF(1) - th;
      DF xd[3];
#pragma unroll
      for (int i = 0; i < 3; ++i) xd[i] = y[i] + th * (r2[i] + u * (r3[i] + th * (r4[i] + u * r5[i])));
      return sgn * df_f(cone_df(L.c, xd));
    };
    float flo = sgn * df_f(cone_df(L.c, y)), fhi = sgn * Fend;
    if (!(flo >= 0.0f)) flo = 0.0f;                 // the start is on its own side
    if (!(fhi < 0.0f)) fhi = -1e-30f;
    float yq[3], q2[3], q3[3], q4[3], q5[3];
#pragma unroll
    for (int i = 0; i < 3; ++i) {
      yq[i] = y[i].hi;
      q2[i] = r2[i].hi;
      q3[i] = r3[i].hi;
      q4[i] = r4[i].hi;
      q5[i] = r5[i].hi;
    }
    ConeModel32 m32;
    m32.init(sgn, sgn * flo, L.c.m0.hi, L.c.m1.hi, L.c.m2.hi, yq, q2, q3, q4, q5);
    DF hi;
    const DF lo = last_nonneg_seeded_df(side, m32, flo, fhi, &hi);
    ++L.nr;
    if (lo.hi < SWITCH_MIN_FRACTION_D) {
      L.c.sig = -L.c.sig;             // already at the cone: switch here
      rhs_df(L.c, L.y, L.f0);
      L.h = h;
    } else {
      constexpr DF past = DF(1.0 + SWITCH_OVERSHOOT);
      L.h_resume = h;
      L.h = h * lo * past;
      L.switching = true;
    }
    return -1;
  }
  if (ok) {
    ++L.na;
    const DF rn2 = yn[0] * yn[0] + yn[1] * yn[1] + yn[2] * yn[2];
    if (!(df_f(ro2 - rn2) > 0.0f)) {
      // |x(th)| = r_out on the continuous extension
      DF r2[6], r3[6], r4[6], r5[6];
#pragma unroll
      for (int i = 0; i < 6; ++i) {
        r2[i] = yn[i] - y[i];
        r3[i] = h * k1[i] - r2[i];
        r4[i] = r2[i] - h * k7[i] - r3[i];
        r5[i] = h * (DPD::d1 * k1[i] + DPD::d3 * k3[i] + DPD::d4 * k4[i] + DPD::d5 * k5[i] +
                     DPD::d6 * k6[i] + DPD::d7 * k7[i]);
      }
      auto inside = [&](DF th) -> float {
        const DF u = DF(1) - th;
        DF xd[3];
#pragma unroll
        for (int i = 0; i < 3; ++i)
          xd[i] = y[i] + th * (r2[i] + u * (r3[i] + th * (r4[i] + u * r5[i])));
        return df_f(ro2 - (xd[0] * xd[0] + xd[1] * xd[1] + xd[2] * xd[2]));
      };
      float flo = df_f(ro2 - (y[0] * y[0] + y[1] * y[1] + y[2] * y[2]));
      if (!(flo >= 0.0f)) flo = 0.0f;
      float fhi = df_f(ro2 - rn2);
      if (!(fhi < 0.0f)) fhi = -1e-30f;
      float yq[3], q2[3], q3[3], q4[3], q5[3];
#pragma unroll
      for (int i = 0; i < 3; ++i) {
        yq[i] = y[i].hi;
        q2[i] = r2[i].hi;
        q3[i] = r3[i].hi;
        q4[i] = r4[i].hi;
        q5[i] = r5[i].hi;
      }
      EscapeModel32 e32;
      e32.init(flo, yq, q2, q3, q4, q5);
      DF hi;
      const DF lo = last_nonneg_seeded_df(inside, e32, flo, fhi, &hi);
      const DF th = (lo + hi) * 0.5f;
      const DF u = DF(1) - th;
      DF ye[6];
#pragma unroll
      for (int i = 0; i < 6; ++i) ye[i] = y[i] + th * (r2[i] + u * (r3[i] + th * (r4[i] + u * r5[i])));
#pragma unroll
      for (int i = 0; i < 6; ++i) L.y[i] = ye[i];
      return RAY_ESCAPED;
    }
#pragma unroll
    for (int i = 0; i < 6; ++i) {
      L.y[i] = yn[i];
      L.f0[i] = k7[i];
    }
    if (rn2.hi <= rc2) return RAY_CAPTURED;
    if (gj && sgn * Fend < 0.0f) {
      L.c.sig = -L.c.sig;             // past the cone: continue on the other side
      rhs_df(L.c, L.y, L.f0);
    }
    if (L.switching) {
      L.h = L.h_resume;
      L.switching = false;
    } else {
      L.h = h * step_factor_df(en, true, L.last_rej);
    }
    L.last_rej = false;
    return -1;
  }
  ++L.nr;
  L.h = h * step_factor_df(en, false, L.last_rej);
  L.last_rej = true;
  return (L.h.hi < 1e-12f) ? RAY_STIFF : -1;
}

__global__ void __launch_bounds__(256) trace_df_kernel(TraceParams p) {
  const int lane = threadIdx.x & 31;
  int64_t ray = -1;
  LaneD L;
  long long acc = 0, rej = 0, traced = 0, esc = 0;
  if (p.ts && threadIdx.x == 0) atomicMin(p.ts, global_ns());
  const DF ro2 = df_of(p.r_out * p.r_out);
  const float rc2 = (float)(p.r_capture * p.r_capture);
  const DF rtol = df_of(p.rtol), atol = df_of(p.atol);
  // one pass over the rays, or COST_BUCKETS passes (cost-ordered claims: the
  // rays that start nearest the null cone first)
  const int64_t nq = p.order ? (int64_t)COST_BUCKETS * p.n : p.n;
  ClaimChunk ch;
  for (;;) {
    claim_items(p.queue, nq, p.refill_min, p.claim_size, ray, ch, [&](int64_t idx) -> int64_t {
      const int pass = p.order ? (int)(idx / p.n) : 0;
      const int64_t i = idx - (int64_t)pass * p.n;
      if (p.status[i] != RAY_READY ||
          (p.order && (cost_bucket(p.stars[find_star_d(p, i)], p.state, p.n, i) != pass ||
                       !status_still(p, i, RAY_READY))))
        return -1;
      load_lane_d(p, i, L);
      return i;
    });
    if (__ballot_sync(FULL, ray != -2) == 0) break;
    if (ray >= 0) {
      const int st = advance_df(p, L, ro2, rc2, rtol, atol);
      if (st >= 0) {
        store_lane_d(p, ray, L, st);
        if (p.ts) atomicMax(p.ts + 1 + find_star_d(p, ray), global_ns());
        acc += L.na;
        rej += L.nr;
        traced += 1;
        esc += (st == RAY_ESCAPED);
        ray = -1;
      }
    }
  }
  if (p.counters) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
      acc += __shfl_down_sync(FULL, acc, o);
      rej += __shfl_down_sync(FULL, rej, o);
      traced += __shfl_down_sync(FULL, traced, o);
      esc += __shfl_down_sync(FULL, esc, o);
    }
    if (lane == 0) {
      atomicAdd((unsigned long long*)&p.counters[CTR_ACC], (unsigned long long)acc);
      atomicAdd((unsigned long long*)&p.counters[CTR_REJ], (unsigned long long)rej);
      atomicAdd((unsigned long long*)&p.counters[CTR_RAYS], (unsigned long long)traced);
      atomicAdd((unsigned long long*)&p.counters[CTR_ESC], (unsigned long long)esc);
    }
  }
}

}  // namespace

cudaError_t launch_trace_df(const TraceParams& p, int block, int blocks_per_sm,
                            cudaStream_t stream) {
  int dev = 0, nsm = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return e;
  e = cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev);
  if (e != cudaSuccess) return e;
  if (block <= 0) block = 128;
  if (block > 256) block = 256;
  block = (block / 32) * 32;
  if (block < 32) block = 32;
  if (blocks_per_sm <= 0) {
    // default: one 128-thread block per SM, one warp per scheduler.  Measured
    // on the eight-step benchmark launch: 2.66-2.69 s against 2.84 s with the
    // two blocks the registers allow; the rays guided along the null cone set
    // the launch's end, and a warp that has its scheduler to itself runs them
    // fastest, while the bulk loses little (the kernel is bound by
    // instruction supply, not by the number of warps)
    int occ = 0;
    e = occupancy_trace_df(block, &occ);
    if (e != cudaSuccess) return e;
    blocks_per_sm = (block >= 128 || occ < 1) ? 1 : (occ < 128 / block ? occ : 128 / block);
  }
  const int64_t warps_needed = (p.n + 31) / 32;
  int64_t grid = (int64_t)nsm * blocks_per_sm;
  const int64_t max_useful = (warps_needed * 32 + block - 1) / block;
  if (grid > max_useful) grid = max_useful;
  if (grid < 1) grid = 1;
  e = cudaMemsetAsync(p.queue, 0, sizeof(unsigned long long), stream);
  if (e != cudaSuccess) return e;
  trace_df_kernel<<<(unsigned)grid, block, 0, stream>>>(p);
  return cudaGetLastError();
}

cudaError_t occupancy_trace_df(int block, int* occ) {
  return cudaOccupancyMaxActiveBlocksPerMultiprocessor(occ, trace_df_kernel, block, 0);
}

}  // namespace rtk
