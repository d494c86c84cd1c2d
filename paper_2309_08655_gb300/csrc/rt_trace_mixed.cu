// Mixed-precision forward tracing: the Dormand-Prince stages (the analytic
// right-hand side and the stage combinations) run in FP32 with FP32
// accumulation of the increments; the ray state is kept in double-float (an
// unevaluated sum of two floats, ~48 significant bits) and receives each
// accepted increment in double-float arithmetic, so that an attempt runs on
// the FP32 pipe alone (on this GPU the FP64 pipe, conversions between FP32
// and FP64 included, has 1/64 of its rate).
//
// Increment splitting.  The position derivative is dx/dl = 2k + c(x, k), where
// the correction c (metric and plasma terms) is small away from the star.  With
// k_j = k_n + dk_j at stage j, the increment is
//   h sum_j b_j (2 k_j + c_j) = 2 h k_n + h sum_j b_j R_j,  R_j = 2 dk_j + c_j,
// (sum_j b_j = 1): the large part 2 h k_n is formed in FP64 from the FP64
// state, and only the small parts R_j pass through FP32.  The embedded error
// estimate of the positions is h sum_j e_j R_j exactly (sum_j e_j = 0), and the
// continuous extension likewise splits (sum_j d_j = 0).  FP32 rounding thus
// acts on small quantities instead of on k itself.
//
// FP32 rounding still puts a noise floor under the error estimate of the
// momenta; where a rejected step's estimate sits on that floor three times in
// a row, or the FP32 step size collapses, the ray is promoted: it is handed,
// from its current state, to the FP64 kernel (resume pass) for the rest of
// its path.  The Goldreich-Julian null cone is crossed by the same located
// branch switch as in rt_trace.cu.
#include <cuda_runtime.h>
#include <stdint.h>

#include "rt_backward.cuh"
#include "rt_df.cuh"
#include "rt_device.cuh"
#include "rt_internal.h"

namespace rtk {

namespace {

constexpr float EPS32 = 5.9604645e-8f;     // unit roundoff 2^-24
constexpr float NOISE_C = 4.0f;             // rounding amplification allowed in a stage
constexpr float NOISE_LIMIT = 0.25f;
constexpr int NOISY_REJECTIONS_TO_PROMOTE = 3;
constexpr float SWITCH_MIN_FRACTION_M = 1e-6f;
constexpr float SWITCH_OVERSHOOT_M = 1e-6f;

// c(x, k) and dk/dl at a point with FP64 position xd and FP32 momentum kf.
// The Goldreich-Julian angular factor F = 3 n_z (m.n) - m_z is a small
// difference of O(1) terms next to the null cone (where rays are guided for
// thousands of steps), so it is formed in FP64 from the FP64 position and
// magnetic axis; everything else runs in FP32.
__device__ __forceinline__ void rhs32c(const RayConst<float>& c, const double* md,
                                       const double* xd, const float* kf, float* f) {
  const double r2 = xd[0] * xd[0] + xd[1] * xd[1] + xd[2] * xd[2];
  const double g = 3.0 * xd[2] * (md[0] * xd[0] + md[1] * xd[1] + md[2] * xd[2]) - md[2] * r2;
  const float F = (float)g * __frcp_rn((float)r2);
  ham_rhs<float, true, true>(c, (float)xd[0], (float)xd[1], (float)xd[2], kf[0], kf[1], kf[2],
                             f[0], f[1], f[2], f[3], f[4], f[5], F);
}

// The same at a stage point x0 + d given in FP32 (xf = x0 + d rounded), with
// F expanded about the step's start x0: F(x0 + d) = F0 + gF.d + 3 d_z (m.d)
// - m_z |d|^2, F0 and gF = grad F(x0) formed once per step in FP64.  The FP32
// terms carry an absolute error ~ eps32 |x| |d|, as the FP64 evaluation at a
// point whose increment d went through FP32 does.
__device__ __forceinline__ void rhs32s(const RayConst<float>& c, float F0, const float* gF,
                                       const float* xf, const float* d, const float* kf,
                                       float* f) {
  const float md = c.m0 * d[0] + c.m1 * d[1] + c.m2 * d[2];
  const float dd = d[0] * d[0] + d[1] * d[1] + d[2] * d[2];
  const float F = F0 + (gF[0] * d[0] + gF[1] * d[1] + gF[2] * d[2]) +
                  (3.0f * d[2] * md - c.m2 * dd);
  const float r2 = xf[0] * xf[0] + xf[1] * xf[1] + xf[2] * xf[2];
  ham_rhs<float, true, true>(c, xf[0], xf[1], xf[2], kf[0], kf[1], kf[2], f[0], f[1], f[2], f[3],
                             f[4], f[5], F * __frcp_rn(r2));
}

__device__ __forceinline__ float side_md(const double* md, double x0, double x1, double x2) {
  return (float)gj_side<double>(md[0], md[1], md[2], x0, x1, x2);
}

__device__ __forceinline__ float step_factor32(float err, bool accepted, bool no_growth) {
  float fac = (err > 0.0f) ? 0.9f * exp2f(-0.2f * log2f(err)) : 5.0f;
  fac = fminf(5.0f, fmaxf(0.2f, fac));
  if (!accepted || no_growth) fac = fminf(fac, 1.0f);
  return fac;
}

// Hairer's initial step, on the full derivative f = (2k + c, dk/dl).
__device__ float initial_step32(const RayConst<float>& c, const double* md, const double* yd,
                                const float* f0c, float rtol, float atol) {
  float y0[6];
#pragma unroll
  for (int i = 0; i < 6; ++i) y0[i] = (float)yd[i];
  float f0[6], dnf = 0.0f, dny = 0.0f;
#pragma unroll
  for (int i = 0; i < 3; ++i) {
    f0[i] = 2.0f * y0[3 + i] + f0c[i];
    f0[3 + i] = f0c[3 + i];
  }
#pragma unroll
  for (int i = 0; i < 6; ++i) {
    const float sk = atol + rtol * fabsf(y0[i]);
    dnf += (f0[i] / sk) * (f0[i] / sk);
    dny += (y0[i] / sk) * (y0[i] / sk);
  }
  float h = (dnf <= 1e-10f || dny <= 1e-10f) ? 1e-6f : sqrtf(dny / dnf) * 0.01f;
  float y1[6], f1c[6];
  double x1d[3];
#pragma unroll
  for (int i = 0; i < 6; ++i) y1[i] = y0[i] + h * f0[i];
#pragma unroll
  for (int i = 0; i < 3; ++i) x1d[i] = yd[i] + (double)(h * f0[i]);
  rhs32c(c, md, x1d, y1 + 3, f1c);
  float der2 = 0.0f;
#pragma unroll
  for (int i = 0; i < 6; ++i) {
    const float f1 = (i < 3) ? 2.0f * y1[3 + i] + f1c[i] : f1c[i];
    const float sk = atol + rtol * fabsf(y0[i]);
    der2 += ((f1 - f0[i]) / sk) * ((f1 - f0[i]) / sk);
  }
  der2 = sqrtf(der2) / h;
  const float der12 = fmaxf(fabsf(der2), sqrtf(dnf));
  const float h1 = (der12 <= 1e-15f) ? fmaxf(1e-6f, h * 1e-3f) : exp2f(0.2f * log2f(0.01f / der12));
  return fminf(100.0f * h, h1);
}

// The Goldreich-Julian angular factor F = 3 z (m.x) - m_z |x|^2 in
// double-float, rounded to FP32 at the end: next to the null cone it is a
// small difference of O(|x|^2) terms.
__device__ __forceinline__ float cone_F2(const DF* y, const DF* m) {
  const DF mx = m[0] * y[0] + m[1] * y[1] + m[2] * y[2];
  const DF r2 = y[0] * y[0] + y[1] * y[1] + y[2] * y[2];
  const DF F = (y[2] * mx) * 3.0f - m[2] * r2;
  return F.hi + F.lo;
}

// c(x, k) and dk/dl with the null-cone factor F given: at the state's FP32
// position xf (the rounding of the double-float state).
__device__ __forceinline__ void rhs32F(const RayConst<float>& c, float F, const float* xf,
                                       const float* kf, float* f) {
  const float r2 = xf[0] * xf[0] + xf[1] * xf[1] + xf[2] * xf[2];
  ham_rhs<float, true, true>(c, xf[0], xf[1], xf[2], kf[0], kf[1], kf[2], f[0], f[1], f[2], f[3],
                             f[4], f[5], F * __frcp_rn(r2));
}

struct LaneM {
  RayConst<float> c;
  DF m[3];             // magnetic axis in double-float (for the null-cone factor)
  DF y[6];             // state (x / R, k / m_a) in double-float; y[i].hi is its FP32 rounding
  float f0[6];         // (c, dk/dl) at y (first-same-as-last)
  float h;
  int na, nr;
  int noisy_rej;       // consecutive rejections on the FP32 noise floor
  bool last_rej;
  bool switching;      // the current attempt ends just past a null-cone crossing
  float h_resume;
  double R_km, ma_eV;
};

__device__ __forceinline__ int find_star_m(const TraceParams& p, int64_t i) {
  if (p.nstars <= 1) return 0;
  int lo = 0, hi = p.nstars - 1;
  while (lo < hi) {
    const int mid = (lo + hi + 1) >> 1;
    if (p.offsets[mid] <= i) lo = mid; else hi = mid - 1;
  }
  return lo;
}

__device__ void load_lane_m(const TraceParams& p, int64_t i, LaneM& L) {
  const StarDev& s = p.stars[find_star_m(p, i)];
  const int64_t n = p.n;
  L.R_km = s.R_km;
  L.ma_eV = s.ma_eV;
  const double iR = 1.0 / s.R_km, im = 1.0 / s.ma_eV;
  double yd[6], md[3];
#pragma unroll
  for (int c = 0; c < 3; ++c) {
    yd[c] = p.state[c * n + i] * iR;
    yd[3 + c] = p.state[(3 + c) * n + i] * im;
  }
  const double om = 1.0 + p.state[6 * n + i];
  double sp, cpsi;
  sincos(p.state[7 * n + i], &sp, &cpsi);
  L.c.rs = (float)s.rs_prop;
  L.c.cp = (float)s.cp;
  L.c.pa = (float)s.plasma_a;
  L.c.W2 = (float)(om * om);
  L.c.iW2 = (float)(1.0 / (om * om));
  md[0] = s.sin_tm * cpsi;
  md[1] = s.sin_tm * sp;
  md[2] = s.cos_tm;
  L.c.m0 = (float)md[0];
  L.c.m1 = (float)md[1];
  L.c.m2 = (float)md[2];
  L.c.disp = s.dispersion;
  L.c.plasma = s.plasma;
  L.c.sig = side_md(md, yd[0], yd[1], yd[2]);
  L.switching = false;
  L.h_resume = 0.0f;
  float kf[3];
#pragma unroll
  for (int c = 0; c < 3; ++c) kf[c] = (float)yd[3 + c];
  rhs32c(L.c, md, yd, kf, L.f0);
  L.h = initial_step32(L.c, md, yd, L.f0, (float)p.rtol, (float)p.atol);
#pragma unroll
  for (int c = 0; c < 6; ++c) L.y[c] = df_of(yd[c]);
#pragma unroll
  for (int c = 0; c < 3; ++c) L.m[c] = df_of(md[c]);
  L.na = 0;
  L.nr = 0;
  L.noisy_rej = 0;
  L.last_rej = false;
}

__device__ void store_lane_m(const TraceParams& p, int64_t i, const LaneM& L, int st) {
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

// Position on the continuous extension at fraction th of a step from the
// FP64 state y (FP64 large part + FP32 small part).
__device__ __forceinline__ void dense_x(const double* y, float h, float th, const float* sR,
                                        const float* r3, const float* r4, const float* r5,
                                        double* xd) {
#pragma unroll
  for (int i = 0; i < 3; ++i)
    xd[i] = y[i] + (double)th * 2.0 * (double)h * y[3 + i] +
            (double)(th * (sR[i] + (1.0f - th) * (r3[i] + th * (r4[i] + (1.0f - th) * r5[i]))));
}

// Observer of accepted steps (forward tracing needs none).
struct NoHookM {
  static constexpr bool active = false;
  __device__ __forceinline__ void on_accept(const LaneM&, const DF*, const float*, float, float,
                                            const float*,
                                            const float*, const float*, const float*,
                                            const float*, const float*, const float*,
                                            const float*, const float*) {}
};

// One attempted step.  Returns -1 to continue, RAY_PROMOTED to hand the ray to
// the FP64 pass, else the final status.  hook.on_accept sees every accepted
// step: its start (L.y) and end (yn) in double-float, the start in FP32 (yf), the step,
// the null-cone factor and its gradient at the start (F0, gF), and the FP32
// small parts of the continuous extension (position: sR, r3, r4, r5 about
// y + 2 h k th; momentum: dK, q3, q4, q5).
template <class Hook>
__device__ int advance_m(const TraceParams& p, LaneM& L, Hook& hook) {
  if (L.na >= p.max_steps || L.na + L.nr >= 4 * p.max_steps) return RAY_MAXSTEPS;
  const float rtol = (float)p.rtol, atol = (float)p.atol;
  float yf[6];
#pragma unroll
  for (int i = 0; i < 6; ++i) yf[i] = L.y[i].hi;
  float h = L.h;
  {
    // displacement of one step at most STEP_REACH x the distance to the centre
    float v2 = 0.0f, r2 = 0.0f;
#pragma unroll
    for (int i = 0; i < 3; ++i) {
      const float vi = 2.0f * yf[3 + i] + L.f0[i];
      v2 += vi * vi;
      r2 += yf[i] * yf[i];
    }
    if (h * h * v2 > (float)(STEP_REACH * STEP_REACH) * r2)
      h = (float)STEP_REACH * sqrtf(r2 / v2);
  }
  // stage derivatives: R (position, small part) and K (momentum), j = 1..7
  float R1[3], R2[3], R3[3], R4[3], R5[3], R6[3], R7[3];
  float K1[3], K2[3], K3[3], K4[3], K5[3], K6[3], K7[3];
#pragma unroll
  for (int i = 0; i < 3; ++i) {
    R1[i] = L.f0[i];
    K1[i] = L.f0[3 + i];
  }
  // null-cone factor F = 3 z (m.x) - m_z |x|^2 at the start in double-float
  // (a small difference of O(|x|^2) terms next to the cone); its gradient gF
  // and its derivative gL along the straight part 2 h k of the step only
  // multiply the step's displacement, FP32
  float F0 = 0.0f, gL = 0.0f, gF[3] = {0.0f, 0.0f, 0.0f};
  if (L.c.plasma == PLASMA_GJ) {
    F0 = cone_F2(L.y, L.m);
    const float mxf = L.c.m0 * yf[0] + L.c.m1 * yf[1] + L.c.m2 * yf[2];
    gF[0] = 3.0f * yf[2] * L.c.m0 - 2.0f * L.c.m2 * yf[0];
    gF[1] = 3.0f * yf[2] * L.c.m1 - 2.0f * L.c.m2 * yf[1];
    gF[2] = 3.0f * mxf + 3.0f * yf[2] * L.c.m2 - 2.0f * L.c.m2 * yf[2];
    gL = 2.0f * h * (gF[0] * yf[3] + gF[1] * yf[4] + gF[2] * yf[5]);
  }
  float t[6], f[6], dks[3], dx[3], xs[3];
#define RT_STAGE(Rout, Kout, cj, SUMR, SUMK)                                          \
  {                                                                                   \
    _Pragma("unroll") for (int i = 0; i < 3; ++i) {                                   \
      dks[i] = h * (SUMK);                                                            \
      dx[i] = 2.0f * h * (float)(cj) * yf[3 + i] + h * (SUMR);                        \
      xs[i] = yf[i] + dx[i];                                                          \
      t[3 + i] = yf[3 + i] + dks[i];                                                  \
    }                                                                                 \
    rhs32s(L.c, F0, gF, xs, dx, t + 3, f);                                            \
    _Pragma("unroll") for (int i = 0; i < 3; ++i) {                                   \
      Rout[i] = 2.0f * dks[i] + f[i];                                                 \
      Kout[i] = f[3 + i];                                                             \
    }                                                                                 \
  }
  RT_STAGE(R2, K2, 1.0 / 5.0, (float)DP::a21 * R1[i], (float)DP::a21 * K1[i]);
  RT_STAGE(R3, K3, 3.0 / 10.0, (float)DP::a31 * R1[i] + (float)DP::a32 * R2[i],
           (float)DP::a31 * K1[i] + (float)DP::a32 * K2[i]);
  RT_STAGE(R4, K4, 4.0 / 5.0,
           (float)DP::a41 * R1[i] + (float)DP::a42 * R2[i] + (float)DP::a43 * R3[i],
           (float)DP::a41 * K1[i] + (float)DP::a42 * K2[i] + (float)DP::a43 * K3[i]);
  RT_STAGE(R5, K5, 8.0 / 9.0,
           (float)DP::a51 * R1[i] + (float)DP::a52 * R2[i] + (float)DP::a53 * R3[i] +
               (float)DP::a54 * R4[i],
           (float)DP::a51 * K1[i] + (float)DP::a52 * K2[i] + (float)DP::a53 * K3[i] +
               (float)DP::a54 * K4[i]);
  RT_STAGE(R6, K6, 1.0,
           (float)DP::a61 * R1[i] + (float)DP::a62 * R2[i] + (float)DP::a63 * R3[i] +
               (float)DP::a64 * R4[i] + (float)DP::a65 * R5[i],
           (float)DP::a61 * K1[i] + (float)DP::a62 * K2[i] + (float)DP::a63 * K3[i] +
               (float)DP::a64 * K4[i] + (float)DP::a65 * K5[i]);
#undef RT_STAGE
  // 5th-order increments: small position part and momentum
  float sR[3], dK[3];
  DF yn[6];
#pragma unroll
  for (int i = 0; i < 3; ++i) {
    sR[i] = h * ((float)DP::b1 * R1[i] + (float)DP::b3 * R3[i] + (float)DP::b4 * R4[i] +
                 (float)DP::b5 * R5[i] + (float)DP::b6 * R6[i]);
    dK[i] = h * ((float)DP::b1 * K1[i] + (float)DP::b3 * K3[i] + (float)DP::b4 * K4[i] +
                 (float)DP::b5 * K5[i] + (float)DP::b6 * K6[i]);
    yn[i] = (L.y[i] + L.y[3 + i] * (2.0f * h)) + sR[i];
    yn[3 + i] = L.y[3 + i] + dK[i];
  }
  // stage 7 at the new point (first-same-as-last)
  float fn[6];
#pragma unroll
  for (int i = 0; i < 6; ++i) t[i] = yn[i].hi;
#pragma unroll
  for (int i = 0; i < 3; ++i) dx[i] = 2.0f * h * yf[3 + i] + sR[i];
  rhs32s(L.c, F0, gF, t, dx, t + 3, fn);
#pragma unroll
  for (int i = 0; i < 3; ++i) {
    R7[i] = 2.0f * dK[i] + fn[i];
    K7[i] = fn[3 + i];
  }
  // F at the step's end by the same expansion (the side test; the next step
  // starts from F in FP64, which settles a crossing this test missed)
  float Fend = 0.0f;
  if (L.c.plasma == PLASMA_GJ) {
    const float md = L.c.m0 * dx[0] + L.c.m1 * dx[1] + L.c.m2 * dx[2];
    const float dd = dx[0] * dx[0] + dx[1] * dx[1] + dx[2] * dx[2];
    Fend = F0 + (gL + (gF[0] * sR[0] + gF[1] * sR[1] + gF[2] * sR[2])) +
           (3.0f * dx[2] * md - L.c.m2 * dd);
  }
  // error estimate (sum_j e_j = 0 removes the 2 h k_n part) and its FP32 floor
  float s = 0.0f, snk = 0.0f;
#pragma unroll
  for (int i = 0; i < 6; ++i) {
    const bool xp = i < 3;
    const int c = xp ? i : i - 3;
    const float v1 = xp ? R1[c] : K1[c], v3 = xp ? R3[c] : K3[c], v4 = xp ? R4[c] : K4[c];
    const float v5 = xp ? R5[c] : K5[c], v6 = xp ? R6[c] : K6[c], v7 = xp ? R7[c] : K7[c];
    const float a1 = (float)DP::e1 * v1, a3 = (float)DP::e3 * v3, a4 = (float)DP::e4 * v4;
    const float a5 = (float)DP::e5 * v5, a6 = (float)DP::e6 * v6, a7 = (float)DP::e7 * v7;
    const float e = h * (a1 + a3 + a4 + a5 + a6 + a7);
    const float sc = atol + rtol * fmaxf(fabsf(yf[i]), fabsf(t[i]));
    s += (e / sc) * (e / sc);
    if (!xp) {
      const float nz = NOISE_C * EPS32 * fabsf(h) *
                       (fabsf(a1) + fabsf(a3) + fabsf(a4) + fabsf(a5) + fabsf(a6) + fabsf(a7));
      snk += (nz / sc) * (nz / sc);
    }
  }
  const float en = sqrtf(s / 6.0f);
  const bool noisy = sqrtf(snk / 6.0f) > NOISE_LIMIT;
  if (!isfinite(en)) {
    ++L.nr;
    L.h = h * 0.2f;
    L.last_rej = true;
    return (L.h < 1e-12f) ? RAY_PROMOTED : -1;    // FP64 decides
  }
  // continuous-extension pieces (small parts), for the event locations
  float r3[3], r4[3], r5[3];
  const bool gj = (L.c.plasma == PLASMA_GJ);
  const bool need_dense = (en <= 1.0f);
  if (need_dense) {
#pragma unroll
    for (int i = 0; i < 3; ++i) {
      r3[i] = h * R1[i] - sR[i];
      r4[i] = sR[i] - h * R7[i] - r3[i];
      r5[i] = h * ((float)DP::d1 * R1[i] + (float)DP::d3 * R3[i] + (float)DP::d4 * R4[i] +
                   (float)DP::d5 * R5[i] + (float)DP::d6 * R6[i] + (float)DP::d7 * R7[i]);
    }
  }
  if (en <= 1.0f && gj && !L.switching && L.c.sig * Fend < 0.0f) {
    // the step crossed the null cone: locate the crossing on the continuous
    // extension and redo the step to end just past it.  F along the step by
    // its expansion about the start, in FP32: with d(th) = th (2 h k + S(th))
    // (S the small parts), F = F0 + th gL + th gF.S(th) + 3 d_z (m.d) - m_z |d|^2,
    // F0 and gL from FP64; its rounding, ~eps32 (|F0| + |gL|), moves a
    // transverse crossing by ~eps32 in th, the resolution of th itself.
    const float sgn = L.c.sig;
    auto side_val = [&](float th) {
      float d[3], gS = 0.0f;
#pragma unroll
      for (int i = 0; i < 3; ++i) {
        const float Si = sR[i] + (1.0f - th) * (r3[i] + th * (r4[i] + (1.0f - th) * r5[i]));
        gS += gF[i] * Si;
        d[i] = th * (2.0f * h * yf[3 + i] + Si);
      }
      const float md = L.c.m0 * d[0] + L.c.m1 * d[1] + L.c.m2 * d[2];
      const float dd = d[0] * d[0] + d[1] * d[1] + d[2] * d[2];
      return sgn * (F0 + th * (gL + gS) + (3.0f * d[2] * md - L.c.m2 * dd));
    };
    float flo = sgn * F0, fhi = sgn * Fend;
    if (!(flo >= 0.0f)) flo = 0.0f;                 // the start is on its own side
    if (!(fhi < 0.0f)) fhi = -1e-30f;
    // plain Illinois to 2^-22 relative (well inside the 1e-6 overshoot), the
    // guarded form only if that stalls
    float lo = 0.0f, hi = 1.0f;
    illinois(side_val, lo, hi, flo, fhi, SEED_TOL32, 40);
    if (hi - lo > SEED_TOL32 * hi) lo = last_nonneg(side_val, flo, fhi, &hi, lo, hi);
    ++L.nr;
    if (lo < SWITCH_MIN_FRACTION_M) {
      L.c.sig = -L.c.sig;
      rhs32F(L.c, F0, yf, yf + 3, L.f0);
      L.h = h;
    } else {
      L.h_resume = h;
      L.h = h * lo * (1.0f + SWITCH_OVERSHOOT_M);
      L.switching = true;
    }
    return -1;
  }
  if (en <= 1.0f) {
    ++L.na;
    L.noisy_rej = 0;
    if (Hook::active) {
      float q3[3], q4[3], q5[3];
#pragma unroll
      for (int i = 0; i < 3; ++i) {
        q3[i] = h * K1[i] - dK[i];
        q4[i] = dK[i] - h * K7[i] - q3[i];
        q5[i] = h * ((float)DP::d1 * K1[i] + (float)DP::d3 * K3[i] + (float)DP::d4 * K4[i] +
                     (float)DP::d5 * K5[i] + (float)DP::d6 * K6[i] + (float)DP::d7 * K7[i]);
      }
      hook.on_accept(L, yn, yf, h, F0, gF, sR, r3, r4, r5, dK, q3, q4, q5);
    }
    // escape and capture tests in FP32 (a step that ends within rounding of
    // r_out escapes at its end point)
    const float rnew2f = t[0] * t[0] + t[1] * t[1] + t[2] * t[2];
    if (rnew2f >= (float)(p.r_out * p.r_out)) {
      // locate |x(th)| = r_out on the continuous extension: r_out^2 - |x(th)|^2
      // by its FP32 expansion about the start, c0 - 2 y.d - |d|^2 with
      // c0 = r_out^2 - |y|^2 from FP64 and d(th) = th (2 h k + S(th)); its
      // rounding moves the root by ~eps32 in th, the resolution of th
      const double ro2 = p.r_out * p.r_out;
      double y0d[6];
#pragma unroll
      for (int i = 0; i < 6; ++i) y0d[i] = df_d(L.y[i]);
      double c0d = ro2 - (y0d[0] * y0d[0] + y0d[1] * y0d[1] + y0d[2] * y0d[2]);
      if (!(c0d >= 0.0)) c0d = 0.0;
      const float c0 = (float)c0d;
      auto inside = [&](float th) {
        float d[3];
#pragma unroll
        for (int i = 0; i < 3; ++i)
          d[i] = th * (2.0f * h * yf[3 + i] +
                       (sR[i] + (1.0f - th) * (r3[i] + th * (r4[i] + (1.0f - th) * r5[i]))));
        return c0 - (2.0f * (yf[0] * d[0] + yf[1] * d[1] + yf[2] * d[2]) +
                     (d[0] * d[0] + d[1] * d[1] + d[2] * d[2]));
      };
      float flo = c0, fhi = inside(1.0f);
      if (!(fhi < 0.0f)) fhi = -1e-30f;
      float lo = 0.0f, hi = 1.0f;
      illinois(inside, lo, hi, flo, fhi, SEED_TOL32, 40);
      if (hi - lo > SEED_TOL32 * hi) lo = last_nonneg(inside, flo, fhi, &hi, lo, hi);
      const float th = 0.5f * (lo + hi);
      double xd[3];
      dense_x(y0d, h, th, sR, r3, r4, r5, xd);
#pragma unroll
      for (int i = 0; i < 3; ++i) {
        const float q3 = h * K1[i] - dK[i];
        const float q4 = dK[i] - h * K7[i] - q3;
        const float q5 = h * ((float)DP::d1 * K1[i] + (float)DP::d3 * K3[i] +
                              (float)DP::d4 * K4[i] + (float)DP::d5 * K5[i] +
                              (float)DP::d6 * K6[i] + (float)DP::d7 * K7[i]);
        L.y[3 + i] = L.y[3 + i] +
                     th * (dK[i] + (1.0f - th) * (q3 + th * (q4 + (1.0f - th) * q5)));
        L.y[i] = df_of(xd[i]);
      }
      return RAY_ESCAPED;
    }
#pragma unroll
    for (int i = 0; i < 6; ++i) L.y[i] = yn[i];
#pragma unroll
    for (int i = 0; i < 6; ++i) L.f0[i] = fn[i];
    if (rnew2f <= (float)(p.r_capture * p.r_capture)) return RAY_CAPTURED;
    if (gj && L.c.sig * Fend < 0.0f) {
      L.c.sig = -L.c.sig;             // past the cone: continue on the other side
      rhs32F(L.c, cone_F2(L.y, L.m), t, t + 3, L.f0);
    }
    if (L.switching) {
      L.h = L.h_resume;
      L.switching = false;
    } else {
      L.h = h * step_factor32(en, true, L.last_rej || noisy);
    }
    L.last_rej = false;
    return -1;
  }
  if (noisy && ++L.noisy_rej >= NOISY_REJECTIONS_TO_PROMOTE) return RAY_PROMOTED;
  if (!noisy) L.noisy_rej = 0;
  ++L.nr;
  L.h = h * step_factor32(en, false, L.last_rej);
  L.last_rej = true;
  return (L.h < 1e-12f) ? RAY_PROMOTED : -1;     // FP64 decides
}

__global__ void __launch_bounds__(256) trace_mixed_kernel(TraceParams p) {
  const int lane = threadIdx.x & 31;
  int64_t ray = -1;
  LaneM L;
  long long acc = 0, rej = 0, traced = 0, esc = 0, promoted = 0;
  if (p.ts && threadIdx.x == 0) atomicMin(p.ts, global_ns());
  // one pass over the rays, or COST_BUCKETS passes (cost-ordered claims: the
  // rays that start nearest the null cone first)
  const int64_t nq = p.order ? (int64_t)COST_BUCKETS * p.n : p.n;
  ClaimChunk ch;
  for (;;) {
    claim_items(p.queue, nq, p.refill_min, p.claim_size, ray, ch, [&](int64_t idx) -> int64_t {
      const int pass = p.order ? (int)(idx / p.n) : 0;
      const int64_t i = idx - (int64_t)pass * p.n;
      if (p.status[i] != RAY_READY ||
          (p.order && (cost_bucket(p.stars[find_star_m(p, i)], p.state, p.n, i) != pass ||
                       !status_still(p, i, RAY_READY))))
        return -1;
      load_lane_m(p, i, L);
      return i;
    });
    if (__ballot_sync(FULL, ray != -2) == 0) break;
    if (ray >= 0) {
      NoHookM nh;
      const int st = advance_m(p, L, nh);
      if (st >= 0) {
        store_lane_m(p, ray, L, st);
        if (p.ts && st != RAY_PROMOTED) atomicMax(p.ts + 1 + find_star_m(p, ray), global_ns());
        acc += L.na;
        rej += L.nr;
        if (st == RAY_PROMOTED) {
          promoted += 1;
        } else {
          traced += 1;
          esc += (st == RAY_ESCAPED);
        }
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
      promoted += __shfl_down_sync(FULL, promoted, o);
    }
    if (lane == 0) {
      atomicAdd((unsigned long long*)&p.counters[CTR_ACC], (unsigned long long)acc);
      atomicAdd((unsigned long long*)&p.counters[CTR_REJ], (unsigned long long)rej);
      atomicAdd((unsigned long long*)&p.counters[CTR_RAYS], (unsigned long long)traced);
      atomicAdd((unsigned long long*)&p.counters[CTR_ESC], (unsigned long long)esc);
      atomicAdd((unsigned long long*)&p.counters[CTR_PROMOTED], (unsigned long long)promoted);
    }
  }
}

// ---------------------------------------------------------------------------
// Backward image plane in mixed precision: the FP32-stage integrator above,
// the crossing search of rt_backward.cuh on the FP64 reconstruction of each
// accepted step's continuous extension (FP64 state + FP32 small parts), FP64
// bisection and FP64 contributions.  A pixel whose FP32 error estimate sits on
// the rounding floor is appended to a list and traced again from the plane by
// the FP64 kernel.

struct CrossingHookM {
  static constexpr bool active = true;
  bool on;              // false: a forward ray of a mixed batch (no crossing search)
  CrossingAcc acc;
  RayConst<double> c;   // the pixel's constants in FP64 (sig follows the lane's)
  __device__ void on_accept(const LaneM& L, const DF* yn, const float* yf, float h, float F0,
                            const float* gF, const float* sR, const float* r3, const float* r4,
                            const float* r5, const float* dK, const float* q3, const float* q4,
                            const float* q5) {
    if (!on) return;
    c.sig = (double)L.c.sig;
    // the screen from the step's own FP32 constants, null-cone factor and pieces
    Screen sc;
    sc.rs = L.c.rs;
    sc.cp = L.c.cp;
    sc.pa = L.c.pa;
    sc.iW2 = L.c.iW2;
    sc.m0 = L.c.m0;
    sc.m1 = L.c.m1;
    sc.m2 = L.c.m2;
    sc.sig = L.c.sig;
    sc.disp = L.c.disp;
    sc.plasma = L.c.plasma;
    sc.F0 = F0;
    sc.gF[0] = gF[0];
    sc.gF[1] = gF[1];
    sc.gF[2] = gF[2];
    float p2[6], p3[6], p4[6], p5[6];
#pragma unroll
    for (int i = 0; i < 3; ++i) {
      p2[i] = 2.0f * h * yf[3 + i] + sR[i];
      p3[i] = r3[i];
      p4[i] = r4[i];
      p5[i] = r5[i];
      p2[3 + i] = dK[i];
      p3[3 + i] = q3[i];
      p4[3 + i] = q4[i];
      p5[3 + i] = q5[i];
    }
    // FP64 points of the continuous extension: FP64 start and increment (from
    // the double-float states, formed only where the search needs a point),
    // FP32 small parts
    auto dense64 = [&](double th, double* yd, double* yp) {
      const double u = 1.0 - th;
#pragma unroll
      for (int i = 0; i < 6; ++i) {
        const double y0 = df_d(L.y[i]);
        const double Q3 = (double)p4[i] + u * (double)p5[i];
        const double Q2 = (double)p3[i] + th * Q3;
        const double Q1 = (df_d(yn[i]) - y0) + u * Q2;
        yd[i] = y0 + th * Q1;
        if (yp) yp[i] = Q1 + th * (u * (Q3 - th * (double)p5[i]) - Q2);
      }
    };
    // the start in FP64 only for the first step's resonance sign; the end
    // from the extension at th = 1 where the screen leaves its sign open
    double y0d[6];
    if (!acc.have_g) {
#pragma unroll
      for (int i = 0; i < 6; ++i) y0d[i] = df_d(L.y[i]);
    }
    acc.scan(c, acc.have_g ? nullptr : y0d, nullptr, sc, yf, p2, p3, p4, p5, dense64);
  }
};

// Returns the distance of the pixel's start point from the centre.
__device__ double load_pixel_m(const BackParams& bp, int64_t pix, LaneM& L, RayConst<double>& c,
                               float rtol, float atol) {
  double yd[6];
  pixel_init(bp, pix, yd, c);
  L.R_km = bp.s.R_km;
  L.ma_eV = bp.s.ma_eV;
  L.c.rs = (float)c.rs;
  L.c.cp = (float)c.cp;
  L.c.pa = (float)c.pa;
  L.c.W2 = (float)c.W2;
  L.c.iW2 = (float)c.iW2;
  const double md[3] = {c.m0, c.m1, c.m2};
  L.c.m0 = (float)c.m0;
  L.c.m1 = (float)c.m1;
  L.c.m2 = (float)c.m2;
  L.c.disp = c.disp;
  L.c.plasma = c.plasma;
  L.c.sig = (float)c.sig;
  L.switching = false;
  L.h_resume = 0.0f;
  float kf[3];
#pragma unroll
  for (int i = 0; i < 3; ++i) kf[i] = (float)yd[3 + i];
  rhs32c(L.c, md, yd, kf, L.f0);
  L.h = initial_step32(L.c, md, yd, L.f0, rtol, atol);
#pragma unroll
  for (int i = 0; i < 6; ++i) L.y[i] = df_of(yd[i]);
#pragma unroll
  for (int i = 0; i < 3; ++i) L.m[i] = df_of(md[i]);
  L.na = 0;
  L.nr = 0;
  L.noisy_rej = 0;
  L.last_rej = false;
  return sqrt(yd[0] * yd[0] + yd[1] * yd[1] + yd[2] * yd[2]);
}

__global__ void __launch_bounds__(256) backward_mixed_kernel(BackParams bp) {
  const int lane = threadIdx.x & 31;
  const int64_t npix = (int64_t)bp.nx * bp.ny;
  TraceParams tp;
  tp.rtol = bp.rtol;
  tp.atol = bp.atol;
  tp.r_out = 0.0;
  tp.lambda_max = 0.0;
  tp.r_capture = bp.r_capture;
  tp.max_steps = bp.max_steps;
  tp.ts = nullptr;
  tp.park = nullptr;
  int64_t pix = -1;
  LaneM L;
  CrossingHookM hk;
  hk.on = true;
  long long acc = 0, rej = 0, done = 0, esc = 0, nc = 0, promoted = 0, srch = 0;
  if (bp.ts && threadIdx.x == 0) atomicMin(bp.ts, global_ns());
  for (;;) {
    const bool need = (pix == -1);
    const unsigned mneed = __ballot_sync(FULL, need);
    if (mneed) {
      const int leader = __ffs(mneed) - 1;
      unsigned long long base = 0;
      if (lane == leader) base = atomicAdd(bp.queue, (unsigned long long)__popc(mneed));
      base = __shfl_sync(FULL, base, leader);
      if (need) {
        const int64_t idx = (int64_t)base + __popc(mneed & ((1u << lane) - 1u));
        if (idx >= npix) {
          pix = -2;
        } else {
          pix = idx;
          // escaped once back at the distance the ray started from
          tp.r_out = load_pixel_m(bp, idx, L, hk.c, (float)bp.rtol, (float)bp.atol);
          hk.acc.reset(&bp.s, bp.W, bp.Lc_cut);
        }
      }
    }
    if (__ballot_sync(FULL, pix != -2) == 0) break;
    if (pix >= 0) {
      const int st = advance_m(tp, L, hk);
      if (st >= 0) {
        acc += L.na;
        rej += L.nr;
        if (st == RAY_PROMOTED) {
          const unsigned long long k = atomicAdd(bp.promo_n, 1ull);
          if (k < (unsigned long long)npix) bp.promo[k] = (int32_t)pix;
          ++promoted;
        } else {
          bp.image[pix] = bp.img_scale * hk.acc.sum;
          if (bp.ts) atomicMax(bp.ts + 1, global_ns());
          bp.status[pix] = (uint8_t)st;
          if (bp.ncross) bp.ncross[pix] = hk.acc.ncross - hk.acc.ncut;
          done += 1;
          esc += (st == RAY_ESCAPED);
          nc += hk.acc.ncross - hk.acc.ncut;
          srch += hk.acc.nsearch;
        }
        pix = -1;
      }
    }
  }
  if (bp.counters) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
      acc += __shfl_down_sync(FULL, acc, o);
      rej += __shfl_down_sync(FULL, rej, o);
      done += __shfl_down_sync(FULL, done, o);
      esc += __shfl_down_sync(FULL, esc, o);
      nc += __shfl_down_sync(FULL, nc, o);
      srch += __shfl_down_sync(FULL, srch, o);
      promoted += __shfl_down_sync(FULL, promoted, o);
    }
    if (lane == 0) {
      atomicAdd((unsigned long long*)&bp.counters[CTR_ACC], (unsigned long long)acc);
      atomicAdd((unsigned long long*)&bp.counters[CTR_REJ], (unsigned long long)rej);
      atomicAdd((unsigned long long*)&bp.counters[CTR_RAYS], (unsigned long long)done);
      atomicAdd((unsigned long long*)&bp.counters[CTR_ESC], (unsigned long long)esc);
      atomicAdd((unsigned long long*)&bp.counters[CTR_CROSS], (unsigned long long)nc);
      atomicAdd((unsigned long long*)&bp.counters[CTR_SEARCH], (unsigned long long)srch);
      atomicAdd((unsigned long long*)&bp.counters[CTR_PROMOTED], (unsigned long long)promoted);
    }
  }
}

// Forward rays and backward pixels of a batch in one persistent launch, FP32
// stages: rays that reach the FP32 floor are left with status RAY_PROMOTED
// for the FP64 pass, pixels are listed for it (t.promo).
__global__ void __launch_bounds__(256) batch_mixed_kernel(TraceParams p, ImgTable t) {
  const int lane = threadIdx.x & 31;
  const int64_t nf = p.n;
  const int64_t total = nf + t.npix;
  TraceParams tp = p;          // r_out per item
  int64_t item = -1;           // -1: needs an item, -2: queue exhausted
  int64_t ray = 0, pix = 0, g = 0;
  int img = 0;
  bool isp = false;
  LaneM L;
  CrossingHookM hk;
  hk.on = false;
  long long acc = 0, rej = 0, done = 0, esc = 0, nc = 0, promoted = 0;
  if (p.ts && threadIdx.x == 0) atomicMin(p.ts, global_ns());
  ClaimChunk ch;
  for (;;) {
    claim_items(p.queue, total, p.refill_min, p.claim_size, item, ch,
                [&](int64_t idx) -> int64_t {
      if (idx < nf) {
        if (p.status[idx] != RAY_READY) return -1;
        isp = false;
        ray = idx;
        load_lane_m(tp, idx, L);
        tp.r_out = p.r_out;
        hk.on = false;
        return idx;
      }
      g = idx - nf;
      img = find_image(t, g);
      pix = g - t.off[img];
      const BackParams& bp = t.img[img];
      // escaped once back at the distance the ray started from
      tp.r_out = load_pixel_m(bp, pix, L, hk.c, (float)p.rtol, (float)p.atol);
      hk.on = true;
      hk.acc.reset(&bp.s, bp.W, bp.Lc_cut);
      isp = true;
      return idx;
    });
    if (__ballot_sync(FULL, item != -2) == 0) break;
    if (item >= 0) {
      const int st = advance_m(tp, L, hk);
      if (st >= 0) {
        acc += L.na;
        rej += L.nr;
        if (!isp) {
          store_lane_m(tp, ray, L, st);
          if (st == RAY_PROMOTED) {
            promoted += 1;
          } else {
            if (p.ts) atomicMax(p.ts + 1 + find_star_m(p, ray), global_ns());
            done += 1;
            esc += (st == RAY_ESCAPED);
          }
        } else if (st == RAY_PROMOTED) {
          const unsigned long long k = atomicAdd(t.promo_n, 1ull);
          if (k < (unsigned long long)t.npix) t.promo[k] = (int32_t)g;
          promoted += 1;
        } else {
          const BackParams& bp = t.img[img];
          bp.image[pix] = bp.img_scale * hk.acc.sum;
          bp.status[pix] = (uint8_t)st;
          if (bp.ncross) bp.ncross[pix] = hk.acc.ncross - hk.acc.ncut;
          if (t.ts) atomicMax(t.ts + img, global_ns());
          nc += hk.acc.ncross - hk.acc.ncut;
          done += 1;
          esc += (st == RAY_ESCAPED);
        }
        item = -1;
      }
    }
  }
  if (p.counters) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
      acc += __shfl_down_sync(FULL, acc, o);
      rej += __shfl_down_sync(FULL, rej, o);
      done += __shfl_down_sync(FULL, done, o);
      esc += __shfl_down_sync(FULL, esc, o);
      nc += __shfl_down_sync(FULL, nc, o);
      promoted += __shfl_down_sync(FULL, promoted, o);
    }
    if (lane == 0) {
      atomicAdd((unsigned long long*)&p.counters[CTR_ACC], (unsigned long long)acc);
      atomicAdd((unsigned long long*)&p.counters[CTR_REJ], (unsigned long long)rej);
      atomicAdd((unsigned long long*)&p.counters[CTR_RAYS], (unsigned long long)done);
      atomicAdd((unsigned long long*)&p.counters[CTR_ESC], (unsigned long long)esc);
      atomicAdd((unsigned long long*)&p.counters[CTR_CROSS], (unsigned long long)nc);
      atomicAdd((unsigned long long*)&p.counters[CTR_PROMOTED], (unsigned long long)promoted);
    }
  }
}

}  // namespace

cudaError_t launch_batch_mixed(const TraceParams& p, const ImgTable& t, int block,
                               int blocks_per_sm, cudaStream_t stream) {
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
    int occ = 0;
    e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, batch_mixed_kernel, block, 0);
    if (e != cudaSuccess) return e;
    blocks_per_sm = occ > 0 ? occ : 1;
  }
  const int64_t items = p.n + t.npix;
  int64_t grid = (int64_t)nsm * blocks_per_sm;
  const int64_t max_useful = (items + block - 1) / block;
  if (grid > max_useful) grid = max_useful;
  if (grid < 1) grid = 1;
  e = cudaMemsetAsync(p.queue, 0, sizeof(unsigned long long), stream);
  if (e != cudaSuccess) return e;
  batch_mixed_kernel<<<(unsigned)grid, block, 0, stream>>>(p, t);
  return cudaGetLastError();
}

cudaError_t launch_backward_mixed(const BackParams& bp, cudaStream_t stream) {
  int dev = 0, nsm = 0, occ = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return e;
  e = cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev);
  if (e != cudaSuccess) return e;
  const int block = 128;
  e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, backward_mixed_kernel, block, 0);
  if (e != cudaSuccess) return e;
  const int64_t npix = (int64_t)bp.nx * bp.ny;
  int64_t grid = (int64_t)nsm * (occ > 0 ? occ : 1);
  const int64_t max_useful = (npix + block - 1) / block;
  if (grid > max_useful) grid = max_useful;
  if (grid < 1) grid = 1;
  e = cudaMemsetAsync(bp.queue, 0, sizeof(unsigned long long), stream);
  if (e != cudaSuccess) return e;
  backward_mixed_kernel<<<(unsigned)grid, block, 0, stream>>>(bp);
  return cudaGetLastError();
}

cudaError_t occupancy_mixed(int block, int* occ) {
  return cudaOccupancyMaxActiveBlocksPerMultiprocessor(occ, trace_mixed_kernel, block, 0);
}

cudaError_t occupancy_batch_mixed(int block, int* occ) {
  return cudaOccupancyMaxActiveBlocksPerMultiprocessor(occ, batch_mixed_kernel, block, 0);
}

cudaError_t launch_trace_mixed(const TraceParams& p, int block, int blocks_per_sm,
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
    int occ = 0;
    e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, trace_mixed_kernel, block, 0);
    if (e != cudaSuccess) return e;
    blocks_per_sm = occ > 0 ? occ : 1;
  }
  const int64_t warps_needed = (p.n + 31) / 32;
  int64_t grid = (int64_t)nsm * blocks_per_sm;
  const int64_t max_useful = (warps_needed * 32 + block - 1) / block;
  if (grid > max_useful) grid = max_useful;
  if (grid < 1) grid = 1;
  e = cudaMemsetAsync(p.queue, 0, sizeof(unsigned long long), stream);
  if (e != cudaSuccess) return e;
  trace_mixed_kernel<<<(unsigned)grid, block, 0, stream>>>(p);
  return cudaGetLastError();
}

}  // namespace rtk
