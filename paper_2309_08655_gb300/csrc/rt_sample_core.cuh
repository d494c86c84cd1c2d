// Forward Monte-Carlo sampling of the resonant conversion surface: the
// per-sample computation shared by the sampling kernel (FP64) and the adjoint
// (dual numbers carrying derivatives with respect to the star parameters).
//
// Per sample (Sec. 3, Eqs. AxionCollInt and ForwardTracingEquation1; Sec. 4.2,
// Eq. PowerCurved; Sec. 4.3, Eq. GaussianDist): a direction n uniform on the
// sphere, a momentum direction khat uniform in the static orthonormal frame,
// the asymptotic axion speed from the Maxwellian, and the rotation phase.
// With khat and omega_inf = -k_t held fixed, the kinematic resonance
// k^a_mu = k^gamma_mu (Sec. 2.4, Sec. 4) on the radial line through n is the
// root of
//   G(r) = P(r) (1 + K2 s2) - (1 + K2),   K2(r) = omega_inf^2 / A(r) - 1,
// (units of m_a; s2 = sin^2 of the angle between khat and the dipole
// direction, constant along the line), obtained by substituting the axion's
// on-shell k into the anisotropic dispersion relation (Eq. AnisotrpoicDisp);
// G > 0 exactly where the LO photon is heavier than the axion.  For the
// isotropic plasma G = P - 1.
//
// Weight.  The power is the phase-space integral
//   P = int d^3k_loc dV sqrt(A) delta(E_gamma - E_a) Psi f_a,
//   Psi = (pi/2) g^2 |B|^2 (E^4 s2 / D) E,  D = c2 P (P - 2E^2) + E^4
// (Eq. PowerCurved with Eq. AngleDefAniso and Eq. CPAnisoCurved; isotropic:
// Psi = (pi/2) g^2 |B|^2 s2 E).  In the sample coordinates (n, khat, k_inf):
//   dV = A^{-1/2} r^2 dr dOmega_n,  d^3k_loc = (k k_inf / A) dk_inf dOmega_k,
//   int dr delta(h) = 1/|h'|,  f_a / pdf(k_inf) = n_inf / (4 pi k_inf^2),
// so W = 4 pi r^2 k n_inf Psi / (A k_inf |h'|), with h = E_gamma - E_a along the
// line and h' = G' / (2 E (E^2 - y_minus)), y_minus = K2 P c2 / E^2 the other
// root of the dispersion quadratic (isotropic: h' = P' / (2E)).
#pragma once
#include <cuda_runtime.h>
#include <stdint.h>

#include <type_traits>

#include "rt_device.cuh"
#include "rt_dual.cuh"

namespace rtk {
namespace sampling {

constexpr double TWO_OVER_SQRTPI = 1.12837916709551257390;

// Inverse CDF of the Maxwellian speed x = |k_inf| / k0, density
// (4/sqrt(pi)) x^2 exp(-x^2).  Lower half: erf(x) - c x e^{-x^2} = u; upper
// half: erfc(x) + c x e^{-x^2} = 1 - u (exact for u >= 1/2), which keeps the
// tail well conditioned.  Safeguarded Newton iteration.
// The start of the FP64 iteration: the same safeguarded Newton iteration in
// FP32 (FP32 exp, erf and erfc issue on the fast pipe) to ~1e-5.  Where FP32
// cannot resolve the equation (u below ~1e-8: erf(x) and x e^{-x^2} cancel) the
// FP64 iteration starts from a poor point and takes more steps, nothing else.
__device__ __forceinline__ float maxwell_seed(bool upper, float v) {
  const float c = (float)TWO_OVER_SQRTPI;
  float lo = 0.0f, hi = 30.0f;
  float x = 1.0876520317f;   // median
  for (int it = 0; it < 40; ++it) {
    const float ex = expf(-x * x);
    const float q = upper ? erfcf(x) + c * x * ex : erff(x) - c * x * ex;
    const float dq = 2.0f * c * x * x * ex * (upper ? -1.0f : 1.0f);
    const bool below = upper ? (q > v) : (q < v);
    if (below) lo = x; else hi = x;
    float xn = x - (q - v) / dq;
    if (!(xn > lo && xn < hi)) xn = 0.5f * (lo + hi);
    if (fabsf(xn - x) <= 1e-5f * x || hi - lo <= 1e-6f * hi) return xn;
    x = xn;
  }
  return x;
}

__device__ __forceinline__ double maxwell_speed(int fa_model, double u) {
  if (fa_model == FA_DELTA) return 1.0;
  const bool upper = u > 0.5;
  const double v = upper ? 1.0 - u : u;
  double lo = 0.0, hi = 30.0;
  double x = (double)maxwell_seed(upper, (float)v);
  if (!(x > lo && x < hi)) x = 1.0876520317;   // median
  for (int it = 0; it < 200; ++it) {
    const double ex = exp(-x * x);
    const double q = upper ? erfc(x) + TWO_OVER_SQRTPI * x * ex
                           : erf(x) - TWO_OVER_SQRTPI * x * ex;
    const double dq = 2.0 * TWO_OVER_SQRTPI * x * x * ex * (upper ? -1.0 : 1.0);
    // bracket update: the CDF increases with x, the tail decreases
    const bool below = upper ? (q > v) : (q < v);
    if (below) lo = x; else hi = x;
    double xn = x - (q - v) / dq;
    if (!(xn > lo && xn < hi)) xn = 0.5 * (lo + hi);
    // converged: a Newton step of a few ulps (one of exactly 1-2 ulps can
    // recur for ever where q - v is a rounding-level difference)
    if (fabs(xn - x) <= 1e-15 * x || hi - lo <= 4e-16 * hi) {
      x = xn;
      break;
    }
    x = xn;
  }
  return x;
}

struct Line {
  int disp, plasma;
  double rs, W2, s2, PR, pa, nz;
};

// P(r) and dP/dr along the radial line.
__device__ __forceinline__ void line_plasma(const Line& L, double r, double& P, double& dP) {
  switch (L.plasma) {
    case PLASMA_GJ: {
      const double ir = 1.0 / r;
      P = L.PR * ir * ir * ir;
      dP = -3.0 * P * ir;
      break;
    }
    case PLASMA_HOMOG: P = L.pa; dP = 0.0; break;
    case PLASMA_LINEAR_Z: P = L.pa * r * L.nz; dP = L.pa * L.nz; break;
    case PLASMA_RADIAL: {
      const double ir = 1.0 / r;
      P = L.pa * ir * ir * ir;
      dP = -3.0 * P * ir;
      break;
    }
    case PLASMA_TWISTED: {
      const double ir = 1.0 / r;
      P = L.PR * ir * ir * ir * ir;
      dP = -4.0 * P * ir;
      break;
    }
    default: P = 0.0; dP = 0.0; break;
  }
}

// G and G' in FP32 for the start of the FP64 root iteration; omega_inf^2 - 1
// (W2m1, a few 1e-6) is passed apart so that K2 keeps its FP32 precision.
__device__ __forceinline__ float line_G32(const Line& L, float W2m1, float r, float* dG) {
  const float ir = 1.0f / r;
  float P = 0.0f, dP = 0.0f;
  switch (L.plasma) {
    case PLASMA_GJ: P = (float)L.PR * ir * ir * ir; dP = -3.0f * P * ir; break;
    case PLASMA_HOMOG: P = (float)L.pa; break;
    case PLASMA_LINEAR_Z: P = (float)L.pa * r * (float)L.nz; dP = (float)(L.pa * L.nz); break;
    case PLASMA_RADIAL: P = (float)L.pa * ir * ir * ir; dP = -3.0f * P * ir; break;
    case PLASMA_TWISTED: P = (float)L.PR * ir * ir * ir * ir; dP = -4.0f * P * ir; break;
    default: break;
  }
  if (L.disp == DISP_ISO) {
    *dG = dP;
    return P - 1.0f;
  }
  const float rsr = (float)L.rs * ir;
  const float A = 1.0f - rsr;
  const float K2 = (W2m1 + rsr) / A;
  const float s2 = (float)L.s2;
  const float dK2 = -(1.0f + W2m1) * rsr * ir / (A * A);
  *dG = dP * (1.0f + K2 * s2) + P * s2 * dK2 - dK2;
  return P * (1.0f + K2 * s2) - (1.0f + K2);
}

__device__ __forceinline__ double line_G(const Line& L, double r, double* dG) {
  double P, dP;
  line_plasma(L, r, P, dP);
  if (L.disp == DISP_ISO) {
    if (dG) *dG = dP;
    return P - 1.0;
  }
  const double A = 1.0 - L.rs / r;
  const double K2 = L.W2 / A - 1.0;
  if (dG) {
    const double dK2 = -L.W2 * L.rs / (r * r * A * A);
    *dG = dP * (1.0 + K2 * L.s2) + P * L.s2 * dK2 - dK2;
  }
  return P * (1.0 + K2 * L.s2) - (1.0 + K2);
}


// Sample constants in the working type T: double for sampling, a dual number
// for the derivatives of the initial state and the weight with respect to the
// star parameters (the adjoint).  Only the fields a parameter can move are T.
template <class T>
struct SampConst {
  T rs, cp, sin_tm, cos_tm, B0_eV2, R_eV, n_inf, ma_eV;
  double v0, psi_fixed, plasma_a, g_eV, w_unit;
  double rlc;     // light-cylinder radius / R (twisted model: open field lines excluded)
  double per_cm3; // 1 cm^-3 in eV^3 (the renormalised weights)
  int disp, plasma, fa_model, phase_mode;
  int weight_mode;
};

template <class T>
struct SampOut {
  T x[3], k[3];   // scaled state: x / R, covariant k / m_a
  T w;            // weight [W]
  double delta, psi;
  bool ok;
};

__device__ __forceinline__ double val(double x) { return x; }
__device__ __forceinline__ double tabs(double x) { return fabs(x); }

// The root r of G as a function of the constants: G(r; c) = 0 gives
// dr = -dG_c / G_r (the value stays the one the bracketed iteration found).
__device__ __forceinline__ double root_of(double r, double /*G*/, double /*dGdr*/) { return r; }

template <class T>
__device__ __forceinline__ void line_plasma_t(int plasma, const T& PR, double pa, double nz,
                                              const T& r, T& P, T& dP) {
  switch (plasma) {
    case PLASMA_GJ: {
      const T ir = rt_rcp(r);
      P = PR * ir * ir * ir;
      dP = T(-3.0) * P * ir;
      break;
    }
    case PLASMA_HOMOG: P = T(pa); dP = T(0.0); break;
    case PLASMA_LINEAR_Z: P = T(pa) * r * T(nz); dP = T(pa * nz); break;
    case PLASMA_RADIAL: {
      const T ir = rt_rcp(r);
      P = T(pa) * ir * ir * ir;
      dP = T(-3.0) * P * ir;
      break;
    }
    case PLASMA_TWISTED: {
      const T ir = rt_rcp(r);
      P = PR * ir * ir * ir * ir;
      dP = T(-4.0) * P * ir;
      break;
    }
    default: P = T(0.0); dP = T(0.0); break;
  }
}

// Gradient of G (units 1/R) at the point x (units of R) of the leaf selected by
// (khat = q, W2 = omega_inf^2): the header's G with the angular factors and
// A evaluated at x itself (dual numbers over x).  Along the radial line it is
// G' of the root search; across it, the tilt of the conversion surface.
__device__ __forceinline__ void grad_G(const SampConst<double>& s, double m0, double m1,
                                       double m2, const double* q, double W2, const double* x,
                                       double* g) {
  typedef Dual<3> D3;
  D3 X[3];
#pragma unroll
  for (int i = 0; i < 3; ++i) X[i] = D3::var(x[i], i);
  const D3 r = rt_sqrt(X[0] * X[0] + X[1] * X[1] + X[2] * X[2]);
  const D3 ir = D3(1.0) / r;
  const D3 n0 = X[0] * ir, n1 = X[1] * ir, n2 = X[2] * ir;
  const D3 mu = D3(m0) * n0 + D3(m1) * n1 + D3(m2) * n2;
  const D3 A = D3(1.0) - D3(s.rs) * ir;
  const D3 K2 = D3(W2) / A - D3(1.0);
  D3 P(0.0);
  switch (s.plasma) {
    case PLASMA_GJ: P = D3(s.cp) * ir * ir * ir * dabs(D3(3.0) * n2 * mu - D3(m2)); break;
    case PLASMA_TWISTED: P = D3(s.cp) * (D3(1.0) - mu * mu) * ir * ir * ir * ir; break;
    case PLASMA_HOMOG: P = D3(s.plasma_a); break;
    case PLASMA_LINEAR_Z: P = D3(s.plasma_a) * X[2]; break;
    case PLASMA_RADIAL: P = D3(s.plasma_a) * ir * ir * ir; break;
    default: break;
  }
  D3 G;
  if (s.disp == DISP_ISO) {
    G = P - D3(1.0);
  } else {
    const D3 b0 = D3(3.0) * mu * n0 - D3(m0), b1 = D3(3.0) * mu * n1 - D3(m1),
             b2 = D3(3.0) * mu * n2 - D3(m2);
    const D3 kb = D3(q[0]) * b0 + D3(q[1]) * b1 + D3(q[2]) * b2;
    const D3 s2 = D3(1.0) - kb * kb / (D3(3.0) * mu * mu + D3(1.0));
    G = P * (D3(1.0) + K2 * s2) - (D3(1.0) + K2);
  }
#pragma unroll
  for (int i = 0; i < 3; ++i) g[i] = G.d[i];
}

// One sample from its six uniforms (the sample coordinates and the weight
// of the header comment).  inv_n: 1 / (number of samples).
template <class T>
__device__ void sample_core(const SampConst<T>& s, const double* u, double nsamp,
                            SampOut<T>& o) {
  // direction of the conversion point and of the momentum
  const double ct = 1.0 - 2.0 * u[0];
  const double st = sqrt(fmax(0.0, (1.0 - ct) * (1.0 + ct)));
  double sph, cph;
  sincospi(2.0 * u[1], &sph, &cph);
  const double n0 = st * cph, n1 = st * sph, n2 = ct;
  const double ck = 1.0 - 2.0 * u[2];
  const double sk = sqrt(fmax(0.0, (1.0 - ck) * (1.0 + ck)));
  double spk, cpk;
  sincospi(2.0 * u[3], &spk, &cpk);
  const double q0 = sk * cpk, q1 = sk * spk, q2 = ck;
  // asymptotic axion speed and the Killing energy omega_inf / m_a = 1 + delta
  const double xs = maxwell_speed(s.fa_model, u[4]);
  const double kinf = xs * s.v0;
  const double delta = kinf * kinf / (sqrt(1.0 + kinf * kinf) + 1.0);
  const double om = 1.0 + delta;
  const double psi = (s.phase_mode == PHASE_UNIFORM) ? 2.0 * PI * u[5] : s.psi_fixed;
  double sps, cps;
  sincos(psi, &sps, &cps);
  const T m0 = s.sin_tm * T(cps), m1 = s.sin_tm * T(sps), m2 = s.cos_tm;
  // dipole direction b = 3 (m.n) n - m (depends on n only)
  const T mu = m0 * T(n0) + m1 * T(n1) + m2 * T(n2);
  const T b0 = T(3.0) * mu * T(n0) - m0, b1 = T(3.0) * mu * T(n1) - m1,
          b2 = T(3.0) * mu * T(n2) - m2;
  const T bb = T(3.0) * mu * mu + T(1.0);
  const T kb = T(q0) * b0 + T(q1) * b1 + T(q2) * b2;
  const T c2 = kb * kb / bb;
  const T s2 = T(1.0) - c2;
  // the angular factor of P along the radial line: Goldreich-Julian
  // |3 n_z (m.n) - m_z|; twisted magnetosphere sin^2 of the magnetic colatitude
  const T PR = (s.plasma == PLASMA_TWISTED) ? s.cp * (T(1.0) - mu * mu)
                                            : s.cp * tabs(T(3.0) * T(n2) * mu - m2);
  Line L;
  L.disp = s.disp;
  L.plasma = s.plasma;
  L.rs = val(s.rs);
  L.W2 = om * om;
  L.s2 = val(s2);
  L.PR = val(PR);
  L.pa = s.plasma_a;
  L.nz = n2;
  o.delta = delta;
  o.psi = psi;
  o.ok = line_G(L, 1.0, nullptr) > 0.0;
  double lo = 1.0, hi = 2.0;
  if (o.ok) {
    int it = 0;
    while (!(line_G(L, hi, nullptr) < 0.0)) {
      lo = hi;
      hi *= 2.0;
      if (++it > 60) { o.ok = false; break; }
    }
  }
  if (!o.ok) return;
  // safeguarded Newton on G, from a start the same iteration finds in FP32
  double r = 0.5 * (lo + hi);
  {
    const float W2m1 = (float)(delta * (2.0 + delta));
    float flo = (float)lo, fhi = (float)hi, fr = (float)r;
    for (int it = 0; it < 40; ++it) {
      float dG;
      const float g = line_G32(L, W2m1, fr, &dG);
      if (g > 0.0f) flo = fr; else fhi = fr;
      float rn = fr - g / dG;
      if (!(rn > flo && rn < fhi)) rn = 0.5f * (flo + fhi);
      const bool done = fabsf(rn - fr) <= 1e-5f * fr || fhi - flo <= 1e-6f * fhi;
      fr = rn;
      if (done) break;
    }
    if ((double)fr > lo && (double)fr < hi) r = (double)fr;
  }
  for (int it = 0; it < 200; ++it) {
    double dG;
    const double g = line_G(L, r, &dG);
    if (g > 0.0) lo = r; else hi = r;
    double rn = r - g / dG;
    if (!(rn > lo && rn < hi)) rn = 0.5 * (lo + hi);
    const bool done = fabs(rn - r) <= 1e-15 * r || hi - lo <= 4e-16 * hi;
    r = rn;
    if (done) break;
  }
  // twisted magnetosphere: no conversion on open field lines, the dipole
  // lines r / sin^2(theta) = L that reach the light cylinder (L >= r_LC)
  if (s.plasma == PLASMA_TWISTED && r >= s.rlc * (1.0 - val(mu) * val(mu))) {
    o.ok = false;
    return;
  }
  // G in the working type at the root, for the root's dependence on the constants
  double dGr;
  line_G(L, r, &dGr);
  T rT;
  {
    T P, dP;
    line_plasma_t(s.plasma, PR, s.plasma_a, n2, T(r), P, dP);
    T G;
    if (s.disp == DISP_ISO) {
      G = P - T(1.0);
    } else {
      const T A = T(1.0) - s.rs * T(1.0 / r);
      const T K2 = T(L.W2) / A - T(1.0);
      G = P * (T(1.0) + K2 * s2) - (T(1.0) + K2);
    }
    rT = root_of(r, G, dGr);
  }
  // quantities at the resonance
  T P, dP;
  line_plasma_t(s.plasma, PR, s.plasma_a, n2, rT, P, dP);
  const T A = T(1.0) - s.rs / rT;
  const T K2 = T(L.W2) / A - T(1.0);
  const T E2 = T(1.0) + K2;
  const T E = rt_sqrt(E2);
  T dhdr, shape, hden;   // hden: dh = dG / hden
  if (s.disp == DISP_ISO) {
    dhdr = dP / (T(2.0) * E);
    hden = T(2.0) * E;
    shape = s2;
  } else {
    const T dK2 = -T(L.W2) * s.rs / (rT * rT * A * A);
    const T dG = dP * (T(1.0) + K2 * s2) + P * s2 * dK2 - dK2;
    const T ym = K2 * P * c2 / E2;
    dhdr = dG / (T(2.0) * E * (E2 - ym));
    hden = T(2.0) * E * (E2 - ym);
    const T D = c2 * P * (P - T(2.0) * E2) + E2 * E2;
    shape = E2 * E2 * s2 / D;
  }
  const T kloc = rt_sqrt(K2);
  const T ir = T(1.0) / rT;
  const T Bmag = s.B0_eV2 * T(0.5) * ir * ir * ir * rt_sqrt(bb);
  const T Psi = T(0.5 * PI * s.g_eV * s.g_eV) * Bmag * Bmag * shape * (E * s.ma_eV);
  const T r_eV = rT * s.R_eV;
  const T dh_eV = tabs(dhdr) * s.ma_eV / s.R_eV;
  // the weight per unit of Psi (the conversion probability's numerator)
  const T W1 = T(4.0 * PI) * r_eV * r_eV * (kloc / T(kinf)) * s.n_inf / (A * dh_eV);
  o.w = W1 * Psi / T(nsamp) * T(s.w_unit);
  if constexpr (std::is_same<T, double>::value) {
    if (s.weight_mode == WEIGHT_UNIT_P || s.weight_mode == WEIGHT_RENORM) {
      // conversion probability set to one (Sec. 5.1): divide by
      // P_agamma = Psi / |k . dE| (Eq. CPAnisoCurved), dE the proper-frame
      // gradient of h = E_gamma - E_a; dh = dG / (2 E (E^2 - y_minus)) (as h')
      const double q[3] = {q0, q1, q2};
      const double xr[3] = {rT * n0, rT * n1, rT * n2};
      double g[3];
      grad_G(s, m0, m1, m2, q, L.W2, xr, g);
      const double gn = g[0] * n0 + g[1] * n1 + g[2] * n2;
      const double sA = sqrt(A);
      double kg = 0.0;
#pragma unroll
      for (int i = 0; i < 3; ++i) {
        const double ni = (i == 0) ? n0 : (i == 1) ? n1 : n2;
        kg += q[i] * (g[i] + (sA - 1.0) * gn * ni);
      }
      const double kdE = kloc * s.ma_eV * fabs(kg / hden) * s.ma_eV / s.R_eV;   // [eV^3]
      o.w = W1 * kdE / nsamp * s.w_unit;
      if (s.weight_mode == WEIGHT_RENORM) {
        // Eq. reweight: x (1 cm^-3 / n_a(r)) (m_a / |k_a|) / sqrt(1 - r_s / r), the
        // focused density of the monochromatic distribution n_inf k_c / k0,
        // k_c^2 = k0^2 + m_a^2 r_s / r (Sec. 4.3)
        const double kc_over_k0 = sqrt(s.v0 * s.v0 + s.rs / rT) / s.v0;
        o.w *= (s.per_cm3 / (s.n_inf * kc_over_k0)) / kloc / sA;
      }
    }
  }
  // photon phase-space point: orthonormal k = |k| khat; covariant Cartesian
  // k = k_o + (1/sqrt(A) - 1) (n.k_o) n
  const T nko = kloc * T(n0 * q0 + n1 * q1 + n2 * q2);
  const T cr = (T(1.0) / rt_sqrt(A) - T(1.0)) * nko;
  o.x[0] = rT * T(n0);
  o.x[1] = rT * T(n1);
  o.x[2] = rT * T(n2);
  o.k[0] = kloc * T(q0) + cr * T(n0);
  o.k[1] = kloc * T(q1) + cr * T(n1);
  o.k[2] = kloc * T(q2) + cr * T(n2);
}

}  // namespace sampling
}  // namespace rtk
