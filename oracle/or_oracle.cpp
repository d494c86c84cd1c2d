// Oracle (test infrastructure only; never linked into the product path).
//
// A plain, slow FP64 CPU implementation of the forward ray-tracing method of
// "Generalized Ray Tracing for Axions in Astrophysical Plasmas" (McDonald &
// Witte): sampling of the resonant conversion surface and the per-ray power
// weight (Sec. 3-4, Eqs. AxionCollInt, ForwardTracingEquation1, PowerCurved,
// CPAnisoCurved, AngleDefAniso, GaussianDist), integration of Hamilton's
// equations (Eq. Hamilton with Eq. StrongBHam) to a large radius, binning of
// the escaped power on the sky and in frequency (Sec. 2.2), and the backward
// image-plane estimator (Sec. 2.1, Eq. BackPower, and the multiple level
// crossings of Sec. 5.1.3).  Only the tests, the smoke check and the CPU
// baseline of the benchmark load this library.
#include <atomic>
#include <cfloat>
#include <cmath>
#include <cstdint>
#include <cstring>
#include <thread>
#include <vector>

#include "or_dopri.hpp"
#include "or_model.hpp"

namespace orc {

enum {
  RAY_READY = 0, RAY_ESCAPED = 1, RAY_CAPTURED = 2, RAY_NO_ROOT = 3, RAY_MAXSTEPS = 4,
  RAY_NAN = 5, RAY_STIFF = 6, RAY_LAMBDA_END = 7
};

// Trace options vector layout (shared with the Python wrapper of the oracle).
// TO_CROSS_GRID selects the backward crossing search: 0 (default) the
// exhaustive search; n > 0 the plain sign test at n points per step with no
// extremum search (a comparison baseline for the tests, never the reference).
enum {
  TO_RTOL = 0, TO_ATOL, TO_R_OUT, TO_MAX_STEPS, TO_LAMBDA_MAX, TO_R_CAPTURE, TO_CROSS_GRID,
  TO_COUNT
};

struct TraceOpts {
  double rtol, atol, r_out, lambda_max, r_capture;
  long max_steps;
  int cross_grid;
};

inline TraceOpts make_opts(const double* t) {
  TraceOpts o;
  o.rtol = t[TO_RTOL];
  o.atol = t[TO_ATOL];
  o.r_out = t[TO_R_OUT];
  o.max_steps = (long)t[TO_MAX_STEPS];
  o.lambda_max = t[TO_LAMBDA_MAX];
  o.r_capture = t[TO_R_CAPTURE];
  o.cross_grid = (int)t[TO_CROSS_GRID];
  return o;
}

static inline double norm3(const double v[3]) {
  return std::sqrt(v[0] * v[0] + v[1] * v[1] + v[2] * v[2]);
}

// ---------------------------------------------------------------------------
// Axion speed at infinity.  Eq. GaussianDist gives the Maxwellian
// f ~ exp(-|k|^2 / k0^2); the speed x = |k_inf| / k0 then has density
// (4/sqrt(pi)) x^2 exp(-x^2) and CDF erf(x) - (2/sqrt(pi)) x exp(-x^2).
// Inverted by bisection; for u > 1/2 the complementary form
// erfc(x) + (2/sqrt(pi)) x exp(-x^2) = 1 - u is solved instead (1 - u is
// exact there), which keeps the tail well conditioned.  Eq. fa_approx's
// monochromatic option gives x = 1.
static double maxwell_speed(int fa_model, double u) {
  if (fa_model == FA_DELTA) return 1.0;
  const double c = 2.0 / std::sqrt(units::PI);
  const bool upper = u > 0.5;
  const double v = upper ? 1.0 - u : u;
  double lo = 0.0, hi = 30.0;
  for (int it = 0; it < 200; ++it) {
    double mid = 0.5 * (lo + hi);
    if (mid <= lo || mid >= hi) break;
    if (upper) {
      double Q = std::erfc(mid) + c * mid * std::exp(-mid * mid);   // decreasing
      if (Q > v) lo = mid; else hi = mid;
    } else {
      double F = std::erf(mid) - c * mid * std::exp(-mid * mid);    // increasing
      if (F < v) lo = mid; else hi = mid;
    }
  }
  return 0.5 * (lo + hi);
}

// ---------------------------------------------------------------------------
// Kinematic resonance (Sec. 2.4 and Sec. 4: k^a_mu = k^gamma_mu).  Along the
// radial line through direction n, with the orthonormal-frame direction khat
// of the momentum and the Killing energy omega_inf = -k_t held fixed, the
// axion has local |k|^2 = omega_inf^2 / A(r) - m_a^2 and energy
// E_a = omega_inf / sqrt(A); the photon with the same k has the LO energy.
// h(r) = E_gamma - E_a vanishes on the leaf of the foliation of Eq.
// Hypersurfaces that this (khat, omega_inf) selects.
template <class T>
static T resonance_h(const Star& s, const double m[3], const double n[3], const double khat[3],
                     double omega_inf, T r, T* E_out = nullptr, T* K2_out = nullptr,
                     T* wp2_out = nullptr, T* cos2_out = nullptr) {
  T A = 1.0 - s.rs / r;
  T K2 = omega_inf * omega_inf / A - 1.0;  // local axion |k|^2 / m_a^2
  T Ea = sqrt(1.0 + K2);
  T x[3] = {r * n[0], r * n[1], r * n[2]};
  T wp2 = plasma_freq2(s, m, x);
  T B[3];
  dipole_field(m, x, B);
  T Bn = sqrt(B[0] * B[0] + B[1] * B[1] + B[2] * B[2]);
  T kb = (khat[0] * B[0] + khat[1] * B[1] + khat[2] * B[2]) / Bn;
  T cos2 = kb * kb;
  T Eg = photon_energy(s.dispersion, K2, wp2, cos2);
  if (E_out) *E_out = Ea;
  if (K2_out) *K2_out = K2;
  if (wp2_out) *wp2_out = wp2;
  if (cos2_out) *cos2_out = cos2;
  return Eg - Ea;
}

// h = E_gamma - E_a at a point x (units of R) of the leaf selected by (khat,
// omega_inf): the local axion momentum is |k| khat with |k|^2 = omega_inf^2 / A
// - m_a^2 there.  Its gradient (dual numbers over x) is the normal of the
// conversion surface.
template <class T>
static T resonance_h_at(const Star& s, const double m[3], const double khat[3],
                        double omega_inf, const T x[3]) {
  T r = sqrt(x[0] * x[0] + x[1] * x[1] + x[2] * x[2]);
  T A = 1.0 - s.rs / r;
  T K2 = omega_inf * omega_inf / A - 1.0;
  T Ea = sqrt(1.0 + K2);
  T wp2 = plasma_freq2(s, m, x);
  T B[3];
  dipole_field(m, x, B);
  T Bn = sqrt(B[0] * B[0] + B[1] * B[1] + B[2] * B[2]);
  T kb = (khat[0] * B[0] + khat[1] * B[1] + khat[2] * B[2]) / Bn;
  return photon_energy(s.dispersion, K2, wp2, kb * kb) - Ea;
}

// Root of h on (1, inf) (units of R): h(1) > 0 is required (the photon is
// heavier than the axion at the surface); the bracket is widened by doubling
// until h < 0 and then bisected to the last representable digit.  h is
// monotone along the radial line for the Goldreich-Julian and the twisted
// profiles outside the surface, so the root is unique.
static bool resonance_root(const Star& s, const double m[3], const double n[3],
                           const double khat[3], double omega_inf, double* r_out) {
  double lo = 1.0;
  if (!(resonance_h<double>(s, m, n, khat, omega_inf, lo) > 0.0)) return false;
  double hi = 2.0;
  int it = 0;
  while (!(resonance_h<double>(s, m, n, khat, omega_inf, hi) < 0.0)) {
    lo = hi;
    hi *= 2.0;
    if (++it > 60) return false;
  }
  for (int k = 0; k < 400; ++k) {
    double mid = 0.5 * (lo + hi);
    if (mid <= lo || mid >= hi) break;
    if (resonance_h<double>(s, m, n, khat, omega_inf, mid) > 0.0) lo = mid; else hi = mid;
  }
  *r_out = 0.5 * (lo + hi);
  return true;
}

// ---------------------------------------------------------------------------
// One forward sample and its weight.  The power of Eq. PowerCurved, with the
// divergence of P_agamma cancelled against cos(theta_n) (Eq. AngleDefAniso,
// Eq. CPAnisoCurved), is the phase-space integral
//   P = int d^3k_loc int dV  A^{1/2} delta(E_gamma - E_a) Psi f_a ,
//   Psi = (pi/2) g^2 |B|^2 (E^4 sin^2 th_B / D) E,
//   D = cos^2 th_B w_p^2 (w_p^2 - 2E^2) + E^4,
// where dV is the proper volume, d^3k_loc the orthonormal-frame momentum
// volume, and A^{1/2} the time dilation dt -> sqrt|g_tt| dt (the A^{1/2}
// prefactor of sqrt|h_k|).  The isotropic plasma uses Psi = (pi/2) g^2 |B|^2
// sin^2 th_B E (Eq. ProbIsoCurved with its power of E made dimensionally
// consistent).  Samples: direction n uniform on the sphere, khat uniform on
// the sphere, |k_inf| from the Maxwellian, and the resonance root r* along n.
// Intermediate quantities of one sample (the tests evaluate the paper's
// uncollapsed Eq. PowerCurved from them).
enum {
  PT_OK = 0, PT_R, PT_N, PT_KHAT = PT_N + 3, PT_E = PT_KHAT + 3, PT_K2, PT_WP2, PT_COS2, PT_BMAG,
  PT_DHDR, PT_GRADH, PT_PSI = PT_GRADH + 3, PT_W1, PT_W, PT_A, PT_KINF, PT_OMEGA, PT_SHAPE,
  PT_COUNT
};

static void sample_one(const Star& s, const double u[6], long N, double st[8], double* w,
                       unsigned char* status, double* parts = nullptr) {
  using units::PI;
  const double ct = 1.0 - 2.0 * u[0];
  const double stt = std::sqrt(std::fmax(0.0, (1.0 - ct) * (1.0 + ct)));
  const double ph = 2.0 * PI * u[1];
  const double n[3] = {stt * std::cos(ph), stt * std::sin(ph), ct};
  const double ck = 1.0 - 2.0 * u[2];
  const double sk = std::sqrt(std::fmax(0.0, (1.0 - ck) * (1.0 + ck)));
  const double pk = 2.0 * PI * u[3];
  const double khat[3] = {sk * std::cos(pk), sk * std::sin(pk), ck};
  const double xs = maxwell_speed(s.fa_model, u[4]);
  const double kinf = xs * s.v0;                       // |k_inf| / m_a
  const double delta = kinf * kinf / (std::sqrt(1.0 + kinf * kinf) + 1.0);
  const double omega_inf = 1.0 + delta;                // omega_inf / m_a
  const double psi = (s.phase_mode == PHASE_UNIFORM) ? 2.0 * PI * u[5] : s.psi;
  double m[3];
  magnetic_axis(s, psi, m);
  for (int i = 0; i < 8; ++i) st[i] = 0.0;
  st[6] = delta;
  st[7] = psi;
  *w = 0.0;
  double r;
  if (!resonance_root(s, m, n, khat, omega_inf, &r)) {
    *status = RAY_NO_ROOT;
    return;
  }
  if (s.plasma == PLASMA_TWISTED) {
    // no conversion on open field lines (Sec. 6): the dipole field line through
    // the point, r / sin^2(theta) = L, reaches the light cylinder (L >= c / Omega)
    const double cos_t = n[0] * m[0] + n[1] * m[1] + n[2] * m[2];
    if (r / (1.0 - cos_t * cos_t) >= s.r_lc) {
      *status = RAY_NO_ROOT;
      return;
    }
  }
  // derivative dh/dr along the leaf (dual numbers)
  double E, K2, wp2, cos2;
  Dual<1> rd = Dual<1>::var(r, 0);
  Dual<1> hd = resonance_h<Dual<1>>(s, m, n, khat, omega_inf, rd);
  resonance_h<double>(s, m, n, khat, omega_inf, r, &E, &K2, &wp2, &cos2);
  const double dhdr = hd.d[0];                          // units m_a / R
  const double A = 1.0 - s.rs / r;
  const double kloc = std::sqrt(K2);
  const double sin2 = 1.0 - cos2;
  // field magnitude [eV^2]
  double x[3] = {r * n[0], r * n[1], r * n[2]};
  double B[3];
  dipole_field(m, x, B);
  const double Bmag = s.B0_eV2 * norm3(B);
  // Psi [eV^3]
  const double Ephys = E * s.ma_eV;
  double shape;
  if (s.dispersion == DISP_ISO) {
    shape = sin2;
  } else {
    const double D = cos2 * wp2 * (wp2 - 2.0 * E * E) + E * E * E * E;
    shape = E * E * E * E * sin2 / D;
  }
  const double Psi = 0.5 * PI * s.g_eV * s.g_eV * Bmag * Bmag * shape * Ephys;
  // Jacobians of the sample space (n, khat, |k_inf|) -> (x, k_loc):
  //   dV          = A^{-1/2} r^2 dr dOmega_n
  //   d^3k_loc    = (k_loc k_inf / A) d|k_inf| dOmega_k       (at fixed r)
  //   int dr delta(h(r)) = 1 / |dh/dr|
  //   f_a / pdf(|k_inf|) = n_inf / (4 pi k_inf^2)  (Maxwellian or delta)
  //   pdf(n) pdf(khat) = 1 / (4 pi)^2
  const double r_eV = r * s.R_inv_eV;                   // [eV^-1]
  const double kloc_eV = kloc * s.ma_eV, kinf_eV = kinf * s.ma_eV;
  const double dhdr_eV = std::fabs(dhdr) * s.ma_eV / s.R_inv_eV;  // [eV^2]
  const double vol = std::pow(A, -0.5) * r_eV * r_eV;
  const double mom = kloc_eV * kinf_eV / A;
  const double tdil = std::sqrt(A);
  const double fa_over_pdf = s.n_inf / (4.0 * PI * kinf_eV * kinf_eV);
  // the weight per unit of Psi (the conversion probability's numerator)
  const double W1 = vol * mom * tdil * fa_over_pdf / dhdr_eV * (4.0 * PI) * (4.0 * PI);
  const double EV2_W = units::EV_J / units::HBAR_EV_S;  // 1 eV^2 of power in W
  *w = W1 * Psi / (double)N * EV2_W;
  if (parts) {
    Dual<3> xd[3];
    for (int i = 0; i < 3; ++i) xd[i] = Dual<3>::var(x[i], i);
    Dual<3> hx = resonance_h_at<Dual<3>>(s, m, khat, omega_inf, xd);
    parts[PT_OK] = 1.0;
    parts[PT_R] = r;
    for (int i = 0; i < 3; ++i) {
      parts[PT_N + i] = n[i];
      parts[PT_KHAT + i] = khat[i];
      parts[PT_GRADH + i] = hx.d[i];
    }
    parts[PT_E] = E;
    parts[PT_K2] = K2;
    parts[PT_WP2] = wp2;
    parts[PT_COS2] = cos2;
    parts[PT_BMAG] = Bmag;
    parts[PT_DHDR] = dhdr;
    parts[PT_PSI] = Psi;
    parts[PT_W1] = W1;
    parts[PT_A] = A;
    parts[PT_KINF] = kinf;
    parts[PT_OMEGA] = omega_inf;
    parts[PT_SHAPE] = shape;
  }
  if (s.weight_mode == WEIGHT_UNIT_P || s.weight_mode == WEIGHT_RENORM) {
    // conversion probability set to one (Sec. 5.1, Fig. flatiso right panel):
    // divide by P_agamma = Psi / |k . dE| (Eq. CPAnisoCurved), with dE the
    // proper-frame gradient of h = E_gamma - E_a, the normal of the surface
    Dual<3> xd[3];
    for (int i = 0; i < 3; ++i) xd[i] = Dual<3>::var(x[i], i);
    Dual<3> hx = resonance_h_at<Dual<3>>(s, m, khat, omega_inf, xd);
    double g[3] = {hx.d[0], hx.d[1], hx.d[2]};           // d h / d(x/R), units m_a
    const double gn = g[0] * n[0] + g[1] * n[1] + g[2] * n[2];
    double kg = 0.0;                                      // khat . proper gradient
    for (int i = 0; i < 3; ++i) kg += khat[i] * (g[i] + (std::sqrt(A) - 1.0) * gn * n[i]);
    const double kdE = kloc_eV * std::fabs(kg) * s.ma_eV / s.R_inv_eV;   // [eV^3]
    *w = W1 * kdE / (double)N * EV2_W;
    if (s.weight_mode == WEIGHT_RENORM) {
      // Eq. reweight: R_i = (1 cm^-3 / n_a(r_i)) (m_a / |k_a(r_i)|) / sqrt(1 - r_s / r_i),
      // with the focused density of the monochromatic distribution (Sec. 4.3),
      // n_a = n_inf k_c / k0, k_c^2 = k0^2 + 2 G M m_a^2 / r
      const double hbarc_cm = units::HBARC_EV_KM * 1e5;
      const double per_cm3 = hbarc_cm * hbarc_cm * hbarc_cm;           // 1 cm^-3 in eV^3
      const double k0 = s.v0 * s.ma_eV;
      const double kc = std::sqrt(k0 * k0 + s.ma_eV * s.ma_eV * s.rs / r);
      const double n_a = s.n_inf * kc / k0;
      *w *= (per_cm3 / n_a) * (s.ma_eV / kloc_eV) / std::sqrt(A);
    }
  }
  // initial photon phase-space point: orthonormal k = |k| khat, covariant
  // Cartesian components k = k_o + (1/sqrt(A) - 1)(n.k_o) n
  double ko[3] = {kloc * khat[0], kloc * khat[1], kloc * khat[2]};
  double nko = n[0] * ko[0] + n[1] * ko[1] + n[2] * ko[2];
  for (int i = 0; i < 3; ++i) {
    st[i] = x[i] * s.R_km;
    st[3 + i] = (ko[i] + (1.0 / std::sqrt(A) - 1.0) * nko * n[i]) * s.ma_eV;
  }
  *status = RAY_READY;
  if (parts) parts[PT_W] = *w;
}

// ---------------------------------------------------------------------------
// Adaptive Dormand-Prince integration of one ray (scaled units), from
// lambda = 0 to the first of: r = r_out (located on the dense output),
// r <= r_capture, lambda = lambda_max (if > 0), max_steps accepted steps.
struct RayRHS {
  const Star* s;
  const double* m;
  double omega_inf;
  int sigma = 0;        // branch of the Goldreich-Julian density (0: |n_e|)
  long nev = 0;
  void operator()(const double y[6], double dy[6]) {
    rhs(*s, m, omega_inf, y, dy, sigma);
    ++nev;
  }
};

// The Goldreich-Julian density |2 Omega . B / e| has a kink on the null cone
// Omega . B = 0 (Eq. GJDensity): omega_p^2 is continuous there but its
// gradient, and so dk/dlambda, jumps.  An embedded error estimate cannot
// resolve a jump inside a step; the step controller would shrink the step to
// rtol-sized slivers at every crossing.  So each step integrates the smooth
// continuation of the side it starts on (sigma = sign(Omega . B)); when an
// accepted step ends on the other side, the crossing is located on the
// continuous extension, the step is redone to end just past it, and sigma is
// switched there.  This integrates the same piecewise-smooth equations.
constexpr double SWITCH_MIN_FRACTION = 1e-6;   // a crossing this close to the start switches at once
constexpr double SWITCH_OVERSHOOT = 1e-10;     // relative overshoot of the redone step

static double locate_switch(const double m[3], const double y[6], const double ynew[6],
                            const double K[7][6], double h, int sigma) {
  // largest th in [0, 1] with sigma * (Omega . B)(x(th)) >= 0, by bisection
  double lo = 0.0, hi = 1.0, yd[6];
  for (int it = 0; it < 200; ++it) {
    double mid = 0.5 * (lo + hi);
    if (mid <= lo || mid >= hi) break;
    dp5_dense(y, ynew, K, h, mid, yd);
    if (sigma * gj_branch(m, yd) >= 0) lo = mid; else hi = mid;
  }
  return lo;
}

// Called after every accepted step with the step's start and end, its stages
// (for the continuous extension) and the null-cone branch in use.
struct StepHook {
  virtual void on_step(const double y[6], const double ynew[6], const double K[7][6], double h,
                       int sigma) = 0;
  virtual ~StepHook() {}
};

// Largest displacement of one step, as a fraction of the distance to the centre.
constexpr double STEP_REACH = 0.5;

static int trace_ray(const Star& s, const double m[3], double omega_inf, double y[6],
                     const TraceOpts& o, long* nacc_out, long* nrej_out, double* lam_out,
                     StepHook* hook = nullptr) {
  RayRHS f{&s, m, omega_inf};
  const bool gj = (s.plasma == PLASMA_GJ);
  if (gj) f.sigma = gj_branch(m, y);
  double f0[6];
  f(y, f0);
  double lam = 0.0;
  double hmax = (o.lambda_max > 0.0) ? o.lambda_max : 1e30;
  double h = dp5_initial_step(f, y, f0, o.rtol, o.atol, hmax);
  long nacc = 0, nrej = 0;
  bool last_rej = false;
  bool switching = false;      // the current attempt ends just past a crossing
  double h_resume = 0.0;       // step size to resume with after the crossing
  int status = RAY_MAXSTEPS;
  double K[7][6], ynew[6], err[6];
  while (true) {
    if (nacc >= o.max_steps || nacc + nrej >= 4 * o.max_steps) { status = RAY_MAXSTEPS; break; }
    // A step may move the ray by at most half its distance from the centre:
    // far from the star the medium is nearly uniform and the error estimate
    // alone would let one step carry the ray across the star and its plasma,
    // which no stage of that step samples.
    const double v2 = f0[0] * f0[0] + f0[1] * f0[1] + f0[2] * f0[2];
    const double r2 = y[0] * y[0] + y[1] * y[1] + y[2] * y[2];
    if (h * h * v2 > STEP_REACH * STEP_REACH * r2) h = STEP_REACH * std::sqrt(r2 / v2);
    bool clipped = false;
    if (o.lambda_max > 0.0 && lam + h >= o.lambda_max) { h = o.lambda_max - lam; clipped = true; }
    dp5_step(f, y, f0, h, ynew, err, K);
    double en = dp5_error_norm(y, ynew, err, o.rtol, o.atol);
    if (!std::isfinite(en)) {
      ++nrej;
      h *= 0.2;
      last_rej = true;
      if (h < 1e-12) { status = RAY_NAN; break; }
      continue;
    }
    if (en <= 1.0) {
      if (gj && !switching && f.sigma * gj_branch(m, ynew) < 0) {
        // the accepted step crossed the null cone: end the step just past it
        double th = locate_switch(m, y, ynew, K, h, f.sigma);
        ++nrej;
        if (th < SWITCH_MIN_FRACTION) {
          f.sigma = -f.sigma;          // already at the cone: switch here
          f(y, f0);
        } else {
          h_resume = h;
          h = h * th * (1.0 + SWITCH_OVERSHOOT);
          switching = true;
        }
        continue;
      }
      ++nacc;
      if (hook) hook->on_step(y, ynew, K, h, f.sigma);
      double rnew = norm3(ynew);
      if (rnew >= o.r_out) {
        // locate |x(th)| = r_out on the continuous extension
        double lo = 0.0, hi = 1.0, yd[6];
        for (int it = 0; it < 200; ++it) {
          double mid = 0.5 * (lo + hi);
          if (mid <= lo || mid >= hi) break;
          dp5_dense(y, ynew, K, h, mid, yd);
          if (norm3(yd) < o.r_out) lo = mid; else hi = mid;
        }
        double th = 0.5 * (lo + hi);
        dp5_dense(y, ynew, K, h, th, yd);
        for (int i = 0; i < 6; ++i) y[i] = yd[i];
        lam += th * h;
        status = RAY_ESCAPED;
        break;
      }
      for (int i = 0; i < 6; ++i) { y[i] = ynew[i]; f0[i] = K[6][i]; }
      lam += h;
      if (rnew <= o.r_capture) { status = RAY_CAPTURED; break; }
      if (clipped) { status = RAY_LAMBDA_END; break; }
      if (gj && f.sigma * gj_branch(m, y) < 0) {
        f.sigma = -f.sigma;            // past the cone: continue on the other side
        f(y, f0);
      }
      if (switching) {
        h = h_resume;
        switching = false;
      } else {
        h *= dp5_step_factor(en, true, last_rej);
      }
      last_rej = false;
    } else {
      ++nrej;
      h *= dp5_step_factor(en, false, last_rej);
      last_rej = true;
      if (h < 1e-12) { status = RAY_STIFF; break; }
    }
  }
  *nacc_out = nacc;
  *nrej_out = nrej;
  if (lam_out) *lam_out = lam;
  return status;
}

// ---------------------------------------------------------------------------
// Forward tracing through a rigidly rotating magnetosphere (Eq. GJDensity with
// its cos(Omega t) kept during the flight; Eq. Hamilton for all four canonical
// pairs).  The same integrator and events as trace_ray on the eight-component
// state y = (x, k, t, k_t) of rhs_rotating; the null cone Omega . B = 0 now
// turns with the star, so its side is taken with the axis at the point's own t.

struct RotRHS {
  const Star* s;
  double psi0;
  int sigma = 0;
  void operator()(const double y[8], double dy[8]) { rhs_rotating(*s, psi0, y, dy, sigma); }
};

static int gj_branch_at(const Star& s, double psi0, const double y[8]) {
  double m[3];
  magnetic_axis(s, psi0 + s.omega_R * y[6], m);
  return gj_branch(m, y);
}

static int trace_ray_rotating(const Star& s, double psi0, double y[8], const TraceOpts& o,
                              long* nacc_out, long* nrej_out, double* lam_out) {
  RotRHS f{&s, psi0};
  const bool gj = (s.plasma == PLASMA_GJ);
  if (gj) f.sigma = gj_branch_at(s, psi0, y);
  double f0[8];
  f(y, f0);
  double lam = 0.0;
  double hmax = (o.lambda_max > 0.0) ? o.lambda_max : 1e30;
  double h = dp5_initial_step<8>(f, y, f0, o.rtol, o.atol, hmax);
  long nacc = 0, nrej = 0;
  bool last_rej = false, switching = false;
  double h_resume = 0.0;
  int status = RAY_MAXSTEPS;
  double K[7][8], ynew[8], err[8], yd[8];
  while (true) {
    if (nacc >= o.max_steps || nacc + nrej >= 4 * o.max_steps) { status = RAY_MAXSTEPS; break; }
    const double v2 = f0[0] * f0[0] + f0[1] * f0[1] + f0[2] * f0[2];
    const double r2 = y[0] * y[0] + y[1] * y[1] + y[2] * y[2];
    if (h * h * v2 > STEP_REACH * STEP_REACH * r2) h = STEP_REACH * std::sqrt(r2 / v2);
    bool clipped = false;
    if (o.lambda_max > 0.0 && lam + h >= o.lambda_max) { h = o.lambda_max - lam; clipped = true; }
    dp5_step(f, y, f0, h, ynew, err, K);
    double en = dp5_error_norm(y, ynew, err, o.rtol, o.atol);
    if (!std::isfinite(en)) {
      ++nrej;
      h *= 0.2;
      last_rej = true;
      if (h < 1e-12) { status = RAY_NAN; break; }
      continue;
    }
    if (en <= 1.0) {
      if (gj && !switching && f.sigma * gj_branch_at(s, psi0, ynew) < 0) {
        // the accepted step crossed the (turning) null cone: largest th whose
        // point is on the start side, by bisection on the continuous extension
        double lo = 0.0, hi = 1.0;
        for (int it = 0; it < 200; ++it) {
          double mid = 0.5 * (lo + hi);
          if (mid <= lo || mid >= hi) break;
          dp5_dense(y, ynew, K, h, mid, yd);
          if (f.sigma * gj_branch_at(s, psi0, yd) >= 0) lo = mid; else hi = mid;
        }
        ++nrej;
        if (lo < SWITCH_MIN_FRACTION) {
          f.sigma = -f.sigma;
          f(y, f0);
        } else {
          h_resume = h;
          h = h * lo * (1.0 + SWITCH_OVERSHOOT);
          switching = true;
        }
        continue;
      }
      ++nacc;
      double rnew = norm3(ynew);
      if (rnew >= o.r_out) {
        double lo = 0.0, hi = 1.0;
        for (int it = 0; it < 200; ++it) {
          double mid = 0.5 * (lo + hi);
          if (mid <= lo || mid >= hi) break;
          dp5_dense(y, ynew, K, h, mid, yd);
          if (norm3(yd) < o.r_out) lo = mid; else hi = mid;
        }
        double th = 0.5 * (lo + hi);
        dp5_dense(y, ynew, K, h, th, yd);
        for (int i = 0; i < 8; ++i) y[i] = yd[i];
        lam += th * h;
        status = RAY_ESCAPED;
        break;
      }
      for (int i = 0; i < 8; ++i) { y[i] = ynew[i]; f0[i] = K[6][i]; }
      lam += h;
      if (rnew <= o.r_capture) { status = RAY_CAPTURED; break; }
      if (clipped) { status = RAY_LAMBDA_END; break; }
      if (gj && f.sigma * gj_branch_at(s, psi0, y) < 0) {
        f.sigma = -f.sigma;
        f(y, f0);
      }
      if (switching) {
        h = h_resume;
        switching = false;
      } else {
        h *= dp5_step_factor(en, true, last_rej);
      }
      last_rej = false;
    } else {
      ++nrej;
      h *= dp5_step_factor(en, false, last_rej);
      last_rej = true;
      if (h < 1e-12) { status = RAY_STIFF; break; }
    }
  }
  *nacc_out = nacc;
  *nrej_out = nrej;
  if (lam_out) *lam_out = lam;
  return status;
}

// ---------------------------------------------------------------------------
// Backward image-plane estimator (Sec. 2.1, Eq. BackPower; every level
// crossing along the worldline contributes, Sec. 5.1.3).
//
// Liouville's theorem carries the forward phase-space integral
//   P = int d^3x d^3k j,   j = sqrt(A) delta(E_gamma - E_a) Psi f_a
// (the integrand behind the forward weights) to the asymptotic phase space of
// the photons crossing a distant plane in direction Omega, where
// d^3x d^3k = dA dt omega^2 domega dOmega in vacuum.  Hence
//   dP/dOmega = int dA int domega omega^2 int_ray j dt,
// and the ray integral of the delta function is a sum over the crossings of
// g = E_gamma - E_a = 0 (the photon on shell meets the axion shell
// omega^2 - |k|^2 = m_a^2 with the same k_mu):
//   int_ray j dt = sum_c sqrt(A) Psi f_a |dt/dl| / |dg/dl|.
// The line is narrow (width ~ v0^2), so the rays are traced at its centre
// omega_0 = m_a sqrt(1 + v0^2) and the frequency integral of f_a is analytic:
//   int domega omega^2 f_a = omega_0 n_inf / (2 pi^{3/2} k0)  (Maxwellian),
//                           omega_0 n_inf / (4 pi k0)         (monochromatic).
// Pixels are rectangles 2 b_max / nx by 2 b_max / ny; each ray goes through a pixel
// centre perpendicular to the plane.  The time-reversed ray (k -> -k, same
// Hamiltonian, H even in k) is integrated inward from the plane.
// IR cut (Sec. 4.4, garbled there): L_c = E / |dE_gamma/ds - dE_a/ds| along the
// ray (a length); crossings with L_c > Lc_cut are dropped when Lc_cut > 0.

// g = E_gamma - E_a at a photon phase-space point (scaled units): omega from
// the Killing energy, the axion energy with the same k.
template <class T>
static T crossing_g(const Star& s, double omega_inf, const T x[3], const T k[3]) {
  T r = sqrt(x[0] * x[0] + x[1] * x[1] + x[2] * x[2]);
  T n[3] = {x[0] / r, x[1] / r, x[2] / r};
  T A = 1.0 - s.rs_prop / r;
  T omega = omega_inf / sqrt(A);
  T kn = n[0] * k[0] + n[1] * k[1] + n[2] * k[2];
  T kk = k[0] * k[0] + k[1] * k[1] + k[2] * k[2] + (A - 1.0) * kn * kn;   // g^{ij} k_i k_j
  return omega - sqrt(1.0 + kk);
}

struct BackwardAcc : StepHook {
  const Star* s;
  const double* m;
  double omega_inf;
  double Lc_cut;        // units of R (0: no cut)
  double sum = 0.0;     // sum over crossings of sqrt(A) Psi |dt/dl| / |dg/dl| [eV^2]
  int ncross = 0, ncut = 0;
  bool have_g = false;
  double g_prev = 0.0;

  double g_at(const double y[6]) const { return crossing_g<double>(*s, omega_inf, y, y + 3); }

  void contribution(const double y[6], int sigma) {
    using units::PI;
    // dg/dl = grad_y g . f(y)  (dual numbers, oracle RHS)
    typedef Dual<6> D;
    D xd[3], kd[3];
    for (int i = 0; i < 3; ++i) {
      xd[i] = D::var(y[i], i);
      kd[i] = D::var(y[3 + i], 3 + i);
    }
    D gd = crossing_g<D>(*s, omega_inf, xd, kd);
    double f[6];
    rhs(*s, m, omega_inf, y, f, sigma);
    double dg = 0.0;
    for (int i = 0; i < 6; ++i) dg += gd.d[i] * f[i];
    // dt/dl = dH/dk_t = -dH/d(omega_inf)
    Dual<1> w = Dual<1>::var(omega_inf, 0);
    Dual<1> xw[3], kw[3];
    for (int i = 0; i < 3; ++i) { xw[i] = Dual<1>(y[i]); kw[i] = Dual<1>(y[3 + i]); }
    Dual<1> Hw = hamiltonian(*s, m, w, xw, kw, sigma);
    const double dtdl = std::fabs(Hw.d[0]);
    // proper speed along the ray, for the conversion length
    const double r = norm3(y);
    const double n[3] = {y[0] / r, y[1] / r, y[2] / r};
    const double A = 1.0 - s->rs_prop / r;
    const double vn = n[0] * f[0] + n[1] * f[1] + n[2] * f[2];
    const double v2 = f[0] * f[0] + f[1] * f[1] + f[2] * f[2] + (1.0 / A - 1.0) * vn * vn;
    const double E = omega_inf / std::sqrt(A);                  // units of m_a
    const double Lc = E * std::sqrt(v2) / std::fabs(dg);        // units of R
    ++ncross;
    if (Lc_cut > 0.0 && Lc > Lc_cut) { ++ncut; return; }
    // Psi at the crossing
    const double wp2 = plasma_freq2<double>(*s, m, y);
    double B[3];
    dipole_field(m, y, B);
    const double Bn = norm3(B);
    const double kn = n[0] * y[3] + n[1] * y[4] + n[2] * y[5];
    double ko[3];
    for (int i = 0; i < 3; ++i) ko[i] = y[3 + i] + (std::sqrt(A) - 1.0) * kn * n[i];
    const double ko2 = ko[0] * ko[0] + ko[1] * ko[1] + ko[2] * ko[2];
    const double kb = (ko[0] * B[0] + ko[1] * B[1] + ko[2] * B[2]);
    const double cos2 = kb * kb / (ko2 * Bn * Bn);
    const double sin2 = 1.0 - cos2;
    double shape;
    if (s->dispersion == DISP_ISO) {
      shape = sin2;
    } else {
      const double Dd = cos2 * wp2 * (wp2 - 2.0 * E * E) + E * E * E * E;
      shape = E * E * E * E * sin2 / Dd;
    }
    const double Bmag = s->B0_eV2 * Bn;
    const double Psi = 0.5 * PI * s->g_eV * s->g_eV * Bmag * Bmag * shape * (E * s->ma_eV);
    // |dt/dl| / |dg/dl| in eV^-2: (R / m_a) x the scaled ratio
    const double ratio = dtdl / std::fabs(dg) * s->R_inv_eV / s->ma_eV;
    sum += std::sqrt(A) * Psi * ratio;
  }

  // Crossing search (every level crossing along the ray counts, Sec. 5.1.3).
  // Within one accepted step the ray is the continuous extension x(th), th in
  // [0, 1].  A crossing is a sign change of g(th).  A ray that grazes the
  // resonance crosses it twice in quick succession: g then has an extremum
  // between the two roots and may keep one sign at every sampled th.  So the
  // step is cut into NSEG equal pieces; on each piece the sign of dg/dth at its
  // ends (dual numbers through the continuous extension) brackets an extremum
  // of g, which is located by bisection on the sign of dg/dth.  Between
  // consecutive break points g is monotone, holds at most one root, and every
  // sign change there is located by bisection on the sign of g.  Only a piece
  // holding two extrema of g (1/NSEG of a step) can hide a pair of roots.
  static constexpr int NSEG = 32;
  int grid = 0;         // > 0: plain sign test at grid points, no extremum search

  // g and dg/dth at th on the step's continuous extension (the same
  // polynomial as dp5_dense, evaluated on a dual number in th)
  void g_slope(const double y[6], const double ynew[6], const double K[7][6], double h,
               double th, double* g, double* dg) const {
    typedef Dual<1> D1;
    const D1 t = D1::var(th, 0);
    D1 yd[6];
    for (int i = 0; i < 6; ++i) {
      const double r2 = ynew[i] - y[i];
      const double r3 = h * K[0][i] - r2;
      const double r4 = r2 - h * K[6][i] - r3;
      double dk = 0.0;
      for (int j = 0; j < 7; ++j) dk += DP5::d[j] * K[j][i];
      const double r5 = h * dk;
      yd[i] = y[i] + t * (r2 + (1.0 - t) * (r3 + t * (r4 + (1.0 - t) * r5)));
    }
    const D1 gd = crossing_g<D1>(*s, omega_inf, yd, yd + 3);
    *g = gd.v;
    *dg = gd.d[0];
  }

  // Locates the sign change of g on [lo, hi] (g(lo) < 0 iff negA) and adds
  // the crossing's contribution.
  void root(const double y[6], const double ynew[6], const double K[7][6], double h, double lo,
            double hi, bool negA, int sigma) {
    double yd[6];
    for (int it = 0; it < 200; ++it) {
      const double mid = 0.5 * (lo + hi);
      if (mid <= lo || mid >= hi) break;
      dp5_dense(y, ynew, K, h, mid, yd);
      if ((g_at(yd) < 0.0) == negA) lo = mid; else hi = mid;
    }
    dp5_dense(y, ynew, K, h, 0.5 * (lo + hi), yd);
    contribution(yd, sigma);
  }

  void on_step(const double y[6], const double ynew[6], const double K[7][6], double h,
               int sigma) override {
    if (!have_g) { g_prev = g_at(y); have_g = true; }
    double yd[6];
    if (grid > 0) {
      double th0 = 0.0, gA = g_prev;
      for (int q = 1; q <= grid; ++q) {
        const double th1 = (double)q / grid;
        double gB;
        if (q == grid) {
          gB = g_at(ynew);
        } else {
          dp5_dense(y, ynew, K, h, th1, yd);
          gB = g_at(yd);
        }
        if ((gA < 0.0) != (gB < 0.0)) root(y, ynew, K, h, th0, th1, gA < 0.0, sigma);
        th0 = th1;
        gA = gB;
      }
      g_prev = gA;
      return;
    }
    double gA = g_prev, sA, gdum;
    g_slope(y, ynew, K, h, 0.0, &gdum, &sA);
    for (int q = 1; q <= NSEG; ++q) {
      const double thA = (double)(q - 1) / NSEG, thB = (double)q / NSEG;
      double gB, sB;
      g_slope(y, ynew, K, h, thB, &gB, &sB);
      if (q == NSEG) gB = g_at(ynew);
      // break points of this piece: its ends and the extremum between them
      double th[3] = {thA, thB, thB}, gv[3] = {gA, gB, gB};
      int np = 2;
      if ((sA < 0.0) != (sB < 0.0)) {
        double lo = thA, hi = thB, gl, sl;
        const bool negS = sA < 0.0;
        for (int it = 0; it < 200; ++it) {
          const double mid = 0.5 * (lo + hi);
          if (mid <= lo || mid >= hi) break;
          g_slope(y, ynew, K, h, mid, &gl, &sl);
          if ((sl < 0.0) == negS) lo = mid; else hi = mid;
        }
        const double te = 0.5 * (lo + hi);
        dp5_dense(y, ynew, K, h, te, yd);
        th[1] = te;
        gv[1] = g_at(yd);
        np = 3;
      }
      for (int k = 1; k < np; ++k)
        if ((gv[k - 1] < 0.0) != (gv[k] < 0.0))
          root(y, ynew, K, h, th[k - 1], th[k], gv[k - 1] < 0.0, sigma);
      gA = gB;
      sA = sB;
    }
    g_prev = gA;
  }
};

static void backward_pixel(const Star& s, const TraceOpts& base, double incl, double D,
                           double bx, double by, double omega_inf, double Lc_cut_km,
                           double* value, unsigned char* status, int* ncross) {
  double m[3];
  magnetic_axis(s, s.psi, m);
  const double o[3] = {std::sin(incl), 0.0, std::cos(incl)};
  const double e1[3] = {std::cos(incl), 0.0, -std::sin(incl)};
  const double e2[3] = {0.0, 1.0, 0.0};
  double y[6];
  for (int i = 0; i < 3; ++i) y[i] = D * o[i] + bx * e1[i] + by * e2[i];
  // on-shell |k| along the orthonormal direction d = -o (time-reversed photon)
  const double r = norm3(y);
  const double n[3] = {y[0] / r, y[1] / r, y[2] / r};
  const double A = 1.0 - s.rs_prop / r;
  const double dn = -(n[0] * o[0] + n[1] * o[1] + n[2] * o[2]);
  auto Hs = [&](double sk) {
    double k[3];
    for (int i = 0; i < 3; ++i) k[i] = sk * (-o[i] + (1.0 / std::sqrt(A) - 1.0) * dn * n[i]);
    return hamiltonian<double>(s, m, omega_inf, y, k);
  };
  double lo = 0.0, hi = 4.0 * omega_inf;
  for (int it = 0; it < 300; ++it) {
    double mid = 0.5 * (lo + hi);
    if (mid <= lo || mid >= hi) break;
    if (Hs(mid) < 0.0) lo = mid; else hi = mid;
  }
  const double sk = 0.5 * (lo + hi);
  for (int i = 0; i < 3; ++i) y[3 + i] = sk * (-o[i] + (1.0 / std::sqrt(A) - 1.0) * dn * n[i]);
  TraceOpts opt = base;
  opt.r_out = r;                 // escaped once back at the plane's distance
  opt.lambda_max = 0.0;
  BackwardAcc acc;
  acc.s = &s;
  acc.m = m;
  acc.omega_inf = omega_inf;
  acc.Lc_cut = Lc_cut_km / s.R_km;
  acc.grid = base.cross_grid;
  long na, nr;
  double lam;
  *status = (unsigned char)trace_ray(s, m, omega_inf, y, opt, &na, &nr, &lam, &acc);
  *value = acc.sum;
  *ncross = acc.ncross - acc.ncut;
}

// Physical SoA state (rows: x[3] km, k[3] eV, delta, psi) <-> scaled ray.
static void load_ray(const Star& s, const double* state, long n, long i, double y[6],
                     double* omega_inf, double m[3]) {
  for (int c = 0; c < 3; ++c) {
    y[c] = state[c * n + i] / s.R_km;
    y[3 + c] = state[(3 + c) * n + i] / s.ma_eV;
  }
  *omega_inf = 1.0 + state[6 * n + i];
  magnetic_axis(s, state[7 * n + i], m);
}

static void store_ray(const Star& s, double* state, long n, long i, const double y[6]) {
  for (int c = 0; c < 3; ++c) {
    state[c * n + i] = y[c] * s.R_km;
    state[(3 + c) * n + i] = y[3 + c] * s.ma_eV;
  }
}

template <class F>
static void parallel_for(long n, int nthreads, F body) {
  if (nthreads <= 1 || n < 2) {
    for (long i = 0; i < n; ++i) body(i);
    return;
  }
  std::atomic<long> next(0);
  std::vector<std::thread> pool;
  for (int t = 0; t < nthreads; ++t)
    pool.emplace_back([&]() {
      for (;;) {
        long i = next.fetch_add(1);
        if (i >= n) break;
        body(i);
      }
    });
  for (auto& th : pool) th.join();
}

// Classical 4th-order Runge-Kutta with a fixed step (brute-force check).
static void rk4_fixed(const Star& s, const double m[3], double omega_inf, double y[6],
                      double lam_end, long nsteps) {
  RayRHS f{&s, m, omega_inf};
  const double h = lam_end / (double)nsteps;
  double k1[6], k2[6], k3[6], k4[6], t[6];
  for (long it = 0; it < nsteps; ++it) {
    f(y, k1);
    for (int i = 0; i < 6; ++i) t[i] = y[i] + 0.5 * h * k1[i];
    f(t, k2);
    for (int i = 0; i < 6; ++i) t[i] = y[i] + 0.5 * h * k2[i];
    f(t, k3);
    for (int i = 0; i < 6; ++i) t[i] = y[i] + h * k3[i];
    f(t, k4);
    for (int i = 0; i < 6; ++i) y[i] += h / 6.0 * (k1[i] + 2.0 * k2[i] + 2.0 * k3[i] + k4[i]);
  }
}

}  // namespace orc

using namespace orc;

extern "C" {

int or_version(void) { return 1; }

// Samples n conversion points.  u: SoA 6 x n uniforms in (0, 1).  state: SoA
// 8 x n (x km, k eV, delta, psi).  Returns the number of rays with a root.
long or_sample(const double* sp, long n, const double* u, double* state, double* weight,
               unsigned char* status, int nthreads) {
  Star s = make_star(sp);
  std::atomic<long> nroot(0);
  parallel_for(n, nthreads, [&](long i) {
    double ui[6], st[8];
    for (int c = 0; c < 6; ++c) ui[c] = u[c * n + i];
    sample_one(s, ui, n, st, &weight[i], &status[i]);
    for (int c = 0; c < 8; ++c) state[c * n + i] = st[c];
    if (status[i] == RAY_READY) nroot.fetch_add(1);
  });
  return nroot.load();
}

// The intermediate quantities of each sample (PT_COUNT doubles per sample,
// row-major n x PT_COUNT; PT_OK = 0 for samples without a root).
void or_sample_parts(const double* sp, long n, const double* u, double* parts, int nthreads) {
  Star s = make_star(sp);
  parallel_for(n, nthreads, [&](long i) {
    double ui[6], st[8], w;
    unsigned char status;
    for (int c = 0; c < 6; ++c) ui[c] = u[c * n + i];
    double* pi = parts + i * PT_COUNT;
    for (int c = 0; c < PT_COUNT; ++c) pi[c] = 0.0;
    sample_one(s, ui, n, st, &w, &status, pi);
  });
}

int or_sample_parts_count(void) { return PT_COUNT; }

// Traces every READY ray in place.  nacc / nrej / lam may be null.
void or_trace_forward(const double* sp, const double* topt, long n, double* state,
                      unsigned char* status, int* nacc, int* nrej, double* lam, int nthreads) {
  Star s = make_star(sp);
  TraceOpts o = make_opts(topt);
  parallel_for(n, nthreads, [&](long i) {
    if (status[i] != RAY_READY) {
      if (nacc) nacc[i] = 0;
      if (nrej) nrej[i] = 0;
      if (lam) lam[i] = 0.0;
      return;
    }
    double y[6], om, m[3];
    load_ray(s, state, n, i, y, &om, m);
    long na = 0, nr = 0;
    double l = 0.0;
    if (s.rotation == ROTATION_RIGID) {
      // the clock starts at the emission phase: t = 0, psi(0) = state row 7;
      // on return row 6 holds the final omega_inf / m_a - 1 = -k_t - 1 and
      // row 7 the rotation phase psi0 + Omega t at the end point
      const double psi0 = state[7 * n + i];
      double y8[8];
      for (int c = 0; c < 6; ++c) y8[c] = y[c];
      y8[6] = 0.0;
      y8[7] = -om;
      status[i] = (unsigned char)trace_ray_rotating(s, psi0, y8, o, &na, &nr, &l);
      for (int c = 0; c < 6; ++c) y[c] = y8[c];
      state[6 * n + i] = -y8[7] - 1.0;
      state[7 * n + i] = psi0 + s.omega_R * y8[6];
    } else {
      status[i] = (unsigned char)trace_ray(s, m, om, y, o, &na, &nr, &l);
    }
    store_ray(s, state, n, i, y);
    if (nacc) nacc[i] = (int)na;
    if (nrej) nrej[i] = (int)nr;
    if (lam) lam[i] = l;
  });
}

// The frequency-integrated axion phase-space density at the line centre,
// int domega omega^2 f_a [eV^3], and the traced omega_inf / m_a.
static double backward_fa(const Star& s, double* omega_inf) {
  using units::PI;
  const double v0 = s.v0;
  *omega_inf = std::sqrt(1.0 + v0 * v0);                       // line centre / m_a
  const double k0 = v0 * s.ma_eV, w0 = *omega_inf * s.ma_eV;   // [eV]
  return (s.fa_model == FA_DELTA) ? w0 * s.n_inf / (4.0 * PI * k0)
                                  : w0 * s.n_inf / (2.0 * std::pow(PI, 1.5) * k0);
}

// Backward image: ny x nx pixels (row-major, y index slow), value = the pixel's
// contribution to dP/dOmega [W / sr] (frequency integrated over the line),
// plus status and the number of crossings counted per pixel.  The star's
// fixed phase psi is used.
void or_trace_backward(const double* sp, const double* topt, int nx, int ny, double incl,
                       double dist_over_R, double bmax_over_R, double Lc_cut_km, double* image,
                       unsigned char* status, int* ncross, int nthreads) {
  Star s = make_star(sp);
  TraceOpts o = make_opts(topt);
  double omega_inf;
  const double Fa = backward_fa(s, &omega_inf);
  const double dbx = 2.0 * bmax_over_R / nx, dby = 2.0 * bmax_over_R / ny;   // units of R
  const double area_eV = (dbx * s.R_inv_eV) * (dby * s.R_inv_eV);          // [eV^-2]
  const double EV2_W = units::EV_J / units::HBAR_EV_S;
  parallel_for((long)nx * ny, nthreads, [&](long p) {
    const int i = (int)(p % nx), j = (int)(p / nx);
    const double bx = -bmax_over_R + (i + 0.5) * dbx;
    const double by = -bmax_over_R + (j + 0.5) * dby;
    double v;
    int nc;
    backward_pixel(s, o, incl, dist_over_R, bx, by, omega_inf, Lc_cut_km, &v, &status[p], &nc);
    image[p] = area_eV * Fa * v * EV2_W;
    if (ncross) ncross[p] = nc;
  });
}

// The backward integrand at arbitrary plane points (bx, by) = b[2i], b[2i+1]
// (units of R): dP/dOmega per unit plane area, [W / sr / R^2], so that a
// quadrature over the plane in units of R gives dP/dOmega.
void or_backward_points(const double* sp, const double* topt, long n, const double* b,
                        double incl, double dist_over_R, double Lc_cut_km, double* value,
                        unsigned char* status, int* ncross, int nthreads) {
  Star s = make_star(sp);
  TraceOpts o = make_opts(topt);
  double omega_inf;
  const double Fa = backward_fa(s, &omega_inf);
  const double unit = s.R_inv_eV * s.R_inv_eV * Fa * units::EV_J / units::HBAR_EV_S;
  parallel_for(n, nthreads, [&](long i) {
    double v;
    int nc;
    backward_pixel(s, o, incl, dist_over_R, b[2 * i], b[2 * i + 1], omega_inf, Lc_cut_km, &v,
                   &status[i], &nc);
    value[i] = unit * v;
    if (ncross) ncross[i] = nc;
  });
}

// Fixed-step RK4 from the given states over lambda in [0, lam_end[i]].
void or_trace_rk4(const double* sp, long n, double* state, const double* lam_end, long nsteps,
                  int nthreads) {
  Star s = make_star(sp);
  parallel_for(n, nthreads, [&](long i) {
    double y[6], om, m[3];
    load_ray(s, state, n, i, y, &om, m);
    rk4_fixed(s, m, om, y, lam_end[i], nsteps);
    store_ray(s, state, n, i, y);
  });
}

// H / m_a^2 and Hamilton's equations (scaled units: d(x/R)/dl, d(k/m_a)/dl)
// at each state column.
void or_hamiltonian(const double* sp, long n, const double* state, double* H, double* dydl) {
  Star s = make_star(sp);
  for (long i = 0; i < n; ++i) {
    double y[6], om, m[3];
    load_ray(s, state, n, i, y, &om, m);
    H[i] = hamiltonian<double>(s, m, om, y, y + 3);
    if (dydl) {
      double dy[6];
      rhs(s, m, om, y, dy);
      for (int c = 0; c < 6; ++c) dydl[c * n + i] = dy[c];
    }
  }
}

// omega_p^2 / m_a^2 at physical positions x (3 x n, km) for magnetic phase psi.
void or_plasma_freq2(const double* sp, long n, const double* x, double psi, double* out) {
  Star s = make_star(sp);
  double m[3];
  magnetic_axis(s, psi, m);
  for (long i = 0; i < n; ++i) {
    double xs[3] = {x[i] / s.R_km, x[n + i] / s.R_km, x[2 * n + i] / s.R_km};
    out[i] = plasma_freq2<double>(s, m, xs);
  }
}

// LO (or isotropic) photon energy for given |k|^2, omega_p^2, cos^2.
double or_photon_energy(int dispersion, double K2, double wp2, double cos2) {
  return photon_energy<double>(dispersion, K2, wp2, cos2);
}

// Inverse CDF of the Maxwellian speed (units of k0).
double or_maxwell_speed(int fa_model, double u) { return maxwell_speed(fa_model, u); }

// Resonance function and root along a radial line (units of R and m_a).
double or_resonance_h(const double* sp, const double* n, const double* khat, double omega_inf,
                      double psi, double r, double* dhdr) {
  Star s = make_star(sp);
  double m[3];
  magnetic_axis(s, psi, m);
  Dual<1> hd = resonance_h<Dual<1>>(s, m, n, khat, omega_inf, Dual<1>::var(r, 0));
  if (dhdr) *dhdr = hd.d[0];
  return hd.v;
}

int or_resonance_root(const double* sp, const double* n, const double* khat, double omega_inf,
                      double psi, double* r) {
  Star s = make_star(sp);
  double m[3];
  magnetic_axis(s, psi, m);
  return resonance_root(s, m, n, khat, omega_inf, r) ? 1 : 0;
}

// Derived star constants: [rs/R, omega_p^2(R, magnetic pole)/m_a^2 /2 (the
// coefficient of r^-3 |3 cos(th) m.n - cos(th_m)|), B0 in eV^2, R in eV^-1,
// n_inf in eV^3, GJ density coefficient Omega B0 / (e) in cm^-3].
void or_star_constants(const double* sp, double* out) {
  Star s = make_star(sp);
  out[0] = s.rs;
  out[1] = s.e_hl * s.omega_eV * s.B0_eV2 / units::ME_EV / (s.ma_eV * s.ma_eV);
  out[2] = s.B0_eV2;
  out[3] = s.R_inv_eV;
  out[4] = s.n_inf;
  const double hbarc_cm = units::HBARC_EV_KM * 1e5;
  out[5] = s.omega_eV * s.B0_eV2 / s.e_hl / (hbarc_cm * hbarc_cm * hbarc_cm);
}

// Sky / frequency histogram of ESCAPED rays.  Sky direction = orthonormal
// momentum direction at the end point; theta uniform on [0, pi] (nth bins),
// phi on [0, 2 pi) (nph bins); frequency variable y = delta / (v0^2 / 2) on
// [nu_lo, nu_hi) (nnu bins).  hist is nth x nph x nnu (row-major), in W per
// bin; out_of_range receives the weight with y outside the range.
void or_bin(const double* sp, long n, const double* state, const double* weight,
            const unsigned char* status, int nth, int nph, int nnu, double nu_lo, double nu_hi,
            double* hist, double* out_of_range) {
  Star s = make_star(sp);
  std::memset(hist, 0, sizeof(double) * (size_t)nth * nph * nnu);
  *out_of_range = 0.0;
  for (long i = 0; i < n; ++i) {
    if (status[i] != RAY_ESCAPED) continue;
    double x[3], k[3];
    for (int c = 0; c < 3; ++c) {
      x[c] = state[c * n + i] / s.R_km;
      k[c] = state[(3 + c) * n + i];
    }
    double r = norm3(x);
    double nn[3] = {x[0] / r, x[1] / r, x[2] / r};
    double A = 1.0 - s.rs_prop / r;
    double kn = nn[0] * k[0] + nn[1] * k[1] + nn[2] * k[2];
    double ko[3];
    for (int c = 0; c < 3; ++c) ko[c] = k[c] + (std::sqrt(A) - 1.0) * kn * nn[c];
    double kmag = norm3(ko);
    double cz = std::fmax(-1.0, std::fmin(1.0, ko[2] / kmag));
    double th = std::acos(cz);
    double ph = std::atan2(ko[1], ko[0]);
    if (ph < 0.0) ph += 2.0 * units::PI;
    int ith = (int)std::floor(th / (units::PI / nth));
    if (ith >= nth) ith = nth - 1;
    int iph = (int)std::floor(ph / (2.0 * units::PI / nph));
    if (iph >= nph) iph -= nph;
    double y = state[6 * n + i] / (0.5 * s.v0 * s.v0);
    if (!(y >= nu_lo && y < nu_hi)) { *out_of_range += weight[i]; continue; }
    int inu = (int)std::floor((y - nu_lo) / ((nu_hi - nu_lo) / nnu));
    if (inu >= nnu) inu = nnu - 1;
    hist[((size_t)ith * nph + iph) * nnu + inu] += weight[i];
  }
}

// The Dormand-Prince tableau as used above: c[7], a[7*6], b[7], bh[7], e[7], d[7].
void or_dp5_tableau(double* c, double* a, double* b, double* bh, double* e, double* d) {
  for (int i = 0; i < 7; ++i) {
    c[i] = DP5::c[i]; b[i] = DP5::b[i]; bh[i] = DP5::bh[i]; e[i] = DP5::e[i]; d[i] = DP5::d[i];
    for (int j = 0; j < 6; ++j) a[i * 6 + j] = DP5::a[i][j];
  }
}

// The same adaptive integrator (initial step, dp5_step, error norm,
// controller) on the linear test equation y' = M y, y in R^6, from 0 to T.
// Returns the number of accepted steps; y is overwritten by y(T).
long or_dp5_linear(const double* M, double* y, double T, double rtol, double atol) {
  struct Lin {
    const double* M;
    void operator()(const double v[6], double dv[6]) {
      for (int i = 0; i < 6; ++i) {
        double acc = 0.0;
        for (int j = 0; j < 6; ++j) acc += M[i * 6 + j] * v[j];
        dv[i] = acc;
      }
    }
  } f{M};
  double f0[6], K[7][6], ynew[6], err[6];
  f(y, f0);
  double t = 0.0, h = dp5_initial_step(f, y, f0, rtol, atol, T);
  long nacc = 0;
  bool last_rej = false;
  while (t < T && nacc < 10000000) {
    if (t + h > T) h = T - t;
    dp5_step(f, y, f0, h, ynew, err, K);
    double en = dp5_error_norm(y, ynew, err, rtol, atol);
    if (en <= 1.0) {
      for (int i = 0; i < 6; ++i) { y[i] = ynew[i]; f0[i] = K[6][i]; }
      t += h;
      ++nacc;
      h *= dp5_step_factor(en, true, last_rej);
      last_rej = false;
    } else {
      h *= dp5_step_factor(en, false, last_rej);
      last_rej = true;
    }
  }
  return nacc;
}

// One step of size h on y' = M y followed by the continuous extension at th.
void or_dp5_linear_dense(const double* M, const double* y0, double h, double th, double* out) {
  struct Lin {
    const double* M;
    void operator()(const double v[6], double dv[6]) {
      for (int i = 0; i < 6; ++i) {
        double acc = 0.0;
        for (int j = 0; j < 6; ++j) acc += M[i * 6 + j] * v[j];
        dv[i] = acc;
      }
    }
  } f{M};
  double f0[6], K[7][6], ynew[6], err[6];
  f(y0, f0);
  dp5_step(f, y0, f0, h, ynew, err, K);
  dp5_dense(y0, ynew, K, h, th, out);
}

}  // extern "C"
