// Oracle (test infrastructure only; never linked into the product path).
//
// The star, plasma and photon Hamiltonian of the paper, written literally:
//   * Schwarzschild metric, A = 1 - r_s/r, static plasma frame (Eq.
//     SchwarzshildMetric1 and the fluid velocity that follows it, Sec. 4.1),
//     expressed in Cartesianised coordinates x^i (r = |x|) so that the polar
//     axis is not a coordinate singularity: g^{ij} = delta^{ij} + (A-1) n^i n^j.
//   * Dipole field with surface polar strength B0 and magnetic axis m(psi),
//     Goldreich-Julian density n = 2 Omega.B / e (Eq. GJDensity, Sec. 5).
//   * Strong-field Hamiltonian H = g^{mu nu} k_mu k_nu
//     + (omega^2 - k_par^2) omega_p^2 / omega^2 (Eq. StrongBHam, Sec. 4.1), or
//     the isotropic one g^{mu nu} k_mu k_nu + omega_p^2 (Eq. DispIsotropic).
//   * The LO-mode energy (Eq. AnisotropicDisp, '+' root).
// Internally lengths are in units of the stellar radius R and momenta in units
// of the axion mass m_a; H then only changes by the constant factor m_a^2,
// which rescales the worldline parameter and leaves the rays unchanged.
#pragma once
#include <cmath>

#include "or_dual.hpp"

namespace orc {

namespace units {
constexpr double PI = 3.14159265358979323846;
constexpr double HBARC_EV_KM = 1.973269804e-10;  // hbar c [eV km], CODATA 2018
constexpr double HBAR_EV_S = 6.582119569e-16;     // hbar [eV s], CODATA 2018
constexpr double ALPHA = 7.2973525693e-3;         // fine-structure constant, CODATA 2018
constexpr double ME_EV = 510998.95;               // electron mass [eV], CODATA 2018
constexpr double EV_J = 1.602176634e-19;          // 1 eV in J (exact, SI 2019)
constexpr double C_KM_S = 299792.458;             // speed of light [km/s] (exact)
constexpr double GM_SUN_KM = 1.4766250;           // G M_sun / c^2 [km], IAU 2015 nominal
}  // namespace units

// Model switches (test models exist so that closed forms can pin the tracer).
enum { DISP_ANISO = 0, DISP_ISO = 1 };
enum {
  PLASMA_GJ = 0, PLASMA_VACUUM = 1, PLASMA_HOMOG = 2, PLASMA_LINEAR_Z = 3, PLASMA_RADIAL = 4,
  PLASMA_TWISTED = 5
};
enum { METRIC_FULL = 0, METRIC_FLAT = 1 };
enum { FA_MAXWELL = 0, FA_DELTA = 1 };
enum { WEIGHT_PAG = 0, WEIGHT_UNIT_P = 1, WEIGHT_RENORM = 2 };
enum { PHASE_FIXED = 0, PHASE_UNIFORM = 1 };
// Snapshot: the plasma frozen at the emission phase for the whole flight, so
// k_t is conserved (the reading of Sec. 5 used for every figure of the paper).
// Rigid: the magnetosphere keeps rotating while the photon flies (the time
// dependence that Eq. GJDensity writes through cos(Omega t)); k_t evolves.
enum { ROTATION_SNAPSHOT = 0, ROTATION_RIGID = 1 };

// Parameter vector layout shared with the Python wrapper of the oracle.
enum {
  SP_M_SUN = 0, SP_R_KM, SP_B0_G, SP_P_S, SP_THETA_M, SP_PSI, SP_MA_EV, SP_G_GEV,
  SP_RHO_GEV_CM3, SP_V0_KMS, SP_DISPERSION, SP_RESONANCE, SP_FA_MODEL, SP_WEIGHT_MODE,
  SP_PROP_METRIC, SP_PHASE_MODE, SP_PLASMA, SP_PLASMA_A, SP_ROTATION, SP_COUNT
};

struct Star {
  // physical inputs
  double M_sun, R_km, B0_G, P_s, theta_m, psi, ma_eV, g_GeV, rho, v0_kms;
  int dispersion, resonance, fa_model, weight_mode, prop_metric, phase_mode, plasma, rotation;
  double plasma_a;
  // derived
  double rs;        // r_s / R (geometry of the initial conditions)
  double rs_prop;   // r_s / R used in the propagation Hamiltonian
  double e_hl;      // electron charge in natural Heaviside-Lorentz units
  double omega_eV;  // rotation frequency hbar*Omega [eV]
  double B0_eV2;    // polar surface field [eV^2]
  double v0;        // axion velocity dispersion [c]
  double R_inv_eV;  // R in eV^-1
  double n_inf;     // asymptotic axion number density [eV^3]
  double g_eV;      // coupling [eV^-1]
  double r_lc;      // light-cylinder radius c / Omega, units of R
  double omega_R;   // Omega R / c: rotation rate per unit of t (t in units of R / c)
};

inline Star make_star(const double* p) {
  using namespace units;
  Star s;
  s.M_sun = p[SP_M_SUN]; s.R_km = p[SP_R_KM]; s.B0_G = p[SP_B0_G]; s.P_s = p[SP_P_S];
  s.theta_m = p[SP_THETA_M]; s.psi = p[SP_PSI]; s.ma_eV = p[SP_MA_EV]; s.g_GeV = p[SP_G_GEV];
  s.rho = p[SP_RHO_GEV_CM3]; s.v0_kms = p[SP_V0_KMS];
  s.dispersion = (int)p[SP_DISPERSION]; s.resonance = (int)p[SP_RESONANCE];
  s.fa_model = (int)p[SP_FA_MODEL]; s.weight_mode = (int)p[SP_WEIGHT_MODE];
  s.prop_metric = (int)p[SP_PROP_METRIC]; s.phase_mode = (int)p[SP_PHASE_MODE];
  s.plasma = (int)p[SP_PLASMA]; s.plasma_a = p[SP_PLASMA_A];
  s.rotation = (int)p[SP_ROTATION];
  s.rs = 2.0 * s.M_sun * GM_SUN_KM / s.R_km;
  s.rs_prop = (s.prop_metric == METRIC_FLAT) ? 0.0 : s.rs;
  s.e_hl = std::sqrt(4.0 * PI * ALPHA);
  s.omega_eV = HBAR_EV_S * 2.0 * PI / s.P_s;
  const double hbarc_cm = HBARC_EV_KM * 1e5;
  const double erg_eV = 1e-7 / EV_J;
  // B^2/2 (Heaviside-Lorentz) = B_G^2 / (8 pi) erg/cm^3, and 1 erg/cm^3 in eV^4:
  s.B0_eV2 = s.B0_G * std::sqrt(erg_eV * hbarc_cm * hbarc_cm * hbarc_cm / (4.0 * PI));
  s.v0 = s.v0_kms / C_KM_S;
  s.R_inv_eV = s.R_km / HBARC_EV_KM;
  s.n_inf = s.rho * 1e9 * hbarc_cm * hbarc_cm * hbarc_cm / s.ma_eV;
  s.g_eV = s.g_GeV * 1e-9;
  s.r_lc = C_KM_S * s.P_s / (2.0 * PI) / s.R_km;
  s.omega_R = 1.0 / s.r_lc;
  return s;
}

// Magnetic axis at rotation phase psi (misalignment theta_m from the z axis,
// which is the rotation axis; Sec. 5, below Eq. GJDensity).
template <class T>
inline void magnetic_axis(const Star& s, T psi, T m[3]) {
  m[0] = std::sin(s.theta_m) * cos(psi);
  m[1] = std::sin(s.theta_m) * sin(psi);
  m[2] = T(std::cos(s.theta_m));
}

// Dipole field in the static orthonormal frame, in units of B0, at the point
// x (units of R): B = (1/2) r^-3 [3 (m.n) n - m]; |B| = B0 at the magnetic pole
// of the surface.
template <class T, class M>
inline void dipole_field(const M m[3], const T x[3], T B[3]) {
  T r = sqrt(x[0] * x[0] + x[1] * x[1] + x[2] * x[2]);
  T n[3] = {x[0] / r, x[1] / r, x[2] / r};
  T mu = n[0] * m[0] + n[1] * m[1] + n[2] * m[2];
  T f = 0.5 / (r * r * r);
  for (int i = 0; i < 3; ++i) B[i] = f * (3.0 * mu * n[i] - m[i]);
}

// Sign of Omega . B at x (the Goldreich-Julian charge changes sign on the null
// cone Omega . B = 0, where |n_e| has a kink).
inline int gj_branch(const double m[3], const double x[3]) {
  double B[3];
  dipole_field(m, x, B);
  return B[2] < 0.0 ? -1 : 1;
}

// omega_p^2 / m_a^2 at x (units of R).  sigma = 0 evaluates |n_e|; sigma = +-1
// evaluates sigma * n_e, the smooth continuation of one side of the null cone
// (used inside an integration step, see trace_ray).
template <class T, class M>
inline T plasma_freq2(const Star& s, const M m[3], const T x[3], int sigma = 0) {
  switch (s.plasma) {
    case PLASMA_VACUUM: return T(0.0);
    case PLASMA_HOMOG: return T(s.plasma_a);
    case PLASMA_LINEAR_Z: return s.plasma_a * x[2];
    case PLASMA_RADIAL: {
      // spherical test profile a (R / r)^3
      T r2 = x[0] * x[0] + x[1] * x[1] + x[2] * x[2];
      return s.plasma_a / (r2 * sqrt(r2));
    }
    case PLASMA_TWISTED: {
      // twisted magnetar magnetosphere (Sec. 6, Eq. neMag): the current of a
      // globally twisted dipole, j = (psi sin^2 theta / r) B, with charge
      // multiplicity lambda over the minimal density 2|j|/e, and |B| taken as
      // B0 (R/r)^3:  n_e = lambda psi sin^2(theta) B0 (R/r)^3 / (e r),
      // theta the colatitude from the magnetic axis; omega_p^2 = e^2 n_e / m_e.
      T r = sqrt(x[0] * x[0] + x[1] * x[1] + x[2] * x[2]);
      T cos_t = (m[0] * x[0] + m[1] * x[1] + m[2] * x[2]) / r;
      T sin2 = 1.0 - cos_t * cos_t;
      T r_eV = r * s.R_inv_eV;                              // [eV^-1]
      T n_e = s.plasma_a * sin2 * s.B0_eV2 / (r * r * r) / (s.e_hl * r_eV);   // [eV^3]
      T wp2 = s.e_hl * s.e_hl * n_e / units::ME_EV;         // [eV^2]
      return wp2 / (s.ma_eV * s.ma_eV);
    }
    default: break;
  }
  // Goldreich-Julian: n_e = 2 |Omega . B| / e (Eq. GJDensity, charge sign
  // dropped), omega_p^2 = e^2 n_e / m_e (Heaviside-Lorentz natural units).
  T Bhat[3];
  dipole_field(m, x, Bhat);
  T omega_dot_B = s.omega_eV * Bhat[2] * s.B0_eV2;     // Omega along z
  T absOB = (sigma == 0) ? fabs(omega_dot_B) : double(sigma) * omega_dot_B;
  T n_e = 2.0 * absOB / s.e_hl;                       // [eV^3]
  T wp2 = s.e_hl * s.e_hl * n_e / units::ME_EV;       // [eV^2]
  return wp2 / (s.ma_eV * s.ma_eV);
}

// The photon Hamiltonian H(x, k) / m_a^2 with k_t = -omega_inf fixed (static
// snapshot of the plasma, so dk_t/dlambda = 0).
template <class T, class W = double, class M = double>
inline T hamiltonian(const Star& s, const M m[3], W omega_inf, const T x[3],
                     const T k[3], int sigma = 0) {
  T r = sqrt(x[0] * x[0] + x[1] * x[1] + x[2] * x[2]);
  T n[3] = {x[0] / r, x[1] / r, x[2] / r};
  T A = 1.0 - s.rs_prop / r;
  T omega2 = omega_inf * omega_inf / A;          // omega^2 = -g^{tt} k_t^2
  // |k|^2 = g^{ij} k_i k_j with g^{ij} = delta^{ij} + (A - 1) n^i n^j
  T kk = T(0.0);
  for (int i = 0; i < 3; ++i)
    for (int j = 0; j < 3; ++j) {
      T gij = (A - 1.0) * n[i] * n[j];
      if (i == j) gij = gij + 1.0;
      kk = kk + gij * k[i] * k[j];
    }
  T g_kk = kk - omega2;                          // g^{mu nu} k_mu k_nu
  T wp2 = plasma_freq2(s, m, x, sigma);
  if (s.dispersion == DISP_ISO) return g_kk + wp2;
  // components of k in the static orthonormal frame: radial sqrt(A) k_r,
  // tangential unchanged
  T kn = n[0] * k[0] + n[1] * k[1] + n[2] * k[2];
  T sA = sqrt(A);
  T ko[3];
  for (int i = 0; i < 3; ++i) ko[i] = k[i] + (sA - 1.0) * kn * n[i];
  T B[3];
  dipole_field(m, x, B);
  T Bn = sqrt(B[0] * B[0] + B[1] * B[1] + B[2] * B[2]);
  T kpar = (ko[0] * B[0] + ko[1] * B[1] + ko[2] * B[2]) / Bn;
  return g_kk + (omega2 - kpar * kpar) * wp2 / omega2;
}

// Photon energy in the plasma frame for local |k|^2 = K2 (units of m_a):
// LO root of Eq. AnisotropicDisp, or the isotropic E^2 = |k|^2 + omega_p^2.
template <class T>
inline T photon_energy(int dispersion, T K2, T wp2, T cos2) {
  if (dispersion == DISP_ISO) return sqrt(K2 + wp2);
  T disc = K2 * K2 + wp2 * wp2 + 2.0 * K2 * wp2 * (1.0 - 2.0 * cos2);
  return sqrt(0.5 * (K2 + wp2 + sqrt(disc)));
}

// Hamilton's equations (Eq. Hamilton): dx/dlambda = dH/dk, dk/dlambda = -dH/dx,
// derivatives by dual numbers (sigma: see plasma_freq2).
inline void rhs(const Star& s, const double m[3], double omega_inf, const double y[6],
                double dy[6], int sigma = 0) {
  typedef Dual<6> D;
  D x[3], k[3];
  for (int i = 0; i < 3; ++i) {
    x[i] = D::var(y[i], i);
    k[i] = D::var(y[3 + i], 3 + i);
  }
  D H = hamiltonian(s, m, omega_inf, x, k, sigma);
  for (int i = 0; i < 3; ++i) {
    dy[i] = H.d[3 + i];
    dy[3 + i] = -H.d[i];
  }
}

// Rigidly rotating magnetosphere: the magnetic axis turns about z,
// m(t) = m(psi0 + Omega t), while the photon flies, so the Hamiltonian
// depends on the coordinate time t and the state is the full canonical pair
// (x^mu, k_mu) of Eq. Hamilton: y = (x, k, t, k_t), eight components, with
// omega_inf = -k_t no longer a constant.  Derivatives by dual numbers in all
// eight: dx/dl = dH/dk, dk/dl = -dH/dx, dt/dl = dH/dk_t, dk_t/dl = -dH/dt.
inline void rhs_rotating(const Star& s, double psi0, const double y[8], double dy[8],
                         int sigma = 0) {
  typedef Dual<8> D;
  D x[3], k[3];
  for (int i = 0; i < 3; ++i) {
    x[i] = D::var(y[i], i);
    k[i] = D::var(y[3 + i], 3 + i);
  }
  const D t = D::var(y[6], 6);
  const D kt = D::var(y[7], 7);
  D m[3];
  magnetic_axis(s, psi0 + s.omega_R * t, m);
  D H = hamiltonian(s, m, -kt, x, k, sigma);
  for (int i = 0; i < 3; ++i) {
    dy[i] = H.d[3 + i];
    dy[3 + i] = -H.d[i];
  }
  dy[6] = H.d[7];
  dy[7] = -H.d[6];
}

}  // namespace orc
