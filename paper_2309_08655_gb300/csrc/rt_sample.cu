// Forward Monte-Carlo sampling of the resonant conversion surface (FP64).
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
#include <cuda_runtime.h>
#include <stdint.h>

#include "rt_device.cuh"
#include "rt_internal.h"

namespace rtk {

namespace {

constexpr double TWO_OVER_SQRTPI = 1.12837916709551257390;

// Inverse CDF of the Maxwellian speed x = |k_inf| / k0, density
// (4/sqrt(pi)) x^2 exp(-x^2).  Lower half: erf(x) - c x e^{-x^2} = u; upper
// half: erfc(x) + c x e^{-x^2} = 1 - u (exact for u >= 1/2), which keeps the
// tail well conditioned.  Safeguarded Newton iteration.
__device__ double maxwell_speed(int fa_model, double u) {
  if (fa_model == FA_DELTA) return 1.0;
  const bool upper = u > 0.5;
  const double v = upper ? 1.0 - u : u;
  double lo = 0.0, hi = 30.0;
  double x = 1.0876520317;   // median
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
    if (fabs(xn - x) <= 2e-16 * x || hi - lo <= 4e-16 * hi) {
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
    default: P = 0.0; dP = 0.0; break;
  }
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

__global__ void sample_kernel(SampleParams p) {
  const StarDev& s = p.s;
  const int64_t n = p.n, ld = p.ld;   // count and SoA row stride
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n;
       i += (int64_t)gridDim.x * blockDim.x) {
    const double u0 = p.u[i], u1 = p.u[ld + i], u2 = p.u[2 * ld + i];
    const double u3 = p.u[3 * ld + i], u4 = p.u[4 * ld + i], u5 = p.u[5 * ld + i];
    // direction of the conversion point and of the momentum
    const double ct = 1.0 - 2.0 * u0;
    const double st = sqrt(fmax(0.0, (1.0 - ct) * (1.0 + ct)));
    double sph, cph;
    sincospi(2.0 * u1, &sph, &cph);
    const double n0 = st * cph, n1 = st * sph, n2 = ct;
    const double ck = 1.0 - 2.0 * u2;
    const double sk = sqrt(fmax(0.0, (1.0 - ck) * (1.0 + ck)));
    double spk, cpk;
    sincospi(2.0 * u3, &spk, &cpk);
    const double q0 = sk * cpk, q1 = sk * spk, q2 = ck;
    // asymptotic axion speed and the Killing energy omega_inf / m_a = 1 + delta
    const double xs = maxwell_speed(s.fa_model, u4);
    const double kinf = xs * s.v0;
    const double delta = kinf * kinf / (sqrt(1.0 + kinf * kinf) + 1.0);
    const double om = 1.0 + delta;
    const double psi = (s.phase_mode == PHASE_UNIFORM) ? 2.0 * PI * u5 : s.psi_fixed;
    double sps, cps;
    sincos(psi, &sps, &cps);
    const double m0 = s.sin_tm * cps, m1 = s.sin_tm * sps, m2 = s.cos_tm;
    // dipole direction b = 3 (m.n) n - m (depends on n only)
    const double mu = m0 * n0 + m1 * n1 + m2 * n2;
    const double b0 = 3.0 * mu * n0 - m0, b1 = 3.0 * mu * n1 - m1, b2 = 3.0 * mu * n2 - m2;
    const double bb = 3.0 * mu * mu + 1.0;
    const double kb = q0 * b0 + q1 * b1 + q2 * b2;
    const double c2 = kb * kb / bb;
    Line L;
    L.disp = s.dispersion;
    L.plasma = s.plasma;
    L.rs = s.rs;
    L.W2 = om * om;
    L.s2 = 1.0 - c2;
    L.PR = s.cp * fabs(3.0 * n2 * mu - m2);
    L.pa = s.plasma_a;
    L.nz = n2;
    // outputs for a sample without a resonance
    p.state[6 * ld + i] = delta;
    p.state[7 * ld + i] = psi;
    bool ok = line_G(L, 1.0, nullptr) > 0.0;
    double lo = 1.0, hi = 2.0;
    if (ok) {
      int it = 0;
      while (!(line_G(L, hi, nullptr) < 0.0)) {
        lo = hi;
        hi *= 2.0;
        if (++it > 60) { ok = false; break; }
      }
    }
    if (!ok) {
#pragma unroll
      for (int c = 0; c < 6; ++c) p.state[c * ld + i] = 0.0;
      p.weight[i] = 0.0;
      p.status[i] = RAY_NO_ROOT;
      continue;
    }
    // safeguarded Newton on G
    double r = 0.5 * (lo + hi);
    for (int it = 0; it < 200; ++it) {
      double dG;
      const double g = line_G(L, r, &dG);
      if (g > 0.0) lo = r; else hi = r;
      double rn = r - g / dG;
      if (!(rn > lo && rn < hi)) rn = 0.5 * (lo + hi);
      const bool done = fabs(rn - r) <= 1e-16 * r || hi - lo <= 4e-16 * hi;
      r = rn;
      if (done) break;
    }
    // quantities at the resonance
    double P, dP, dG;
    line_plasma(L, r, P, dP);
    line_G(L, r, &dG);
    const double A = 1.0 - s.rs / r;
    const double K2 = L.W2 / A - 1.0;
    const double E2 = 1.0 + K2;
    const double E = sqrt(E2);
    double dhdr, shape;
    if (s.dispersion == DISP_ISO) {
      dhdr = dP / (2.0 * E);
      shape = L.s2;
    } else {
      const double ym = K2 * P * c2 / E2;
      dhdr = dG / (2.0 * E * (E2 - ym));
      const double D = c2 * P * (P - 2.0 * E2) + E2 * E2;
      shape = E2 * E2 * L.s2 / D;
    }
    const double kloc = sqrt(K2);
    const double ir = 1.0 / r;
    const double Bmag = s.B0_eV2 * 0.5 * ir * ir * ir * sqrt(bb);
    const double Psi = 0.5 * PI * s.g_eV * s.g_eV * Bmag * Bmag * shape * (E * s.ma_eV);
    const double r_eV = r * s.R_eV;
    const double dh_eV = fabs(dhdr) * s.ma_eV / s.R_eV;
    const double W = 4.0 * PI * r_eV * r_eV * (kloc / kinf) * s.n_inf * Psi / (A * dh_eV);
    p.weight[i] = W / (double)n * s.w_unit;
    // photon phase-space point: orthonormal k = |k| khat; covariant Cartesian
    // k = k_o + (1/sqrt(A) - 1) (n.k_o) n
    const double nko = kloc * (n0 * q0 + n1 * q1 + n2 * q2);
    const double cr = (1.0 / sqrt(A) - 1.0) * nko;
    p.state[i] = r * n0 * s.R_km;
    p.state[ld + i] = r * n1 * s.R_km;
    p.state[2 * ld + i] = r * n2 * s.R_km;
    p.state[3 * ld + i] = (kloc * q0 + cr * n0) * s.ma_eV;
    p.state[4 * ld + i] = (kloc * q1 + cr * n1) * s.ma_eV;
    p.state[5 * ld + i] = (kloc * q2 + cr * n2) * s.ma_eV;
    p.status[i] = RAY_READY;
  }
}

}  // namespace

cudaError_t launch_sample(const SampleParams& p, cudaStream_t stream) {
  if (p.n <= 0) return cudaSuccess;
  int dev = 0, nsm = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return e;
  e = cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev);
  if (e != cudaSuccess) return e;
  const int block = 128;
  int64_t grid = (p.n + block - 1) / block;
  const int64_t cap = (int64_t)nsm * 8;
  if (grid > cap) grid = cap;
  sample_kernel<<<(unsigned)grid, block, 0, stream>>>(p);
  return cudaGetLastError();
}

}  // namespace rtk
