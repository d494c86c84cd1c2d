// Device-side model of the magnetosphere and the photon Hamiltonian, with
// hand-derived analytic gradients for Hamilton's equations.
//
// Units inside kernels: lengths in the stellar radius R, momenta in the axion
// mass m_a.  The Hamiltonian (Eq. StrongBHam, Sec. 4.1) on Schwarzschild
// (Eq. SchwarzshildMetric1) in Cartesianised coordinates, static plasma frame,
// k_t = -omega_inf conserved, is (divided by m_a^2)
//
//   H = -W2/A + |k|^2 + (A-1)(n.k)^2 + P - P A Kp^2 / W2          (anisotropic)
//   H = -W2/A + |k|^2 + (A-1)(n.k)^2 + P                          (isotropic)
//
// with A = 1 - rs/r, n = x/r, W2 = omega_inf^2, P = omega_p^2 and
// Kp = k_par = k_o . b/|b| the momentum component along the dipole direction
// b = 3 (m.n) n - m in the static orthonormal frame, whose radial momentum
// component is sqrt(A) (n.k).  Goldreich-Julian (Eq. GJDensity):
// P = cp r^-3 |3 n_z (m.n) - m_z|.
#pragma once
#include <cuda_runtime.h>
#include <stdint.h>

#define RT_HD __host__ __device__

namespace rtk {

constexpr double PI = 3.14159265358979323846;
// 1 cm^-3 in eV^3: (hbar c)^3 with hbar c = 1.973269804e-5 eV cm (CODATA 2018)
constexpr double PER_CM3_EV3 = 1.973269804e-5 * 1.973269804e-5 * 1.973269804e-5;

// Per-star constants (device copy built by rt_init_star).
struct StarDev {
  double rs;          // r_s / R used for the initial conditions
  double rs_prop;     // r_s / R in the propagation Hamiltonian (0 for flat propagation)
  double cp;          // omega_p^2 coefficient / m_a^2 (Goldreich-Julian)
  double plasma_a;    // test-medium parameter
  double cos_tm, sin_tm, psi_fixed;
  double v0;          // Maxwellian dispersion [c]
  double R_km, ma_eV;
  double R_eV;        // R in eV^-1
  double B0_eV2;      // polar surface field [eV^2]
  double g_eV;        // coupling [eV^-1]
  double n_inf;       // asymptotic axion number density [eV^3]
  double w_unit;      // 1 eV^2 of power in W
  double rlc;         // light-cylinder radius / R (open field lines of the twisted model)
  int32_t dispersion, plasma, fa_model, phase_mode;
  int32_t weight_mode;  // WEIGHT_PAG, WEIGHT_UNIT_P or WEIGHT_RENORM
  int32_t rotation;     // ROTATION_SNAPSHOT or ROTATION_RIGID (rt_trace_rot.cu)
};

enum { DISP_ANISO = 0, DISP_ISO = 1 };
enum {
  PLASMA_GJ = 0, PLASMA_VACUUM = 1, PLASMA_HOMOG = 2, PLASMA_LINEAR_Z = 3, PLASMA_RADIAL = 4,
  PLASMA_TWISTED = 5
};
enum { FA_MAXWELL = 0, FA_DELTA = 1 };
enum { WEIGHT_PAG = 0, WEIGHT_UNIT_P = 1, WEIGHT_RENORM = 2 };
enum { PHASE_FIXED = 0, PHASE_UNIFORM = 1 };
enum { ROTATION_SNAPSHOT = 0, ROTATION_RIGID = 1 };
enum {
  RAY_READY = 0, RAY_ESCAPED = 1, RAY_CAPTURED = 2, RAY_NO_ROOT = 3, RAY_MAXSTEPS = 4,
  RAY_NAN = 5, RAY_STIFF = 6, RAY_LAMBDA_END = 7,
  RAY_PROMOTED = 8,  // internal: handed from the FP32 pass to the FP64 pass
  RAY_EXPRESS = 9    // internal: traced by the express groups of the FP64 launch
};

// (The host branches exist for host-side instantiation in tests of the formula.)
RT_HD __forceinline__ double rt_rsqrt(double v) {
#ifdef __CUDA_ARCH__
  return rsqrt(v);
#else
  return 1.0 / sqrt(v);
#endif
}
RT_HD __forceinline__ float rt_rsqrt(float v) {
#ifdef __CUDA_ARCH__
  return rsqrtf(v);
#else
  return 1.0f / sqrtf(v);
#endif
}
RT_HD __forceinline__ double rt_sqrt(double v) { return sqrt(v); }
RT_HD __forceinline__ float rt_sqrt(float v) { return sqrtf(v); }
RT_HD __forceinline__ double rt_rcp(double v) { return 1.0 / v; }
RT_HD __forceinline__ float rt_rcp(float v) {
#ifdef __CUDA_ARCH__
  return __frcp_rn(v);
#else
  return 1.0f / v;
#endif
}

// Constants of one ray in the working precision T.
template <class T>
struct RayConst {
  T rs;          // r_s / R (propagation)
  T cp;          // GJ coefficient
  T pa;          // test-medium parameter
  T W2, iW2;     // omega_inf^2 and its inverse
  T m0, m1, m2;  // magnetic axis
  T sig;         // side of the Goldreich-Julian null cone being integrated (+-1)
  int disp, plasma;
};

// Sign of Omega . B (that of 3 z (m.x) - m_z |x|^2): the Goldreich-Julian
// density |2 Omega . B / e| has a kink where it vanishes.
template <class T>
RT_HD __forceinline__ T gj_side(const T m0, const T m1, const T m2, const T x0, const T x1,
                                const T x2) {
  const T g = T(3) * x2 * (m0 * x0 + m1 * x1 + m2 * x2) - m2 * (x0 * x0 + x1 * x1 + x2 * x2);
  return g < T(0) ? T(-1) : T(1);
}

// dx/dl = dH/dk, dk/dl = -dH/dx (Eq. Hamilton), analytic.  With XCORR the
// position derivative is returned without its flat-space part 2k (the caller
// then adds 2k itself, in higher precision).  With DW also *dw = dH/dW2, the
// derivative with respect to omega_inf^2 = k_t^2 (for a Hamiltonian in which
// k_t evolves).  (Host-callable only for the flop-counting scalar of
// rt_flops.cu.)
template <class T, bool XCORR = false, bool FIN = false, bool DW = false>
RT_HD __forceinline__ void ham_rhs(const RayConst<T>& c, const T x0, const T x1,
                                        const T x2, const T k0, const T k1, const T k2, T& dx0,
                                        T& dx1, T& dx2, T& dk0, T& dk1, T& dk2,
                                        const T F_in = T(0), T* dw = nullptr) {
  const T r2 = x0 * x0 + x1 * x1 + x2 * x2;
  const T ir = rt_rsqrt(r2);
  const T n0 = x0 * ir, n1 = x1 * ir, n2 = x2 * ir;
  const T ir2 = ir * ir;
  const T A = T(1) - c.rs * ir;
  const T Am1 = -c.rs * ir;
  const T qA = rt_rsqrt(A);                    // one special for 1/A, sqrt(A), 1/sqrt(A)
  const T iA = qA * qA;
  const T W = c.W2 * iA;                       // omega^2
  const T kr = n0 * k0 + n1 * k1 + n2 * k2;    // n.k
  // metric part: H_g = -W2/A + k.k + (A-1) kr^2
  //   dH_g/dk = 2k + 2(A-1) kr n
  //   dH_g/dx = (W/A + kr^2) dA + 2(A-1) kr dkr,  dA = rs r^-2 n, dkr = (k - kr n)/r
  T gk0 = T(2) * ((XCORR ? T(0) : k0) + Am1 * kr * n0);
  T gk1 = T(2) * ((XCORR ? T(0) : k1) + Am1 * kr * n1);
  T gk2 = T(2) * ((XCORR ? T(0) : k2) + Am1 * kr * n2);
  const T cA = (W * iA + kr * kr) * c.rs * ir2;
  const T ckr = T(2) * Am1 * kr * ir;
  T gx0 = cA * n0 + ckr * (k0 - kr * n0);
  T gx1 = cA * n1 + ckr * (k1 - kr * n1);
  T gx2 = cA * n2 + ckr * (k2 - kr * n2);
  // plasma frequency and its gradient
  const T mu = c.m0 * n0 + c.m1 * n1 + c.m2 * n2;   // m.n
  T P = T(0), dP0 = T(0), dP1 = T(0), dP2 = T(0);
  if (c.plasma == PLASMA_GJ) {
    // within a step: the smooth continuation sig * F of the side the step
    // started on (the integrator switches sig where a step crosses F = 0).
    // FIN: F supplied by the caller (evaluated in higher precision: near the
    // null cone F is a small difference of O(1) terms)
    const T F = FIN ? F_in : T(3) * n2 * mu - c.m2;
    const T sF = c.sig;
    const T ir3 = ir2 * ir;
    P = c.cp * ir3 * (F * sF);
    // dF = 3/r (mu z + n_z m - 2 mu n_z n)
    const T t = c.cp * ir3 * sF * T(3) * ir;
    const T m3 = T(-3) * P * ir;
    const T two_mu_nz = T(2) * mu * n2;
    dP0 = m3 * n0 + t * (n2 * c.m0 - two_mu_nz * n0);
    dP1 = m3 * n1 + t * (n2 * c.m1 - two_mu_nz * n1);
    dP2 = m3 * n2 + t * (mu + n2 * c.m2 - two_mu_nz * n2);
  } else if (c.plasma == PLASMA_HOMOG) {
    P = c.pa;
  } else if (c.plasma == PLASMA_LINEAR_Z) {
    P = c.pa * x2;
    dP2 = c.pa;
  } else if (c.plasma == PLASMA_RADIAL) {
    P = c.pa * ir2 * ir;
    const T m3 = T(-3) * P * ir;
    dP0 = m3 * n0;
    dP1 = m3 * n1;
    dP2 = m3 * n2;
  } else if (c.plasma == PLASMA_TWISTED) {
    // twisted magnetosphere (Eq. neMag): P = cp (1 - mu^2) r^-4, so
    // dP = cp r^-5 (-2 mu (m - mu n) - 4 (1 - mu^2) n) = cp r^-5 (-2 mu m + (6 mu^2 - 4) n)
    const T ir4 = ir2 * ir2;
    P = c.cp * (T(1) - mu * mu) * ir4;
    const T q = c.cp * ir4 * ir;
    const T am = T(-2) * q * mu;
    const T an = q * (T(6) * mu * mu - T(4));
    dP0 = am * c.m0 + an * n0;
    dP1 = am * c.m1 + an * n1;
    dP2 = am * c.m2 + an * n2;
  }
  if (c.disp == DISP_ISO) {
    gx0 += dP0;
    gx1 += dP1;
    gx2 += dP2;
    if (DW) *dw = -iA;                            // d(-W2/A)/dW2
  } else {
    // anisotropic term H_a = P - P A Kp^2 / W2 with Kp = U / |b|,
    // U = k.b + (sqrt(A) - 1) (n.k)(n.b), n.b = 2 mu, |b|^2 = 3 mu^2 + 1
    const T ib = rt_rsqrt(T(3) * mu * mu + T(1));
    const T sA = A * qA;
    const T km = k0 * c.m0 + k1 * c.m1 + k2 * c.m2;
    const T U = T(3) * mu * kr - km + T(2) * mu * kr * (sA - T(1));
    const T Kp = U * ib;
    const T Kp2iW2 = Kp * Kp * c.iW2;
    const T fac = P * A * Kp * c.iW2;             // dH_a/dKp = -2 fac
    const T opsA = T(1) + T(2) * sA;
    // dKp/dk = |b|^-1 (mu (1 + 2 sqrt(A)) n - m)
    const T c1 = mu * opsA;
    const T g2 = T(-2) * fac * ib;
    gk0 += g2 * (c1 * n0 - c.m0);
    gk1 += g2 * (c1 * n1 - c.m1);
    gk2 += g2 * (c1 * n2 - c.m2);
    // dKp/dx = a1 dmu + a2 dkr + a3 n with dmu = (m - mu n)/r, dkr = (k - kr n)/r
    const T ib3 = ib * ib * ib;
    const T a1 = ib * opsA * kr - T(3) * mu * U * ib3;
    const T a2 = ib * opsA * mu;
    const T a3 = ib * mu * kr * c.rs * ir2 * qA;
    const T a1r = a1 * ir, a2r = a2 * ir;
    const T an = a3 - a1r * mu - a2r * kr;
    const T dK0 = a1r * c.m0 + a2r * k0 + an * n0;
    const T dK1 = a1r * c.m1 + a2r * k1 + an * n1;
    const T dK2 = a1r * c.m2 + a2r * k2 + an * n2;
    // dH_a/dx = dP (1 - A Kp^2/W2) - P Kp^2/W2 dA - 2 fac dKp
    const T one_m = T(1) - A * Kp2iW2;
    const T cdA = -P * Kp2iW2 * c.rs * ir2;
    const T m2f = T(-2) * fac;
    if (DW) *dw = Kp2iW2 * P * A * c.iW2 - iA;    // d(-W2/A - P A Kp^2/W2)/dW2
    gx0 += dP0 * one_m + cdA * n0 + m2f * dK0;
    gx1 += dP1 * one_m + cdA * n1 + m2f * dK1;
    gx2 += dP2 * one_m + cdA * n2 + m2f * dK2;
  }
  dx0 = gk0;
  dx1 = gk1;
  dx2 = gk2;
  dk0 = -gx0;
  dk1 = -gx1;
  dk2 = -gx2;
}

// The value of H (diagnostics).
template <class T>
__device__ __forceinline__ T ham_value(const RayConst<T>& c, const T* x, const T* k) {
  const T r2 = x[0] * x[0] + x[1] * x[1] + x[2] * x[2];
  const T ir = rt_rsqrt(r2);
  const T n0 = x[0] * ir, n1 = x[1] * ir, n2 = x[2] * ir;
  const T A = T(1) - c.rs * ir;
  const T kr = n0 * k[0] + n1 * k[1] + n2 * k[2];
  const T kk = k[0] * k[0] + k[1] * k[1] + k[2] * k[2];
  T H = -c.W2 / A + kk + (A - T(1)) * kr * kr;
  const T mu = c.m0 * n0 + c.m1 * n1 + c.m2 * n2;
  T P = T(0);
  if (c.plasma == PLASMA_GJ) {
    T F = T(3) * n2 * mu - c.m2;
    P = c.cp * ir * ir * ir * (F < T(0) ? -F : F);
  } else if (c.plasma == PLASMA_HOMOG) {
    P = c.pa;
  } else if (c.plasma == PLASMA_LINEAR_Z) {
    P = c.pa * x[2];
  } else if (c.plasma == PLASMA_RADIAL) {
    P = c.pa * ir * ir * ir;
  } else if (c.plasma == PLASMA_TWISTED) {
    P = c.cp * (T(1) - mu * mu) * ir * ir * ir * ir;
  }
  if (c.disp == DISP_ISO) return H + P;
  const T ib = rt_rsqrt(T(3) * mu * mu + T(1));
  const T sA = rt_sqrt(A);
  const T km = k[0] * c.m0 + k[1] * c.m1 + k[2] * c.m2;
  const T Kp = (T(3) * mu * kr - km + T(2) * mu * kr * (sA - T(1))) * ib;
  return H + P - P * A * Kp * Kp * c.iW2;
}

// Claiming work from the global queue of a persistent kernel.  item: -1 the
// lane needs work, -2 the queue is exhausted for it, >= 0 the item in flight.
// A lane that needs work first takes the next entry of the chunk it claimed
// last (claim_size consecutive queue entries); the lanes whose chunks are
// spent claim fresh chunks together -- one atomicAdd per warp -- once at least
// refill_min of them wait, or at once when no lane of the warp holds an item.
// take(e) loads queue entry e and returns its item index, or -1 for an entry
// that is not to be traced.  refill_min = claim_size = 1 claims one entry per
// waiting lane at every call (a warp refills as soon as any lane is free).
struct ClaimChunk {
  int64_t next = 0, end = 0;
};

template <class Take>
__device__ __forceinline__ void claim_items(unsigned long long* queue, int64_t nq,
                                            int refill_min, int claim_size, int64_t& item,
                                            ClaimChunk& ch, Take&& take) {
  constexpr unsigned ALL = 0xffffffffu;
  while (item == -1 && ch.next < ch.end) item = take(ch.next++);
  const bool need = (item == -1);
  const unsigned mneed = __ballot_sync(ALL, need);
  if (!mneed) return;
  if (__popc(mneed) < refill_min && __ballot_sync(ALL, item >= 0) != 0u) return;
  const int lane = threadIdx.x & 31;
  const int leader = __ffs(mneed) - 1;
  unsigned long long base = 0;
  if (lane == leader)
    base = atomicAdd(queue, (unsigned long long)__popc(mneed) * (unsigned long long)claim_size);
  base = __shfl_sync(ALL, base, leader);
  if (need) {
    ch.next = (int64_t)base + (int64_t)__popc(mneed & ((1u << lane) - 1u)) * claim_size;
    ch.end = ch.next + claim_size < nq ? ch.next + claim_size : nq;
    if (ch.next >= nq) {
      item = -2;
      return;
    }
    while (item == -1 && ch.next < ch.end) item = take(ch.next++);
  }
}

// Nanosecond global timer of the GPU (for per-instance completion times).
__device__ __forceinline__ unsigned long long global_ns() {
  unsigned long long t;
  asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
  return t;
}

// Largest displacement of one integration step, as a fraction of the distance
// to the centre: far from the star the medium is nearly uniform and the
// embedded error estimate alone would let one step carry a ray across the star
// and its plasma, which no stage of that step samples.
constexpr double STEP_REACH = 0.5;

// Dormand-Prince 5(4) coefficients (Dormand & Prince 1980) and the
// continuous extension of Hairer, Norsett & Wanner (Sec. II.6).
struct DP {
  static constexpr double a21 = 1.0 / 5.0;
  static constexpr double a31 = 3.0 / 40.0, a32 = 9.0 / 40.0;
  static constexpr double a41 = 44.0 / 45.0, a42 = -56.0 / 15.0, a43 = 32.0 / 9.0;
  static constexpr double a51 = 19372.0 / 6561.0, a52 = -25360.0 / 2187.0,
                          a53 = 64448.0 / 6561.0, a54 = -212.0 / 729.0;
  static constexpr double a61 = 9017.0 / 3168.0, a62 = -355.0 / 33.0, a63 = 46732.0 / 5247.0,
                          a64 = 49.0 / 176.0, a65 = -5103.0 / 18656.0;
  static constexpr double b1 = 35.0 / 384.0, b3 = 500.0 / 1113.0, b4 = 125.0 / 192.0,
                          b5 = -2187.0 / 6784.0, b6 = 11.0 / 84.0;
  static constexpr double e1 = 71.0 / 57600.0, e3 = -71.0 / 16695.0, e4 = 71.0 / 1920.0,
                          e5 = -17253.0 / 339200.0, e6 = 22.0 / 525.0, e7 = -1.0 / 40.0;
  static constexpr double d1 = -12715105075.0 / 11282082432.0,
                          d3 = 87487479700.0 / 32700410799.0,
                          d4 = -10690763975.0 / 1880347072.0,
                          d5 = 701980252875.0 / 199316789632.0,
                          d6 = -1453857185.0 / 822651844.0, d7 = 69997945.0 / 29380423.0;
};

}  // namespace rtk
