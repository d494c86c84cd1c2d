// Backward image plane: shared by the FP64 kernel (rt_trace.cu) and the
// mixed-precision kernel (rt_trace_mixed.cu).
//
// Backward image plane (Sec. 2.1, Eq. BackPower; all level crossings,
// Sec. 5.1.3).  By Liouville's theorem the forward phase-space integral
// P = int d^3x d^3k j, j = sqrt(A) delta(E_gamma - E_a) Psi f_a, equals
// dP/dOmega = int dA int domega omega^2 int_ray j dt over the photons crossing
// a distant plane; the ray integral of the delta function is a sum over the
// crossings of g = E_gamma - E_a = omega - sqrt(m_a^2 + |k|^2) along the ray,
// sum_c sqrt(A) Psi f_a |dt/dl| / |dg/dl|.  Each pixel's time-reversed ray
// (k -> -k; H is even in k) is traced inward from the plane.  Within each
// accepted step the ray is the continuous extension y(th), th in [0, 1]; the
// step is cut into BACK_SUBDIV pieces, and a crossing is either a sign change
// of g across a piece or, where the ray grazes the resonance, a pair of roots
// around an extremum of g inside a piece with no sign change at its ends.  The
// sign of g at the piece ends is screened in FP32 (FP64 where the screen is
// not certain); the slope of the screened quantity along th, also in FP32,
// brackets the extrema of g that turn toward zero, and where a tangent-line
// bound lets such a dip reach zero the extremum is located in FP64 by
// bisection on the sign of dg/dth.  Every root is located by FP64 bisection.

#pragma once
#include <cuda_runtime.h>
#include <stdint.h>

#include "rt_device.cuh"
#include "rt_integrator.cuh"

namespace rtk {

constexpr int BACK_SUBDIV = 16;
// A grazing pair inside a piece needs g near zero there: the slope of the
// screened N is formed only where |N| < SLOPE_NEAR at an end of the piece
// (far from the resonance N ~ -1; a smooth dip of N by more than 0.5 within a
// sixteenth of a step that resolves the ray to rtol does not occur).
constexpr float SLOPE_NEAR = 0.5f;

struct BackParams {
  StarDev s;
  int nx, ny;
  double incl, D, bmax;
  double W;             // omega_inf / m_a at the line centre
  double Lc_cut;        // conversion-length cut, units of R (0: none)
  double img_scale;     // pixel area x frequency-integrated f_a x unit conversion
  double* image;
  uint8_t* status;
  int32_t* ncross;
  int64_t* counters;
  unsigned long long* queue;
  double rtol, atol, r_capture;
  int max_steps;
  unsigned long long* ts;
  // mixed kernel: pixels handed to the FP64 kernel (appended, count in *promo_n)
  int32_t* promo;
  unsigned long long* promo_n;
  // FP64 kernel: trace only the pixels listed (list[0 .. *list_n)), if set
  const int32_t* list;
  const unsigned long long* list_n;
};

// rt_trace_mixed.cu: the mixed-precision kernel over all pixels (appends the
// pixels it hands over to bp.promo; *bp.promo_n must be 0 at launch).
cudaError_t launch_backward_mixed(const BackParams& bp, cudaStream_t stream);

// The backward images of a batch, traced in the same persistent launch as the
// batch's forward rays: queue items 0 .. n-1 are the rays, n .. n+npix-1 the
// pixels, image after image (image j's pixels at off[j] .. off[j+1]-1, each
// image's BackParams pointing at its slices of the output buffers).
struct ImgTable {
  const BackParams* img;            // device, nimg entries
  const int64_t* off;               // device, nimg + 1 pixel offsets
  int nimg;
  int64_t npix;
  int32_t* promo;                   // mixed: pixels handed to FP64 (index over all images)
  unsigned long long* promo_n;
  const int32_t* list;              // FP64 pass: only these pixels, and only rays with
  const unsigned long long* list_n; // status claim_status, when set
  unsigned long long* ts;           // optional: nimg last-pixel stamps (max)
};

__device__ __forceinline__ int find_image(const ImgTable& t, int64_t q) {
  int lo = 0, hi = t.nimg - 1;      // off[j] <= q < off[j + 1]
  while (lo < hi) {
    const int mid = (lo + hi + 1) >> 1;
    if (t.off[mid] <= q) lo = mid; else hi = mid - 1;
  }
  return lo;
}

// rt_trace.cu (FP64) and rt_trace_mixed.cu: one persistent launch over a
// batch's rays (those with status p.claim_status) and pixels.
cudaError_t launch_batch_fp64(const TraceParams& p, const ImgTable& t, int block,
                              int blocks_per_sm, cudaStream_t stream);
cudaError_t launch_batch_mixed(const TraceParams& p, const ImgTable& t, int block,
                               int blocks_per_sm, cudaStream_t stream);

__device__ __forceinline__ double crossing_g(const RayConst<double>& c, double W,
                                             const double* y) {
  const double r2 = y[0] * y[0] + y[1] * y[1] + y[2] * y[2];
  const double ir = rsqrt(r2);
  const double A = 1.0 - c.rs * ir;
  const double kr = (y[0] * y[3] + y[1] * y[4] + y[2] * y[5]) * ir;
  const double kk = y[3] * y[3] + y[4] * y[4] + y[5] * y[5] + (A - 1.0) * kr * kr;
  return W * rsqrt(A) - sqrt(1.0 + kk);
}

// g and dg/dth at a point y of the continuous extension with y' = dy/dth.
__device__ __forceinline__ void crossing_g_slope(const RayConst<double>& c, double W,
                                                 const double* y, const double* yp, double* g,
                                                 double* dg) {
  const double r2 = y[0] * y[0] + y[1] * y[1] + y[2] * y[2];
  const double ir = rsqrt(r2);
  const double n0 = y[0] * ir, n1 = y[1] * ir, n2 = y[2] * ir;
  const double A = 1.0 - c.rs * ir;
  const double kr = n0 * y[3] + n1 * y[4] + n2 * y[5];
  const double kk = y[3] * y[3] + y[4] * y[4] + y[5] * y[5] + (A - 1.0) * kr * kr;
  const double Ea = sqrt(1.0 + kk);
  const double om = W * rsqrt(A);
  *g = om - Ea;
  // dg/dx = (d omega / dA - d|k|^2/dA / 2E_a) dA/dx - (d|k|^2/dkr / 2E_a) dkr/dx
  const double dAr = c.rs * ir * ir;                       // dA/dx = dAr n
  const double c_om = -0.5 * om / A * dAr;
  const double ckr = 2.0 * (A - 1.0) * kr * ir;
  const double iEa = 0.5 / Ea;
  double d = 0.0;
#pragma unroll
  for (int i = 0; i < 3; ++i) {
    const double ni = (i == 0) ? n0 : (i == 1) ? n1 : n2;
    const double dkk_dx = kr * kr * dAr * ni + ckr * (y[3 + i] - kr * ni);
    const double dkk_dk = 2.0 * (y[3 + i] + (A - 1.0) * kr * ni);
    d += (c_om * ni - dkk_dx * iEa) * yp[i] - dkk_dk * iEa * yp[3 + i];
  }
  *dg = d;
}

// Sign of g at a sample point, decided in FP32 where it is certain.  g is a
// difference of two nearly equal terms, but on shell (H = 0)
//   W^2/A - |k|_g^2 = P G - H,  G = 1 - A Kp^2 / W^2 (anisotropic) or 1,
// so g = W/sqrt(A) - sqrt(1 + |k|_g^2) has the sign of N - H with N = P G - 1,
// and N is well conditioned away from the resonance itself.  H is the
// integrator's drift (of order rtol) and N carries the FP32 rounding of the
// sample point; where |N| exceeds a margin that bounds both by orders of
// magnitude, sign(g) = sign(N) and the FP64 evaluation of g is skipped.
// Elsewhere g is evaluated in FP64, so every sampled sign, and with it every
// crossing found, is that of the FP64 evaluation.  P is the plasma term of the
// side being integrated (sig), as in the integrated Hamiltonian.
struct Screen {
  float rs, cp, pa, iW2, m0, m1, m2, sig;
  float F0, gF[3];   // 3 z (m.x) - m_z |x|^2 and its gradient at the step start (FP64-formed)
  int disp, plasma;
};

__device__ __forceinline__ Screen make_screen(const RayConst<double>& c, const double* y) {
  Screen s;
  s.rs = (float)c.rs;
  s.cp = (float)c.cp;
  s.pa = (float)c.pa;
  s.iW2 = (float)c.iW2;
  s.m0 = (float)c.m0;
  s.m1 = (float)c.m1;
  s.m2 = (float)c.m2;
  s.sig = (float)c.sig;
  s.disp = c.disp;
  s.plasma = c.plasma;
  s.F0 = 0.0f;
  s.gF[0] = s.gF[1] = s.gF[2] = 0.0f;
  if (c.plasma == PLASMA_GJ) {
    const double mx = c.m0 * y[0] + c.m1 * y[1] + c.m2 * y[2];
    const double r2 = y[0] * y[0] + y[1] * y[1] + y[2] * y[2];
    s.F0 = (float)(3.0 * y[2] * mx - c.m2 * r2);
    s.gF[0] = (float)(3.0 * y[2] * c.m0 - 2.0 * c.m2 * y[0]);
    s.gF[1] = (float)(3.0 * y[2] * c.m1 - 2.0 * c.m2 * y[1]);
    s.gF[2] = (float)(3.0 * mx + 3.0 * y[2] * c.m2 - 2.0 * c.m2 * y[2]);
  }
  return s;
}

// +1 / -1: g > 0 / g < 0 for certain; 0: evaluate g in FP64.  x = x0 + d
// (FP32), d the displacement from the step start, k the momentum.  *Nout:
// N = P G - 1 (the screened quantity, of the sign of g up to the drift H).
__device__ __forceinline__ int screen_sign(const Screen& s, const float* x, const float* d,
                                           const float* k, float* Nout) {
  const float r2 = x[0] * x[0] + x[1] * x[1] + x[2] * x[2];
  const float ir = rsqrtf(r2);
  const float A = 1.0f - s.rs * ir;
  float P = 0.0f, dP = 0.0f;
  if (s.plasma == PLASMA_GJ) {
    // the null-cone factor expanded about the step start (exact quadratic)
    const float md = s.m0 * d[0] + s.m1 * d[1] + s.m2 * d[2];
    const float dd = d[0] * d[0] + d[1] * d[1] + d[2] * d[2];
    const float Fu = s.F0 + (s.gF[0] * d[0] + s.gF[1] * d[1] + s.gF[2] * d[2]) +
                     (3.0f * d[2] * md - s.m2 * dd);
    const float pre = s.cp * ir * ir * ir * ir * ir;       // cp r^-5
    P = pre * Fu * s.sig;
    // FP32 rounding of F0, gF and the expansion: |terms| <= 20 (r^2 + |d|^2)
    dP = pre * 1e-5f * (r2 + dd);
  } else if (s.plasma == PLASMA_HOMOG) {
    P = s.pa;
  } else if (s.plasma == PLASMA_LINEAR_Z) {
    P = s.pa * x[2];
    dP = 1e-6f * fabsf(P);
  } else if (s.plasma == PLASMA_RADIAL) {
    P = s.pa * ir * ir * ir;
  } else if (s.plasma == PLASMA_TWISTED) {
    const float mu = (s.m0 * x[0] + s.m1 * x[1] + s.m2 * x[2]) * ir;
    P = s.cp * (1.0f - mu * mu) * ir * ir * ir * ir;
    dP = 1e-6f * fabsf(P);
  }
  float G = 1.0f, t = 0.0f;
  if (s.disp != DISP_ISO) {
    const float n0 = x[0] * ir, n1 = x[1] * ir, n2 = x[2] * ir;
    const float mu = s.m0 * n0 + s.m1 * n1 + s.m2 * n2;
    const float kr = n0 * k[0] + n1 * k[1] + n2 * k[2];
    const float km = s.m0 * k[0] + s.m1 * k[1] + s.m2 * k[2];
    const float Kpb = 3.0f * mu * kr - km + 2.0f * mu * kr * (sqrtf(A) - 1.0f);
    t = A * Kpb * Kpb * s.iW2 / (3.0f * mu * mu + 1.0f);
    G = 1.0f - t;
  }
  const float PG = P * G;
  const float N = PG - 1.0f;
  const float margin = 0.05f * (1.0f + fabsf(PG)) + dP * fabsf(G) + 1e-5f * fabsf(P) * (1.0f + t);
  *Nout = N;
  if (!(fabsf(N) > margin)) return 0;      // also NaN
  return N > 0.0f ? 1 : -1;
}

// dN/dth of the screened N = P G - 1 along the continuous extension, in FP32:
// x = x0 + d, k, and their th-derivatives xp, kp.  Only its sign is used, to
// bracket extrema of g between sample points (FP32 suffices on this chip,
// where FP32 arithmetic is ~64 times cheaper than FP64).
__device__ __forceinline__ float screen_slope(const Screen& s, const float* x, const float* d,
                                              const float* k, const float* xp,
                                              const float* kp) {
  const float r2 = x[0] * x[0] + x[1] * x[1] + x[2] * x[2];
  const float ir = rsqrtf(r2);
  const float n0 = x[0] * ir, n1 = x[1] * ir, n2 = x[2] * ir;
  const float rp = n0 * xp[0] + n1 * xp[1] + n2 * xp[2];          // dr/dth
  const float lr = rp * ir;                                       // dln r/dth
  const float A = 1.0f - s.rs * ir;
  const float mu = s.m0 * n0 + s.m1 * n1 + s.m2 * n2;
  const float mxp = s.m0 * xp[0] + s.m1 * xp[1] + s.m2 * xp[2];
  const float mup = (mxp - mu * rp) * ir;                         // d(m.n)/dth
  float P = 0.0f, Pp = 0.0f;
  if (s.plasma == PLASMA_GJ) {
    const float md = s.m0 * d[0] + s.m1 * d[1] + s.m2 * d[2];
    const float dd = d[0] * d[0] + d[1] * d[1] + d[2] * d[2];
    const float Fu = s.F0 + (s.gF[0] * d[0] + s.gF[1] * d[1] + s.gF[2] * d[2]) +
                     (3.0f * d[2] * md - s.m2 * dd);
    const float Fp = (s.gF[0] + 3.0f * d[2] * s.m0 - 2.0f * s.m2 * d[0]) * xp[0] +
                     (s.gF[1] + 3.0f * d[2] * s.m1 - 2.0f * s.m2 * d[1]) * xp[1] +
                     (s.gF[2] + 3.0f * d[2] * s.m2 + 3.0f * md - 2.0f * s.m2 * d[2]) * xp[2];
    const float pre = s.cp * ir * ir * ir * ir * ir;               // cp r^-5
    P = pre * Fu * s.sig;
    Pp = pre * s.sig * (Fp - 5.0f * Fu * lr);
  } else if (s.plasma == PLASMA_LINEAR_Z) {
    P = s.pa * x[2];
    Pp = s.pa * xp[2];
  } else if (s.plasma == PLASMA_RADIAL) {
    P = s.pa * ir * ir * ir;
    Pp = -3.0f * P * lr;
  } else if (s.plasma == PLASMA_TWISTED) {
    const float q = s.cp * ir * ir * ir * ir;
    P = q * (1.0f - mu * mu);
    Pp = -2.0f * q * mu * mup - 4.0f * P * lr;
  } else if (s.plasma == PLASMA_HOMOG) {
    P = s.pa;
  }
  if (s.disp == DISP_ISO) return Pp;
  // G = 1 - t, t = A Kpb^2 iW2 / (3 mu^2 + 1), Kpb = mu kr (1 + 2 sqrt(A)) - m.k
  const float rsA = rsqrtf(A);
  const float sA = A * rsA;
  const float Ap = s.rs * ir * lr;                                // dA/dth
  const float kr = n0 * k[0] + n1 * k[1] + n2 * k[2];
  const float krp = ((xp[0] - n0 * rp) * k[0] + (xp[1] - n1 * rp) * k[1] +
                     (xp[2] - n2 * rp) * k[2]) * ir +
                    n0 * kp[0] + n1 * kp[1] + n2 * kp[2];
  const float km = s.m0 * k[0] + s.m1 * k[1] + s.m2 * k[2];
  const float kmp = s.m0 * kp[0] + s.m1 * kp[1] + s.m2 * kp[2];
  const float Kpb = mu * kr * (1.0f + 2.0f * sA) - km;
  const float Kpbp = (mup * kr + mu * krp) * (1.0f + 2.0f * sA) + mu * kr * Ap * rsA - kmp;
  const float ibb = __fdividef(1.0f, 3.0f * mu * mu + 1.0f);      // only the sign is used
  const float t = A * Kpb * Kpb * s.iW2 * ibb;
  const float tp = (s.iW2 * (Ap * Kpb * Kpb + 2.0f * A * Kpb * Kpbp) - t * 6.0f * mu * mup) * ibb;
  return Pp * (1.0f - t) - P * tp;
}

// The continuous extension's displacement d(th) = th (p2 + u (p3 + th (p4 +
// u p5))), u = 1 - th, and its derivative dd/dth, in FP32.
__device__ __forceinline__ void dense32(float t, const float* p2, const float* p3,
                                        const float* p4, const float* p5, float* d) {
  const float u = 1.0f - t;
#pragma unroll
  for (int i = 0; i < 6; ++i) d[i] = t * (p2[i] + u * (p3[i] + t * (p4[i] + u * p5[i])));
}
__device__ __forceinline__ void dense32_slope(float t, const float* p2, const float* p3,
                                              const float* p4, const float* p5, float* dp) {
  const float u = 1.0f - t;
#pragma unroll
  for (int i = 0; i < 6; ++i) {
    const float Q3 = p4[i] + u * p5[i];
    const float Q2 = p3[i] + t * Q3;
    dp[i] = p2[i] + u * Q2 + t * (u * (Q3 - t * p5[i]) - Q2);
  }
}

// Crossing search and estimator of one pixel's ray.
struct CrossingAcc {
  const StarDev* s;
  double W, Lc_cut;
  double sum;
  int ncross, ncut;
  int nsearch;       // FP64 extremum searches (pieces where a dip could reach zero)
  bool have_g;
  bool neg_prev;     // g < 0 at the end of the previous accepted step

  __device__ void reset(const StarDev* star, double W_, double Lc) {
    s = star;
    W = W_;
    Lc_cut = Lc;
    sum = 0.0;
    ncross = 0;
    ncut = 0;
    nsearch = 0;
    have_g = false;
    neg_prev = false;
  }

  // sqrt(A) Psi |dt/dl| / |dg/dl| at a crossing (scaled), analytic gradients.
  __device__ void contribution(const RayConst<double>& c, const double* y) {
    double f[6];
    rhs64(c, y, f);
    const double r2 = y[0] * y[0] + y[1] * y[1] + y[2] * y[2];
    const double ir = rsqrt(r2);
    const double n0 = y[0] * ir, n1 = y[1] * ir, n2 = y[2] * ir;
    const double A = 1.0 - c.rs * ir;
    const double sA = sqrt(A);
    const double kr = n0 * y[3] + n1 * y[4] + n2 * y[5];
    const double kk = y[3] * y[3] + y[4] * y[4] + y[5] * y[5] + (A - 1.0) * kr * kr;
    const double Ea = sqrt(1.0 + kk);
    const double om = W / sA;
    // dg/dl = (d omega/dx - d|k|^2/dx / 2E_a) . xdot - (d|k|^2/dk / 2E_a) . kdot
    const double dAr = c.rs * ir * ir;                       // dA/dx = dAr n
    const double c_om = -0.5 * om / A * dAr;                  // d omega/dx = c_om n
    const double ckr = 2.0 * (A - 1.0) * kr * ir;
    double dg = 0.0;
#pragma unroll
    for (int i = 0; i < 3; ++i) {
      const double ni = (i == 0) ? n0 : (i == 1) ? n1 : n2;
      const double dkk_dx = kr * kr * dAr * ni + ckr * (y[3 + i] - kr * ni);
      const double dkk_dk = 2.0 * (y[3 + i] + (A - 1.0) * kr * ni);
      dg += (c_om * ni - 0.5 * dkk_dx / Ea) * f[i] - 0.5 * dkk_dk / Ea * f[3 + i];
    }
    // plasma and field at the crossing
    const double mu = c.m0 * n0 + c.m1 * n1 + c.m2 * n2;
    double P = 0.0;
    if (c.plasma == PLASMA_GJ) {
      const double F = 3.0 * n2 * mu - c.m2;
      P = c.cp * ir * ir * ir * fabs(F);
    } else if (c.plasma == PLASMA_HOMOG) {
      P = c.pa;
    } else if (c.plasma == PLASMA_LINEAR_Z) {
      P = c.pa * y[2];
    } else if (c.plasma == PLASMA_RADIAL) {
      P = c.pa * ir * ir * ir;
    } else if (c.plasma == PLASMA_TWISTED) {
      P = c.cp * (1.0 - mu * mu) * ir * ir * ir * ir;
    }
    const double bb = 3.0 * mu * mu + 1.0;
    const double km = y[3] * c.m0 + y[4] * c.m1 + y[5] * c.m2;
    const double Kpb = 3.0 * mu * kr - km + 2.0 * mu * kr * (sA - 1.0);   // k_o . b
    const double Kp2 = Kpb * Kpb / bb;                                     // k_par^2
    // dt/dl = dH/dk_t with k_t = -omega_inf
    const double dtdl =
        fabs((c.disp == DISP_ISO) ? 2.0 * W / A : 2.0 * W / A - 2.0 * P * A * Kp2 / (W * W * W));
    // conversion length E / |dg/ds| (units of R), s the proper length
    const double vn = n0 * f[0] + n1 * f[1] + n2 * f[2];
    const double v2 = f[0] * f[0] + f[1] * f[1] + f[2] * f[2] + (1.0 / A - 1.0) * vn * vn;
    const double Lc = om * sqrt(v2) / fabs(dg);
    ++ncross;
    if (Lc_cut > 0.0 && Lc > Lc_cut) {
      ++ncut;
      return;
    }
    const double ko2 = kk;                                    // |k_o|^2 = g^{ij} k_i k_j
    const double cos2 = Kp2 / ko2;
    const double sin2 = 1.0 - cos2;
    double shape;
    if (c.disp == DISP_ISO) {
      shape = sin2;
    } else {
      const double E2 = om * om;
      const double Dd = cos2 * P * (P - 2.0 * E2) + E2 * E2;
      shape = E2 * E2 * sin2 / Dd;
    }
    const double Bmag = s->B0_eV2 * 0.5 * ir * ir * ir * sqrt(bb);
    const double Psi = 0.5 * PI * s->g_eV * s->g_eV * Bmag * Bmag * shape * (om * s->ma_eV);
    const double ratio = dtdl / fabs(dg) * s->R_eV / s->ma_eV;
    sum += sA * Psi * ratio;
  }

  // Locates the sign change of g on [lo, hi] (g(lo) < 0 iff negA) by FP64
  // bisection on dense64 and adds its contribution.
  template <class Dense64>
  __device__ void root(const RayConst<double>& c, double lo, double hi, bool negA,
                       Dense64& dense64) {
    double yd[6];
    for (int it = 0; it < 200; ++it) {
      const double mid = 0.5 * (lo + hi);
      if (mid <= lo || mid >= hi) break;
      dense64(mid, yd, nullptr);
      if ((crossing_g(c, W, yd) < 0.0) == negA) lo = mid; else hi = mid;
    }
    dense64(0.5 * (lo + hi), yd, nullptr);
    contribution(c, yd);
  }

  // A piece [a, b] whose ends have the same sign of g (negative iff neg)
  // while g turns toward zero inside: the extremum is located by FP64
  // bisection on the sign of dg/dth; if g has the other sign there, the two
  // roots on either side are located and counted.
  template <class Dense64>
  __device__ void graze(const RayConst<double>& c, double a, double b, bool neg,
                        Dense64& dense64) {
    double yd[6], yp[6], g, ga, gb;
    dense64(a, yd, yp);
    crossing_g_slope(c, W, yd, yp, &g, &ga);
    dense64(b, yd, yp);
    crossing_g_slope(c, W, yd, yp, &g, &gb);
    // a minimum of |g| on the side of neg: g' < 0 then > 0 for g > 0
    if (neg ? !(ga > 0.0 && gb < 0.0) : !(ga < 0.0 && gb > 0.0)) return;
    // Illinois (regula falsi with halving of the stale end) on dg/dth
    double lo = a, hi = b, flo = ga, fhi = gb;
    int side = 0;
    for (int it = 0; it < 100 && hi - lo > 1e-13; ++it) {
      double mid = (lo * fhi - hi * flo) / (fhi - flo);
      if (!(mid > lo && mid < hi)) mid = 0.5 * (lo + hi);
      dense64(mid, yd, yp);
      double gm;
      crossing_g_slope(c, W, yd, yp, &g, &gm);
      if ((gm < 0.0) == (flo < 0.0)) {
        lo = mid;
        flo = gm;
        if (side == -1) fhi *= 0.5;
        side = -1;
      } else {
        hi = mid;
        fhi = gm;
        if (side == 1) flo *= 0.5;
        side = 1;
      }
    }
    const double te = 0.5 * (lo + hi);
    dense64(te, yd, nullptr);
    if ((crossing_g(c, W, yd) < 0.0) == neg) return;      // the dip stays on its side
    root(c, a, te, neg, dense64);
    root(c, te, b, !neg, dense64);
  }

  // One accepted step from y to yn with the continuous extension y(th): the
  // sign of g at BACK_SUBDIV + 1 points, screened in FP32 on the pieces
  // p2..p5 of y(th) - y = th (p2 + (1 - th) (p3 + th (p4 + (1 - th) p5)))
  // about y32, evaluated in FP64 at dense64(th) where the screen leaves it
  // open; every sign change located by FP64 bisection; and between two
  // samples of one sign, an extremum of g turning toward zero (bracketed by
  // the FP32 slope of the screened N) searched in FP64 where the two tangent
  // lines at the samples meet within the screen's margin of zero.
  // dense64(th, yd, yp) gives the FP64 point and, if yp is set, dy/dth.  y
  // (read only on a ray's first step) and yn may be null: then dense64 at
  // th = 0 and 1.
  template <class Dense64>
  __device__ void scan(const RayConst<double>& c, const double* y, const double* yn,
                       const Screen& sc, const float* y32, const float* p2, const float* p3,
                       const float* p4, const float* p5, Dense64& dense64) {
    double yd[6];
    if (!have_g) {
      if (!y) dense64(0.0, yd, nullptr);
      neg_prev = crossing_g(c, W, y ? y : yd) < 0.0;
      have_g = true;
    }
    double th0 = 0.0;
    bool negA = neg_prev;
    float NA, slA;
    // pieces whose dip is searched after the loop (bit q - 1), and their sign
    unsigned dips = 0u, dip_neg = 0u;
    {
      const float d[6] = {0.0f, 0.0f, 0.0f, 0.0f, 0.0f, 0.0f};
      float xs[3], ks[3];
#pragma unroll
      for (int i = 0; i < 3; ++i) {
        xs[i] = y32[i];
        ks[i] = y32[3 + i];
      }
      (void)screen_sign(sc, xs, d, ks, &NA);
      slA = 0.0f;
      if (fabsf(NA) < SLOPE_NEAR) {
        float dp[6];
        dense32_slope(0.0f, p2, p3, p4, p5, dp);
        slA = screen_slope(sc, xs, d, ks, dp, dp + 3);
      }
    }
    for (int q = 1; q <= BACK_SUBDIV; ++q) {
      const double th1 = (double)q / BACK_SUBDIV;
      const float t = (float)q * (1.0f / BACK_SUBDIV);
      float d[6], xs[3], ks[3];
      dense32(t, p2, p3, p4, p5, d);
      if (q == BACK_SUBDIV) {
#pragma unroll
        for (int i = 0; i < 6; ++i) d[i] = p2[i];          // the step's own increment
      }
#pragma unroll
      for (int i = 0; i < 3; ++i) {
        xs[i] = y32[i] + d[i];
        ks[i] = y32[3 + i] + d[3 + i];
      }
      float NB;
      const int sg = screen_sign(sc, xs, d, ks, &NB);
      // the slope is needed only where a dip could reach zero: near the
      // resonance at one end of a piece
      const bool nearB = fabsf(NB) < SLOPE_NEAR;
      float slB = 0.0f;
      if (nearB || fabsf(NA) < SLOPE_NEAR) {
        float dp[6];
        if (!(fabsf(NA) < SLOPE_NEAR)) {             // slope at th0 not formed yet
          const float t0 = t - 1.0f / BACK_SUBDIV;
          float d0[6], x0[3], k0[3];
          dense32(t0, p2, p3, p4, p5, d0);
          dense32_slope(t0, p2, p3, p4, p5, dp);
#pragma unroll
          for (int i = 0; i < 3; ++i) {
            x0[i] = y32[i] + d0[i];
            k0[i] = y32[3 + i] + d0[3 + i];
          }
          slA = screen_slope(sc, x0, d0, k0, dp, dp + 3);
        }
        dense32_slope(t, p2, p3, p4, p5, dp);
        slB = screen_slope(sc, xs, d, ks, dp, dp + 3);
      }
      bool negB;
      if (sg != 0) {
        negB = sg < 0;
      } else if (q == BACK_SUBDIV && yn) {
        negB = crossing_g(c, W, yn) < 0.0;
      } else {
        dense64(th1, yd, nullptr);
        negB = crossing_g(c, W, yd) < 0.0;
      }
      if (negA != negB) {
        root(c, th0, th1, negA, dense64);
      } else {
        // s N decreasing at th0 and increasing at th1 (s = sign of g): a dip
        // toward zero between them; the tangent lines at both ends meet at
        // s N = L, a lower bound of the dip where s N is convex
        const float sgn = negA ? -1.0f : 1.0f;
        const float a0 = sgn * NA, a1 = sgn * NB, s0 = sgn * slA, s1 = sgn * slB;
        if (s0 < 0.0f && s1 > 0.0f) {
          const float dth = 1.0f / BACK_SUBDIV;
          float tx = (a1 - a0 - s0 * dth) / (s0 - s1);          // meeting point - th1
          tx = fminf(0.0f, fmaxf(-dth, tx));
          const float L = a1 + s1 * tx;
          const float margin = 0.05f * (2.0f + fabsf(NA) + fabsf(NB));
          if (!(L > margin)) {
            dips |= 1u << (q - 1);
            if (negA) dip_neg |= 1u << (q - 1);
          }
        }
      }
      th0 = th1;
      negA = negB;
      NA = NB;
      slA = slB;
    }
    neg_prev = negA;
    nsearch += __popc(dips);
    while (dips) {
      const int q = __ffs(dips);                   // piece q: [(q - 1), q] / BACK_SUBDIV
      dips &= dips - 1u;
      graze(c, (double)(q - 1) / BACK_SUBDIV, (double)q / BACK_SUBDIV,
            ((dip_neg >> (q - 1)) & 1u) != 0u, dense64);
    }
  }

  // The same from the FP64 pieces y + th (r2 + (1 - th) (r3 + th (r4 + (1 - th)
  // r5))) of the FP64 integrator.
  __device__ void scan_step(const RayConst<double>& c, const double* y, const double* yn,
                            const double* r2, const double* r3, const double* r4,
                            const double* r5) {
    const Screen sc = make_screen(c, y);
    float y32[6], p2[6], p3[6], p4[6], p5[6];
#pragma unroll
    for (int i = 0; i < 6; ++i) {
      y32[i] = (float)y[i];
      p2[i] = (float)r2[i];
      p3[i] = (float)r3[i];
      p4[i] = (float)r4[i];
      p5[i] = (float)r5[i];
    }
    auto dense64 = [&](double th, double* yd, double* yp) {
      const double u = 1.0 - th;
#pragma unroll
      for (int i = 0; i < 6; ++i) {
        const double Q3 = r4[i] + u * r5[i];
        const double Q2 = r3[i] + th * Q3;
        const double Q1 = r2[i] + u * Q2;
        yd[i] = y[i] + th * Q1;
        if (yp) yp[i] = Q1 + th * (u * (Q3 - th * r5[i]) - Q2);
      }
    };
    scan(c, y, yn, sc, y32, p2, p3, p4, p5, dense64);
  }
};

// Initial state of pixel p: position on the plane, time-reversed momentum on
// shell along -o (orthonormal frame); y and the ray constants c in FP64.
__device__ __forceinline__ void pixel_init(const BackParams& bp, int64_t p, double* y,
                                           RayConst<double>& c) {
  const StarDev& s = bp.s;
  const int i = (int)(p % bp.nx), j = (int)(p / bp.nx);
  const double bx = -bp.bmax + (i + 0.5) * (2.0 * bp.bmax / bp.nx);
  const double by = -bp.bmax + (j + 0.5) * (2.0 * bp.bmax / bp.ny);
  double si, ci;
  sincos(bp.incl, &si, &ci);
  const double o[3] = {si, 0.0, ci}, e1[3] = {ci, 0.0, -si};
  y[0] = bp.D * o[0] + bx * e1[0];
  y[1] = by;
  y[2] = bp.D * o[2] + bx * e1[2];
  double sp, cpsi;
  sincos(s.psi_fixed, &sp, &cpsi);
  c.rs = s.rs_prop;
  c.cp = s.cp;
  c.pa = s.plasma_a;
  c.W2 = bp.W * bp.W;
  c.iW2 = 1.0 / (bp.W * bp.W);
  c.m0 = s.sin_tm * cpsi;
  c.m1 = s.sin_tm * sp;
  c.m2 = s.cos_tm;
  c.disp = s.dispersion;
  c.plasma = s.plasma;
  c.sig = gj_side<double>(c.m0, c.m1, c.m2, y[0], y[1], y[2]);
  const double r2 = y[0] * y[0] + y[1] * y[1] + y[2] * y[2];
  const double ir = rsqrt(r2);
  const double n0 = y[0] * ir, n1 = y[1] * ir, n2 = y[2] * ir;
  const double A = 1.0 - c.rs * ir;
  const double dn = -(n0 * o[0] + n1 * o[1] + n2 * o[2]);         // n . d, d = -o
  const double mu = c.m0 * n0 + c.m1 * n1 + c.m2 * n2;
  double P = 0.0;
  if (c.plasma == PLASMA_GJ) P = c.cp * ir * ir * ir * fabs(3.0 * n2 * mu - c.m2);
  else if (c.plasma == PLASMA_HOMOG) P = c.pa;
  else if (c.plasma == PLASMA_LINEAR_Z) P = c.pa * y[2];
  else if (c.plasma == PLASMA_RADIAL) P = c.pa * ir * ir * ir;
  else if (c.plasma == PLASMA_TWISTED) P = c.cp * (1.0 - mu * mu) * ir * ir * ir * ir;
  // H(s) = -W2/A + s^2 + P - P A (s Kd)^2 / W2, Kd = d . bhat (orthonormal)
  const double bn = rsqrt(3.0 * mu * mu + 1.0);
  const double Kd = (3.0 * mu * dn - (-(c.m0 * o[0] + c.m2 * o[2]))) * bn;
  const double den = (c.disp == DISP_ISO) ? 1.0 : 1.0 - P * A * Kd * Kd * c.iW2;
  const double sk = sqrt((c.W2 / A - P) / den);
  const double cr = (1.0 / sqrt(A) - 1.0) * dn;
  y[3] = sk * (-o[0] + cr * n0);
  y[4] = sk * (cr * n1);
  y[5] = sk * (-o[2] + cr * n2);
}

}  // namespace rtk
