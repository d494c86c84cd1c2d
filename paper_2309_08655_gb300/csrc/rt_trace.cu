// Persistent forward ray-tracing kernel: one thread per ray, Dormand-Prince
// 5(4) adaptive integration of Hamilton's equations (Eq. Hamilton) with the
// analytic right-hand side of rt_device.cuh, warp-level refill of finished
// lanes from a global work queue (ballot + popc prefix, one atomic per warp
// refill).  Termination (Sec. 2.2): r = r_out located on the dense output,
// capture at r <= r_capture, lambda_max, or the step bounds.
#include <cuda_runtime.h>
#include <stdint.h>

#include "rt_device.cuh"
#include "rt_integrator.cuh"
#include "rt_internal.h"

namespace rtk {

namespace {

__device__ __forceinline__ int find_star(const TraceParams& p, int64_t i) {
  if (p.nstars <= 1) return 0;
  int lo = 0, hi = p.nstars - 1;   // offsets[s] <= i < offsets[s + 1]
  while (lo < hi) {
    const int mid = (lo + hi + 1) >> 1;
    if (p.offsets[mid] <= i) lo = mid; else hi = mid - 1;
  }
  return lo;
}

__device__ void load_lane(const TraceParams& p, int64_t i, Lane& L) {
  const StarDev& s = p.stars[find_star(p, i)];
  const int64_t n = p.n;
  L.R_km = s.R_km;
  L.ma_eV = s.ma_eV;
  const double iR = 1.0 / s.R_km, im = 1.0 / s.ma_eV;
  L.y[0] = p.state[i] * iR;
  L.y[1] = p.state[n + i] * iR;
  L.y[2] = p.state[2 * n + i] * iR;
  L.y[3] = p.state[3 * n + i] * im;
  L.y[4] = p.state[4 * n + i] * im;
  L.y[5] = p.state[5 * n + i] * im;
  const double om = 1.0 + p.state[6 * n + i];
  const double psi = p.state[7 * n + i];
  double sp, cpsi;
  sincos(psi, &sp, &cpsi);
  L.c.rs = s.rs_prop;
  L.c.cp = s.cp;
  L.c.pa = s.plasma_a;
  L.c.W2 = om * om;
  L.c.iW2 = 1.0 / (om * om);
  L.c.m0 = s.sin_tm * cpsi;
  L.c.m1 = s.sin_tm * sp;
  L.c.m2 = s.cos_tm;
  L.c.disp = s.dispersion;
  L.c.plasma = s.plasma;
  L.c.sig = gj_side<double>(L.c.m0, L.c.m1, L.c.m2, L.y[0], L.y[1], L.y[2]);
  L.switching = false;
  L.h_resume = 0.0;
  rhs64(L.c, L.y, L.f0);
  const double hmax = (p.lambda_max > 0.0) ? p.lambda_max : 1e30;
  L.h = initial_step(L.c, L.y, L.f0, p.rtol, p.atol, hmax);
  L.lam = 0.0;
  L.na = 0;
  L.nr = 0;
  if (p.claim_status == RAY_PROMOTED) {   // resume a ray handed over by the FP32 pass
    if (p.nacc) L.na = p.nacc[i];
    if (p.nrej) L.nr = p.nrej[i];
  }
  L.last_rej = false;
}

__device__ void store_lane(const TraceParams& p, int64_t i, const Lane& L, int st) {
  const int64_t n = p.n;
  p.state[i] = L.y[0] * L.R_km;
  p.state[n + i] = L.y[1] * L.R_km;
  p.state[2 * n + i] = L.y[2] * L.R_km;
  p.state[3 * n + i] = L.y[3] * L.ma_eV;
  p.state[4 * n + i] = L.y[4] * L.ma_eV;
  p.state[5 * n + i] = L.y[5] * L.ma_eV;
  p.status[i] = (uint8_t)st;
  if (p.nacc) p.nacc[i] = L.na;
  if (p.nrej) p.nrej[i] = L.nr;
}

__global__ void __launch_bounds__(128) trace_fp64_kernel(TraceParams p) {
  const int lane = threadIdx.x & 31;
  int64_t ray = -1;   // -1: needs a ray, -2: queue exhausted
  Lane L;
  long long acc = 0, rej = 0, traced = 0, esc = 0;
  int na0 = 0, nr0 = 0;   // steps a resumed ray had already taken in FP32
  if (p.ts && threadIdx.x == 0) atomicMin(p.ts, global_ns());
  for (;;) {
    const bool need = (ray == -1);
    const unsigned mneed = __ballot_sync(FULL, need);
    if (mneed) {
      const int leader = __ffs(mneed) - 1;
      unsigned long long base = 0;
      if (lane == leader) base = atomicAdd(p.queue, (unsigned long long)__popc(mneed));
      base = __shfl_sync(FULL, base, leader);
      if (need) {
        const int64_t idx = (int64_t)base + __popc(mneed & ((1u << lane) - 1u));
        if (idx >= p.n) {
          ray = -2;
        } else if (p.status[idx] != p.claim_status) {
          ray = -1;
        } else {
          ray = idx;
          load_lane(p, idx, L);
          na0 = L.na;
          nr0 = L.nr;
        }
      }
    }
    const unsigned live = __ballot_sync(FULL, ray != -2);
    if (live == 0) break;
    if (p.park) {
      // the queue has drained and this warp holds few rays: park them for the
      // six-lanes-per-ray tail kernel (the complete integrator state)
      const unsigned has = __ballot_sync(FULL, ray >= 0);
      const unsigned drained = __ballot_sync(FULL, ray == -2);
      if (drained && has && __popc(has) <= p.park_live && ray >= 0) {
        const unsigned long long slot = atomicAdd(p.park_count, 1ull);
        if (slot < (unsigned long long)p.park_cap) {
          double* pe = p.park + slot * PARKREC;
#pragma unroll
          for (int j = 0; j < 6; ++j) pe[j] = L.y[j];
          pe[6] = L.h;
          pe[7] = L.h_resume;
          pe[8] = L.c.sig;
          pe[9] = (double)((L.last_rej ? 1 : 0) | (L.switching ? 2 : 0));
          pe[10] = (double)L.na;
          pe[11] = (double)L.nr;
          pe[12] = (double)ray;
          pe[13] = L.lam;
          acc += L.na - na0;
          rej += L.nr - nr0;
          ray = -2;
        }
      }
    }
    if (ray >= 0) {
      NoHook nh;
      const int st = advance(p, L, nh);
      if (st >= 0) {
        store_lane(p, ray, L, st);
        if (p.ts) atomicMax(p.ts + 1 + find_star(p, ray), global_ns());
        acc += L.na - na0;
        rej += L.nr - nr0;
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
      if (p.claim_status == RAY_PROMOTED)
        atomicAdd((unsigned long long*)&p.counters[CTR_PROMOTED_STEPS],
                  (unsigned long long)(acc + rej));
    }
  }
}

// ---------------------------------------------------------------------------
// Backward image plane (Sec. 2.1, Eq. BackPower; all level crossings,
// Sec. 5.1.3).  By Liouville's theorem the forward phase-space integral
// P = int d^3x d^3k j, j = sqrt(A) delta(E_gamma - E_a) Psi f_a, equals
// dP/dOmega = int dA int domega omega^2 int_ray j dt over the photons crossing
// a distant plane; the ray integral of the delta function is a sum over the
// crossings of g = E_gamma - E_a = omega - sqrt(m_a^2 + |k|^2) along the ray,
// sum_c sqrt(A) Psi f_a |dt/dl| / |dg/dl|.  Each pixel's time-reversed ray
// (k -> -k; H is even in k) is traced inward from the plane; the sign of g is
// sampled at BACK_SUBDIV points of every accepted step on the continuous
// extension (a ray turning near the resonance crosses it twice within one
// step) and every sign change is located by bisection.

constexpr int BACK_SUBDIV = 16;

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
};

__device__ __forceinline__ double crossing_g(const RayConst<double>& c, double W,
                                             const double* y) {
  const double r2 = y[0] * y[0] + y[1] * y[1] + y[2] * y[2];
  const double ir = rsqrt(r2);
  const double A = 1.0 - c.rs * ir;
  const double kr = (y[0] * y[3] + y[1] * y[4] + y[2] * y[5]) * ir;
  const double kk = y[3] * y[3] + y[4] * y[4] + y[5] * y[5] + (A - 1.0) * kr * kr;
  return W * rsqrt(A) - sqrt(1.0 + kk);
}

struct CrossingHook {
  const StarDev* s;
  double W, Lc_cut;
  double sum;
  int ncross, ncut;
  bool have_g;
  double g_prev;

  // sqrt(A) Psi |dt/dl| / |dg/dl| at a crossing (scaled), analytic gradients.
  __device__ void contribution(const Lane& L, const double* y) {
    const RayConst<double>& c = L.c;
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

  __device__ void on_accept(const Lane& L, const double* y, const double* yn, const double* k1,
                            const double* k3, const double* k4, const double* k5,
                            const double* k6, const double* k7, double h) {
    if (!have_g) {
      g_prev = crossing_g(L.c, W, y);
      have_g = true;
    }
    double r2[6], r3[6], r4[6], r5[6];
#pragma unroll
    for (int i = 0; i < 6; ++i) {
      r2[i] = yn[i] - y[i];
      r3[i] = h * k1[i] - r2[i];
      r4[i] = r2[i] - h * k7[i] - r3[i];
      r5[i] = h * (DP::d1 * k1[i] + DP::d3 * k3[i] + DP::d4 * k4[i] + DP::d5 * k5[i] +
                   DP::d6 * k6[i] + DP::d7 * k7[i]);
    }
    double yd[6];
    double th0 = 0.0, gA = g_prev;
    for (int q = 1; q <= BACK_SUBDIV; ++q) {
      const double th1 = (double)q / BACK_SUBDIV;
      double gB;
      if (q == BACK_SUBDIV) {
        gB = crossing_g(L.c, W, yn);
      } else {
#pragma unroll
        for (int i = 0; i < 6; ++i)
          yd[i] = y[i] + th1 * (r2[i] + (1.0 - th1) * (r3[i] + th1 * (r4[i] + (1.0 - th1) * r5[i])));
        gB = crossing_g(L.c, W, yd);
      }
      if ((gA < 0.0) != (gB < 0.0)) {
        double lo = th0, hi = th1;
        const bool negA = gA < 0.0;
        for (int it = 0; it < 200; ++it) {
          const double mid = 0.5 * (lo + hi);
          if (mid <= lo || mid >= hi) break;
#pragma unroll
          for (int i = 0; i < 6; ++i)
            yd[i] = y[i] + mid * (r2[i] + (1.0 - mid) * (r3[i] + mid * (r4[i] + (1.0 - mid) * r5[i])));
          if ((crossing_g(L.c, W, yd) < 0.0) == negA) lo = mid; else hi = mid;
        }
        const double th = 0.5 * (lo + hi);
#pragma unroll
        for (int i = 0; i < 6; ++i)
          yd[i] = y[i] + th * (r2[i] + (1.0 - th) * (r3[i] + th * (r4[i] + (1.0 - th) * r5[i])));
        contribution(L, yd);
      }
      th0 = th1;
      gA = gB;
    }
    g_prev = gA;
  }
};

// Initial state of pixel p: position on the plane, time-reversed momentum on
// shell along -o (orthonormal frame).
__device__ void load_pixel(const BackParams& bp, int64_t p, Lane& L) {
  const StarDev& s = bp.s;
  const int i = (int)(p % bp.nx), j = (int)(p / bp.nx);
  const double bx = -bp.bmax + (i + 0.5) * (2.0 * bp.bmax / bp.nx);
  const double by = -bp.bmax + (j + 0.5) * (2.0 * bp.bmax / bp.ny);
  double si, ci;
  sincos(bp.incl, &si, &ci);
  const double o[3] = {si, 0.0, ci}, e1[3] = {ci, 0.0, -si};
  L.y[0] = bp.D * o[0] + bx * e1[0];
  L.y[1] = by;
  L.y[2] = bp.D * o[2] + bx * e1[2];
  L.R_km = s.R_km;
  L.ma_eV = s.ma_eV;
  double sp, cpsi;
  sincos(s.psi_fixed, &sp, &cpsi);
  L.c.rs = s.rs_prop;
  L.c.cp = s.cp;
  L.c.pa = s.plasma_a;
  L.c.W2 = bp.W * bp.W;
  L.c.iW2 = 1.0 / (bp.W * bp.W);
  L.c.m0 = s.sin_tm * cpsi;
  L.c.m1 = s.sin_tm * sp;
  L.c.m2 = s.cos_tm;
  L.c.disp = s.dispersion;
  L.c.plasma = s.plasma;
  L.c.sig = gj_side<double>(L.c.m0, L.c.m1, L.c.m2, L.y[0], L.y[1], L.y[2]);
  const double r2 = L.y[0] * L.y[0] + L.y[1] * L.y[1] + L.y[2] * L.y[2];
  const double ir = rsqrt(r2);
  const double n0 = L.y[0] * ir, n1 = L.y[1] * ir, n2 = L.y[2] * ir;
  const double A = 1.0 - L.c.rs * ir;
  const double dn = -(n0 * o[0] + n1 * o[1] + n2 * o[2]);         // n . d, d = -o
  const double mu = L.c.m0 * n0 + L.c.m1 * n1 + L.c.m2 * n2;
  double P = 0.0;
  if (L.c.plasma == PLASMA_GJ) P = L.c.cp * ir * ir * ir * fabs(3.0 * n2 * mu - L.c.m2);
  else if (L.c.plasma == PLASMA_HOMOG) P = L.c.pa;
  else if (L.c.plasma == PLASMA_LINEAR_Z) P = L.c.pa * L.y[2];
  else if (L.c.plasma == PLASMA_RADIAL) P = L.c.pa * ir * ir * ir;
  // H(s) = -W2/A + s^2 + P - P A (s Kd)^2 / W2, Kd = d . bhat (orthonormal)
  const double bn = rsqrt(3.0 * mu * mu + 1.0);
  const double Kd = (3.0 * mu * dn - (-(L.c.m0 * o[0] + L.c.m2 * o[2]))) * bn;
  const double den = (L.c.disp == DISP_ISO) ? 1.0 : 1.0 - P * A * Kd * Kd * L.c.iW2;
  const double sk = sqrt((L.c.W2 / A - P) / den);
  const double cr = (1.0 / sqrt(A) - 1.0) * dn;
  L.y[3] = sk * (-o[0] + cr * n0);
  L.y[4] = sk * (cr * n1);
  L.y[5] = sk * (-o[2] + cr * n2);
  L.switching = false;
  L.h_resume = 0.0;
  rhs64(L.c, L.y, L.f0);
  L.h = initial_step(L.c, L.y, L.f0, bp.rtol, bp.atol, 1e30);
  L.lam = 0.0;
  L.na = 0;
  L.nr = 0;
  L.last_rej = false;
}

__global__ void __launch_bounds__(128) backward_kernel(BackParams bp) {
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
  Lane L;
  CrossingHook hk;
  long long acc = 0, rej = 0, done = 0, esc = 0, nc = 0;
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
          load_pixel(bp, idx, L);
          // escaped once back at the distance the ray started from
          tp.r_out = sqrt(L.y[0] * L.y[0] + L.y[1] * L.y[1] + L.y[2] * L.y[2]);
          hk.s = &bp.s;
          hk.W = bp.W;
          hk.Lc_cut = bp.Lc_cut;
          hk.sum = 0.0;
          hk.ncross = 0;
          hk.ncut = 0;
          hk.have_g = false;
          hk.g_prev = 0.0;
        }
      }
    }
    if (__ballot_sync(FULL, pix != -2) == 0) break;
    if (pix >= 0) {
      const int st = advance(tp, L, hk);
      if (st >= 0) {
        bp.image[pix] = bp.img_scale * hk.sum;
        if (bp.ts) atomicMax(bp.ts + 1, global_ns());
        bp.status[pix] = (uint8_t)st;
        if (bp.ncross) bp.ncross[pix] = hk.ncross - hk.ncut;
        acc += L.na;
        rej += L.nr;
        done += 1;
        esc += (st == RAY_ESCAPED);
        nc += hk.ncross - hk.ncut;
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
    }
    if (lane == 0) {
      atomicAdd((unsigned long long*)&bp.counters[CTR_ACC], (unsigned long long)acc);
      atomicAdd((unsigned long long*)&bp.counters[CTR_REJ], (unsigned long long)rej);
      atomicAdd((unsigned long long*)&bp.counters[CTR_RAYS], (unsigned long long)done);
      atomicAdd((unsigned long long*)&bp.counters[CTR_ESC], (unsigned long long)esc);
      atomicAdd((unsigned long long*)&bp.counters[CTR_CROSS], (unsigned long long)nc);
    }
  }
}

}  // namespace

cudaError_t launch_backward(const BackLaunch& b, cudaStream_t stream) {
  int dev = 0, nsm = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return e;
  e = cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev);
  if (e != cudaSuccess) return e;
  BackParams bp;
  bp.s = *b.star;
  bp.nx = b.nx;
  bp.ny = b.ny;
  bp.incl = b.incl;
  bp.D = b.D;
  bp.bmax = b.bmax;
  bp.W = b.W;
  bp.Lc_cut = b.Lc_cut;
  bp.img_scale = b.img_scale;
  bp.image = b.image;
  bp.status = b.status;
  bp.ncross = b.ncross;
  bp.counters = b.counters;
  bp.queue = b.queue;
  bp.rtol = b.rtol;
  bp.atol = b.atol;
  bp.r_capture = b.r_capture;
  bp.ts = b.ts;
  bp.max_steps = b.max_steps;
  const int block = 128;
  int occ = 0;
  e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, backward_kernel, block, 0);
  if (e != cudaSuccess) return e;
  const int64_t npix = (int64_t)b.nx * b.ny;
  int64_t grid = (int64_t)nsm * (occ > 0 ? occ : 1);
  const int64_t max_useful = (npix + block - 1) / block;
  if (grid > max_useful) grid = max_useful;
  if (grid < 1) grid = 1;
  e = cudaMemsetAsync(b.queue, 0, sizeof(unsigned long long), stream);
  if (e != cudaSuccess) return e;
  backward_kernel<<<(unsigned)grid, block, 0, stream>>>(bp);
  return cudaGetLastError();
}

namespace {
__global__ void ts_reset_kernel(unsigned long long* ts, int n) {
  for (int i = threadIdx.x; i <= n; i += blockDim.x) ts[i] = (i == 0) ? ~0ull : 0ull;
}
}  // namespace

cudaError_t launch_ts_reset(unsigned long long* ts, int n, cudaStream_t stream) {
  ts_reset_kernel<<<1, 256, 0, stream>>>(ts, n);
  return cudaGetLastError();
}

cudaError_t occupancy_fp64(int block, int* occ) {
  return cudaOccupancyMaxActiveBlocksPerMultiprocessor(occ, trace_fp64_kernel, block, 0);
}

cudaError_t launch_trace_fp64(const TraceParams& p, int block, int blocks_per_sm,
                              cudaStream_t stream) {
  int dev = 0, nsm = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return e;
  e = cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev);
  if (e != cudaSuccess) return e;
  if (block <= 0) block = 128;
  if (block > 128) block = 128;            // __launch_bounds__(128)
  block = (block / 32) * 32;
  if (block < 32) block = 32;
  if (blocks_per_sm <= 0) {
    int occ = 0;
    e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, trace_fp64_kernel, block, 0);
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
  if (p.park) {
    e = cudaMemsetAsync(p.park_count, 0, 2 * sizeof(unsigned long long), stream);
    if (e != cudaSuccess) return e;
  }
  trace_fp64_kernel<<<(unsigned)grid, block, 0, stream>>>(p);
  e = cudaGetLastError();
  if (e != cudaSuccess || !p.park) return e;
  return launch_tail_fp64(p, stream);
}

}  // namespace rtk
