// Forward tracing through a rigidly rotating magnetosphere.  The magnetic
// axis turns about the rotation axis z while the photon flies (the cos(Omega t)
// that Eq. GJDensity writes into m.n, kept during the flight instead of a
// snapshot), so the Hamiltonian depends on the coordinate time and Hamilton's
// equations (Eq. Hamilton) carry all four canonical pairs.  State of a ray
// (units of R and m_a): y = (x, k, t, omega) with omega = -k_t, and
//
//   dx/dl, dk/dl   ham_rhs with the axis m(psi0 + Omega t) and W2 = omega^2
//   dt/dl        = dH/dk_t = -2 omega dH/dW2
//   domega/dl    = dH/dt   = -Omega [(x x dH/dx)_z + (k x dH/dk)_z]
//
// the last because H depends on t only through a rotation of x and k about z
// by -Omega t (the metric is spherical, and the plasma and the field turn
// rigidly).  So omega - Omega L_z is conserved, L_z = x k_y - y k_x, and the
// frequency at infinity is Doppler shifted by Omega times the change of L_z.
//
// One thread per ray, persistent, with the warp refill of the static kernel;
// the Dormand-Prince 5(4) pair of rt_integrator.cuh on eight components, the
// error norm and the initial step over x and k (t and omega follow the step
// sequence that x and k choose), and the null-cone side taken with the axis
// at each point's own t.
#include <cuda_runtime.h>
#include <stdint.h>

#include "rt_device.cuh"
#include "rt_integrator.cuh"
#include "rt_internal.h"

namespace rtk {

namespace {

struct RotLane {
  RayConst<double> c;  // m0, m1, W2, iW2 rewritten at every evaluation
  double sin_tm, psi0, Om;
  double y[8], f0[8];
  double h, lam, h_resume;
  double om0, delta0;
  int na, nr;
  bool last_rej, switching;
  double R_km, ma_eV;
};

__device__ __forceinline__ void rhs_rot(RotLane& L, const double* y, double* f) {
  double sp, cp;
  sincos(L.psi0 + L.Om * y[6], &sp, &cp);
  L.c.m0 = L.sin_tm * cp;
  L.c.m1 = L.sin_tm * sp;
  L.c.W2 = y[7] * y[7];
  L.c.iW2 = 1.0 / L.c.W2;
  double dw;
  ham_rhs<double, false, false, true>(L.c, y[0], y[1], y[2], y[3], y[4], y[5], f[0], f[1], f[2],
                                      f[3], f[4], f[5], 0.0, &dw);
  f[6] = -2.0 * y[7] * dw;
  // dH/dx = -(f3, f4, f5), dH/dk = (f0, f1, f2)
  f[7] = L.Om * (y[0] * f[4] - y[1] * f[3] - y[3] * f[1] + y[4] * f[0]);
}

// sign of Omega . B at the point (x, t): the side of the turning null cone
__device__ __forceinline__ double side_at(const RotLane& L, const double* y) {
  double sp, cp;
  sincos(L.psi0 + L.Om * y[6], &sp, &cp);
  return gj_side<double>(L.sin_tm * cp, L.sin_tm * sp, L.c.m2, y[0], y[1], y[2]);
}

__device__ __forceinline__ int star_of(const TraceParams& p, int64_t i) {
  if (p.nstars <= 1) return 0;
  int lo = 0, hi = p.nstars - 1;
  while (lo < hi) {
    const int mid = (lo + hi + 1) >> 1;
    if (p.offsets[mid] <= i) lo = mid; else hi = mid - 1;
  }
  return lo;
}

// Hairer's two-evaluation initial step, norms over x and k.
__device__ double initial_step_rot(RotLane& L, double rtol, double atol, double hmax) {
  const double* y0 = L.y;
  const double* f0 = L.f0;
  double dnf = 0.0, dny = 0.0;
#pragma unroll
  for (int i = 0; i < 6; ++i) {
    const double sk = atol + rtol * fabs(y0[i]);
    dnf += (f0[i] / sk) * (f0[i] / sk);
    dny += (y0[i] / sk) * (y0[i] / sk);
  }
  double h = (dnf <= 1e-10 || dny <= 1e-10) ? 1e-6 : sqrt(dny / dnf) * 0.01;
  h = fmin(h, hmax);
  double y1[8], f1[8];
#pragma unroll
  for (int i = 0; i < 8; ++i) y1[i] = y0[i] + h * f0[i];
  rhs_rot(L, y1, f1);
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

__device__ void load_rot(const TraceParams& p, int64_t i, RotLane& L) {
  const StarDev& s = p.stars[star_of(p, i)];
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
  L.delta0 = p.state[6 * n + i];
  L.om0 = 1.0 + L.delta0;
  L.y[6] = 0.0;          // the clock starts at emission, where the phase is psi0
  L.y[7] = L.om0;
  L.psi0 = p.state[7 * n + i];
  L.sin_tm = s.sin_tm;
  L.Om = 1.0 / s.rlc;    // Omega R / c
  L.c.rs = s.rs_prop;
  L.c.cp = s.cp;
  L.c.pa = s.plasma_a;
  L.c.m2 = s.cos_tm;
  L.c.disp = s.dispersion;
  L.c.plasma = s.plasma;
  L.c.sig = side_at(L, L.y);
  L.switching = false;
  L.h_resume = 0.0;
  rhs_rot(L, L.y, L.f0);
  const double hmax = (p.lambda_max > 0.0) ? p.lambda_max : 1e30;
  L.h = initial_step_rot(L, p.rtol, p.atol, hmax);
  L.lam = 0.0;
  L.na = 0;
  L.nr = 0;
  L.last_rej = false;
}

__device__ void store_rot(const TraceParams& p, int64_t i, const RotLane& L, int st) {
  const int64_t n = p.n;
  p.state[i] = L.y[0] * L.R_km;
  p.state[n + i] = L.y[1] * L.R_km;
  p.state[2 * n + i] = L.y[2] * L.R_km;
  p.state[3 * n + i] = L.y[3] * L.ma_eV;
  p.state[4 * n + i] = L.y[4] * L.ma_eV;
  p.state[5 * n + i] = L.y[5] * L.ma_eV;
  p.state[6 * n + i] = L.delta0 + (L.y[7] - L.om0);   // omega_inf / m_a - 1 at the end
  p.state[7 * n + i] = L.psi0 + L.Om * L.y[6];        // rotation phase at the end
  status_after_state(p, i, st);
  if (p.nacc) p.nacc[i] = L.na;
  if (p.nrej) p.nrej[i] = L.nr;
}

// One attempted step; returns -1 to continue, else the final ray status.
__device__ int advance_rot(const TraceParams& p, RotLane& L) {
  if (L.na >= p.max_steps || L.na + L.nr >= 4 * p.max_steps) return RAY_MAXSTEPS;
  bool clipped = false;
  double h = L.h;
  {
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
  double t[8], k2[8], k3[8], k4[8], k5[8], k6[8], k7[8], yn[8];
#pragma unroll
  for (int i = 0; i < 8; ++i) t[i] = y[i] + h * (DP::a21 * k1[i]);
  rhs_rot(L, t, k2);
#pragma unroll
  for (int i = 0; i < 8; ++i) t[i] = y[i] + h * (DP::a31 * k1[i] + DP::a32 * k2[i]);
  rhs_rot(L, t, k3);
#pragma unroll
  for (int i = 0; i < 8; ++i)
    t[i] = y[i] + h * (DP::a41 * k1[i] + DP::a42 * k2[i] + DP::a43 * k3[i]);
  rhs_rot(L, t, k4);
#pragma unroll
  for (int i = 0; i < 8; ++i)
    t[i] = y[i] + h * (DP::a51 * k1[i] + DP::a52 * k2[i] + DP::a53 * k3[i] + DP::a54 * k4[i]);
  rhs_rot(L, t, k5);
#pragma unroll
  for (int i = 0; i < 8; ++i)
    t[i] = y[i] + h * (DP::a61 * k1[i] + DP::a62 * k2[i] + DP::a63 * k3[i] + DP::a64 * k4[i] +
                       DP::a65 * k5[i]);
  rhs_rot(L, t, k6);
#pragma unroll
  for (int i = 0; i < 8; ++i)
    yn[i] = y[i] + h * (DP::b1 * k1[i] + DP::b3 * k3[i] + DP::b4 * k4[i] + DP::b5 * k5[i] +
                        DP::b6 * k6[i]);
  rhs_rot(L, yn, k7);
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
  // continuous extension of the step: y(th) = y + th (r2 + (1-th)(r3 + th(r4 + (1-th) r5)))
  auto dense = [&](double th, double* out, double* r2, double* r3, double* r4, double* r5,
                   int nc) {
    for (int i = 0; i < nc; ++i)
      out[i] = y[i] + th * (r2[i] + (1.0 - th) * (r3[i] + th * (r4[i] + (1.0 - th) * r5[i])));
  };
  const bool gj = (L.c.plasma == PLASMA_GJ);
  if (en <= 1.0 && gj && !L.switching && L.c.sig * side_at(L, yn) < 0.0) {
    // the step crossed the turning null cone: the largest th whose point (x,
    // at its own t) is on the start side, by Illinois on the continuous
    // extension; then redo the step to end just past it
    double r2[8], r3[8], r4[8], r5[8];
#pragma unroll
    for (int i = 0; i < 8; ++i) {
      r2[i] = yn[i] - y[i];
      r3[i] = h * k1[i] - r2[i];
      r4[i] = r2[i] - h * k7[i] - r3[i];
      r5[i] = h * (DP::d1 * k1[i] + DP::d3 * k3[i] + DP::d4 * k4[i] + DP::d5 * k5[i] +
                   DP::d6 * k6[i] + DP::d7 * k7[i]);
    }
    const double sgn = L.c.sig;
    auto side_val = [&](double th) {
      double yd[8];
      dense(th, yd, r2, r3, r4, r5, 8);
      double sp, cp;
      sincos(L.psi0 + L.Om * yd[6], &sp, &cp);
      const double m0 = L.sin_tm * cp, m1 = L.sin_tm * sp, m2 = L.c.m2;
      const double mx = m0 * yd[0] + m1 * yd[1] + m2 * yd[2];
      const double rr = yd[0] * yd[0] + yd[1] * yd[1] + yd[2] * yd[2];
      return sgn * (3.0 * yd[2] * mx - m2 * rr);
    };
    double flo = side_val(0.0), fhi = side_val(1.0);
    if (!(flo >= 0.0)) flo = 0.0;
    if (!(fhi < 0.0)) fhi = -1e-300;
    double hi;
    const double lo = last_nonneg(side_val, flo, fhi, &hi);
    ++L.nr;
    if (lo < SWITCH_MIN_FRACTION) {
      L.c.sig = -L.c.sig;
      rhs_rot(L, L.y, L.f0);
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
    const double rnew2 = yn[0] * yn[0] + yn[1] * yn[1] + yn[2] * yn[2];
    if (rnew2 >= p.r_out * p.r_out) {
      double r2[8], r3[8], r4[8], r5[8];
#pragma unroll
      for (int i = 0; i < 8; ++i) {
        r2[i] = yn[i] - y[i];
        r3[i] = h * k1[i] - r2[i];
        r4[i] = r2[i] - h * k7[i] - r3[i];
        r5[i] = h * (DP::d1 * k1[i] + DP::d3 * k3[i] + DP::d4 * k4[i] + DP::d5 * k5[i] +
                     DP::d6 * k6[i] + DP::d7 * k7[i]);
      }
      const double ro2 = p.r_out * p.r_out;
      auto inside = [&](double th) {
        double xd[3];
        dense(th, xd, r2, r3, r4, r5, 3);
        return ro2 - (xd[0] * xd[0] + xd[1] * xd[1] + xd[2] * xd[2]);
      };
      double flo = ro2 - (y[0] * y[0] + y[1] * y[1] + y[2] * y[2]);
      if (!(flo >= 0.0)) flo = 0.0;
      double fhi = ro2 - rnew2;
      if (!(fhi < 0.0)) fhi = -1e-300;
      double hi;
      const double lo = last_nonneg(inside, flo, fhi, &hi);
      const double th = 0.5 * (lo + hi);
      dense(th, yn, r2, r3, r4, r5, 8);
#pragma unroll
      for (int i = 0; i < 8; ++i) L.y[i] = yn[i];
      L.lam += th * h;
      return RAY_ESCAPED;
    }
#pragma unroll
    for (int i = 0; i < 8; ++i) {
      L.y[i] = yn[i];
      L.f0[i] = k7[i];
    }
    L.lam += h;
    if (rnew2 <= p.r_capture * p.r_capture) return RAY_CAPTURED;
    if (clipped) return RAY_LAMBDA_END;
    if (gj && L.c.sig * side_at(L, L.y) < 0.0) {
      L.c.sig = -L.c.sig;
      rhs_rot(L, L.y, L.f0);
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

__global__ void __launch_bounds__(128) trace_rot_kernel(TraceParams p) {
  const int lane = threadIdx.x & 31;
  int64_t ray = -1;   // -1: needs a ray, -2: queue exhausted
  RotLane L;
  long long acc = 0, rej = 0, traced = 0, esc = 0;
  const int64_t nq = p.order ? (int64_t)COST_BUCKETS * p.n : p.n;   // cost-ordered passes
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
        const int pass = p.order ? (int)(idx / p.n) : 0;
        const int64_t i = idx - (int64_t)pass * p.n;
        if (idx >= nq) {
          ray = -2;
        } else if (p.status[i] != p.claim_status ||
                   (p.order && (cost_bucket(p.stars[star_of(p, i)], p.state, p.n, i) != pass ||
                                !status_still(p, i, p.claim_status)))) {
          ray = -1;
        } else {
          ray = i;
          load_rot(p, i, L);
        }
      }
    }
    if (__ballot_sync(FULL, ray != -2) == 0) break;
    if (ray >= 0) {
      const int st = advance_rot(p, L);
      if (st >= 0) {
        store_rot(p, ray, L, st);
        if (p.ts) atomicMax(p.ts + 1 + star_of(p, ray), global_ns());
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

cudaError_t launch_trace_rot(const TraceParams& p, int block, int blocks_per_sm,
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
    e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, trace_rot_kernel, block, 0);
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
  trace_rot_kernel<<<(unsigned)grid, block, 0, stream>>>(p);
  return cudaGetLastError();
}

}  // namespace rtk
