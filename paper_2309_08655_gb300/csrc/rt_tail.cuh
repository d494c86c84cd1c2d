// Six lanes per ray: the group integrator of the FP64 tail mode (rt_tail.cu)
// and of the express lane of cost-ordered tracing (rt_trace.cu).
//
// On GB300 an FP64 warp instruction occupies its SM sub-partition for the same
// 64 cycles whether 1 or 32 lanes are live, so once the work queue has drained
// a warp that still holds a few long rays (those guided along the
// Goldreich-Julian null cone take 10^4 - 10^5 steps) spends the FP64 pipe on
// one lane per instruction.  Such rays are parked by the persistent kernel
// (their complete integrator state, so the continuation is the same
// computation) and continued with one lane per state component: lane c
// of a six-lane group owns y_c, its stage derivatives and the stage sums, and
// evaluates the c-th component of the right-hand side after the scalar prefix
// that every component shares.  Shuffles within the group (not the FP64 pipe)
// assemble each stage input.  The steps, the error norm, the controller and
// the events are those of advance() in rt_integrator.cuh; the arithmetic of
// the component sums and of the error-norm sum is ordered differently, so
// results agree with the lane-per-ray path to rounding.
#pragma once
#include <cuda_runtime.h>
#include <stdint.h>

#include "rt_device.cuh"
#include "rt_integrator.cuh"
#include "rt_internal.h"

namespace rtk {

namespace {

constexpr int GROUP = 6;           // lanes per ray
constexpr int GROUPS_PER_WARP = 5;

__device__ __forceinline__ int find_star_t(const TraceParams& p, int64_t i) {
  if (p.nstars <= 1) return 0;
  int lo = 0, hi = p.nstars - 1;
  while (lo < hi) {
    const int mid = (lo + hi + 1) >> 1;
    if (p.offsets[mid] <= i) lo = mid; else hi = mid - 1;
  }
  return lo;
}

// Component c (0-2: dx_c/dl, 3-5: dk_{c-3}/dl) of ham_rhs at the full state y.
// The scalar prefix is evaluated by every lane, except that its three dot
// products and its two independent reciprocal square roots are spread over
// the group's lanes (one FP64 instruction sequence for all, then shuffles:
// the same operations and operands, so the same results); each lane then
// takes its component from coefficients that all lanes form.
__device__ double rhs_comp(const RayConst<double>& c, const double* y, int comp, unsigned gm,
                           int base) {
  const double x0 = y[0], x1 = y[1], x2 = y[2], k0 = y[3], k1 = y[4], k2 = y[5];
  const double r2 = x0 * x0 + x1 * x1 + x2 * x2;
  const double ir = rsqrt(r2);
  const double n0 = x0 * ir, n1 = x1 * ir, n2 = x2 * ir;
  const double ir2 = ir * ir;
  const double A = 1.0 - c.rs * ir;
  const double Am1 = -c.rs * ir;
  const int j = comp < 3 ? comp : comp - 3;
  // n.k (lane 0), m.n (lane 1), k.m (lane 2) in one pass
  const double a0 = j == 0 ? n0 : (j == 1 ? c.m0 : k0);
  const double a1 = j == 0 ? n1 : (j == 1 ? c.m1 : k1);
  const double a2 = j == 0 ? n2 : (j == 1 ? c.m2 : k2);
  const double b0 = j == 0 ? k0 : (j == 1 ? n0 : c.m0);
  const double b1 = j == 0 ? k1 : (j == 1 ? n1 : c.m1);
  const double b2 = j == 0 ? k2 : (j == 1 ? n2 : c.m2);
  const double dot = a0 * b0 + a1 * b1 + a2 * b2;
  const double kr = __shfl_sync(gm, dot, base);
  const double mu = __shfl_sync(gm, dot, base + 1);
  const double km = __shfl_sync(gm, dot, base + 2);
  // 1/sqrt(A) (lanes 0-2) and 1/sqrt(3 mu^2 + 1) (lanes 3-5) in one pass
  const double rq = rsqrt(comp < 3 ? A : 3.0 * mu * mu + 1.0);
  const double qA = __shfl_sync(gm, rq, base);
  const double iA = qA * qA;
  const double W = c.W2 * iA;
  const double nj = j == 0 ? n0 : (j == 1 ? n1 : n2);
  const double kj = j == 0 ? k0 : (j == 1 ? k1 : k2);
  const double mj = j == 0 ? c.m0 : (j == 1 ? c.m1 : c.m2);
  double P = 0.0, dPj = 0.0;
  if (c.plasma == PLASMA_GJ) {
    const double F = 3.0 * n2 * mu - c.m2;
    const double ir3 = ir2 * ir;
    P = c.cp * ir3 * (F * c.sig);
    const double t = c.cp * ir3 * c.sig * 3.0 * ir;
    const double m3 = -3.0 * P * ir;
    const double two_mu_nz = 2.0 * mu * n2;
    dPj = m3 * nj + t * (n2 * mj - two_mu_nz * nj) + (j == 2 ? t * mu : 0.0);
  } else if (c.plasma == PLASMA_HOMOG) {
    P = c.pa;
  } else if (c.plasma == PLASMA_LINEAR_Z) {
    P = c.pa * x2;
    dPj = (j == 2) ? c.pa : 0.0;
  } else if (c.plasma == PLASMA_RADIAL) {
    P = c.pa * ir2 * ir;
    dPj = -3.0 * P * ir * nj;
  } else if (c.plasma == PLASMA_TWISTED) {
    const double ir4 = ir2 * ir2;
    P = c.cp * (1.0 - mu * mu) * ir4;
    const double q = c.cp * ir4 * ir;
    dPj = (-2.0 * q * mu) * mj + (q * (6.0 * mu * mu - 4.0)) * nj;
  }
  // the anisotropic scalars both kinds of component use, once
  const bool aniso = (c.disp != DISP_ISO);
  double ib = 0.0, sA = 0.0, U = 0.0, Kp = 0.0, fac = 0.0, opsA = 0.0;
  if (aniso) {
    ib = __shfl_sync(gm, rq, base + 3);
    sA = A * qA;
    U = 3.0 * mu * kr - km + 2.0 * mu * kr * (sA - 1.0);
    Kp = U * ib;
    fac = P * A * Kp * c.iW2;
    opsA = 1.0 + 2.0 * sA;
  }
  // Both kinds of component as out = al k_j + be n_j + ga m_j (+ dP_j one_m):
  // every lane forms both coefficient sets (no divergence), then takes its own.
  // position (c < 3): dH/dk_j = 2 (k_j + (A-1) kr n_j) - 2 fac ib (mu opsA n_j - m_j)
  const double gk_be = 2.0 * Am1 * kr - 2.0 * fac * ib * mu * opsA;
  const double gk_ga = 2.0 * fac * ib;
  // momentum (c >= 3): -dH/dx_j, dH/dx_j = cA n_j + ckr (k_j - kr n_j)
  //   + dP_j one_m + cdA n_j - 2 fac (a1r m_j + a2r k_j + an n_j)
  const double cA = (W * iA + kr * kr) * c.rs * ir2;
  const double ckr = 2.0 * Am1 * kr * ir;
  double gx_al = ckr, gx_be = cA - ckr * kr, gx_ga = 0.0, one_m = 1.0;
  if (aniso) {
    const double Kp2iW2 = Kp * Kp * c.iW2;
    const double ib3 = ib * ib * ib;
    const double a1 = ib * opsA * kr - 3.0 * mu * U * ib3;
    const double a2 = ib * opsA * mu;
    const double a3 = ib * mu * kr * c.rs * ir2 * qA;
    const double a1r = a1 * ir, a2r = a2 * ir;
    const double an = a3 - a1r * mu - a2r * kr;
    one_m = 1.0 - A * Kp2iW2;
    const double cdA = -P * Kp2iW2 * c.rs * ir2;
    const double m2f = -2.0 * fac;
    gx_al += m2f * a2r;
    gx_be += cdA + m2f * an;
    gx_ga = m2f * a1r;
  }
  const bool pos = comp < 3;
  const double al = pos ? 2.0 : -gx_al;
  const double be = pos ? gk_be : -gx_be;
  const double ga = pos ? gk_ga : -gx_ga;
  const double dp = pos ? 0.0 : -dPj * one_m;
  return al * kj + be * nj + ga * mj + dp;
}

// Group state: lane c of a group owns component c; the rest is replicated.
struct GLane {
  RayConst<double> c;
  double yc, f0c;      // own component of the state and of f at the state
  double h, h_resume, lam;
  int na, nr;
  bool last_rej, switching;
  int64_t ray;
  int star;
};

// The group's six values of v, in component order, to every lane of the group.
__device__ __forceinline__ void gather6(unsigned gm, int base, double v, double* out) {
#pragma unroll
  for (int q = 0; q < GROUP; ++q) out[q] = __shfl_sync(gm, v, base + q);
}

// One attempted step of the group's ray; the same decisions as advance().
__device__ int advance_group(const TraceParams& p, GLane& L, int cc, unsigned gm, int base) {
  if (L.na >= p.max_steps || L.na + L.nr >= 4 * p.max_steps) return RAY_MAXSTEPS;
  double yfull[6], t[6];
  gather6(gm, base, L.yc, yfull);
  bool clipped = false;
  double h = L.h;
  {
    double fx[6];
    gather6(gm, base, L.f0c, fx);
    const double v2 = fx[0] * fx[0] + fx[1] * fx[1] + fx[2] * fx[2];
    const double r2 = yfull[0] * yfull[0] + yfull[1] * yfull[1] + yfull[2] * yfull[2];
    if (h * h * v2 > STEP_REACH * STEP_REACH * r2) h = STEP_REACH * sqrt(r2 / v2);
  }
  if (p.lambda_max > 0.0 && L.lam + h >= p.lambda_max) {
    h = p.lambda_max - L.lam;
    clipped = true;
  }
  const double y = L.yc;
  double K1 = L.f0c, K2, K3, K4, K5, K6, K7;
  gather6(gm, base, y + h * (DP::a21 * K1), t);
  K2 = rhs_comp(L.c, t, cc, gm, base);
  gather6(gm, base, y + h * (DP::a31 * K1 + DP::a32 * K2), t);
  K3 = rhs_comp(L.c, t, cc, gm, base);
  gather6(gm, base, y + h * (DP::a41 * K1 + DP::a42 * K2 + DP::a43 * K3), t);
  K4 = rhs_comp(L.c, t, cc, gm, base);
  gather6(gm, base, y + h * (DP::a51 * K1 + DP::a52 * K2 + DP::a53 * K3 + DP::a54 * K4), t);
  K5 = rhs_comp(L.c, t, cc, gm, base);
  gather6(gm, base,
          y + h * (DP::a61 * K1 + DP::a62 * K2 + DP::a63 * K3 + DP::a64 * K4 + DP::a65 * K5),
          t);
  K6 = rhs_comp(L.c, t, cc, gm, base);
  const double yn = y + h * (DP::b1 * K1 + DP::b3 * K3 + DP::b4 * K4 + DP::b5 * K5 + DP::b6 * K6);
  double ynf[6];
  gather6(gm, base, yn, ynf);
  K7 = rhs_comp(L.c, ynf, cc, gm, base);
  const double e = h * (DP::e1 * K1 + DP::e3 * K3 + DP::e4 * K4 + DP::e5 * K5 + DP::e6 * K6 +
                        DP::e7 * K7);
  const double sc = p.atol + p.rtol * fmax(fabs(y), fabs(yn));
  double q6[6];
  gather6(gm, base, (e / sc) * (e / sc), q6);
  const double en = sqrt((q6[0] + q6[1] + q6[2] + q6[3] + q6[4] + q6[5]) / 6.0);
  if (!isfinite(en)) {
    ++L.nr;
    L.h = h * 0.2;
    L.last_rej = true;
    return (L.h < 1e-12) ? RAY_NAN : -1;
  }
  const bool gj = (L.c.plasma == PLASMA_GJ);
  // continuous extension, own component
  const double r2c = yn - y;
  const double r3c = h * K1 - r2c;
  const double r4c = r2c - h * K7 - r3c;
  const double r5c = h * (DP::d1 * K1 + DP::d3 * K3 + DP::d4 * K4 + DP::d5 * K5 + DP::d6 * K6 +
                          DP::d7 * K7);
  if (en <= 1.0 && gj && !L.switching &&
      L.c.sig * gj_side<double>(L.c.m0, L.c.m1, L.c.m2, ynf[0], ynf[1], ynf[2]) < 0.0) {
    // Illinois on the side function along the continuous extension
    const double sgn = L.c.sig;
    auto side_val = [&](double th) {
      double xd[6];
      gather6(gm, base, y + th * (r2c + (1.0 - th) * (r3c + th * (r4c + (1.0 - th) * r5c))), xd);
      const double mx = L.c.m0 * xd[0] + L.c.m1 * xd[1] + L.c.m2 * xd[2];
      const double rr = xd[0] * xd[0] + xd[1] * xd[1] + xd[2] * xd[2];
      return sgn * (3.0 * xd[2] * mx - L.c.m2 * rr);
    };
    double lo = 0.0, hi = 1.0;
    double flo = side_val(0.0), fhi = side_val(1.0);
    if (!(flo >= 0.0)) flo = 0.0;
    if (!(fhi < 0.0)) fhi = -1e-300;
    int last = 0;
    double width = 1.0;
    for (int it = 0; it < 200; ++it) {
      double mid = (lo * fhi - hi * flo) / (fhi - flo);
      if ((it & 1) && hi - lo > 0.5 * width) mid = 0.5 * (lo + hi);
      if (!(mid > lo && mid < hi)) mid = 0.5 * (lo + hi);
      if (mid <= lo || mid >= hi) break;
      if (it & 1) width = hi - lo;
      const double fm = side_val(mid);
      if (fm >= 0.0) {
        lo = mid;
        flo = fm;
        if (last > 0) fhi *= 0.5;
        last = 1;
      } else {
        hi = mid;
        fhi = fm;
        if (last < 0) flo *= 0.5;
        last = -1;
      }
    }
    ++L.nr;
    if (lo < SWITCH_MIN_FRACTION) {
      L.c.sig = -L.c.sig;
      L.f0c = rhs_comp(L.c, yfull, cc, gm, base);
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
    const double rnew2 = ynf[0] * ynf[0] + ynf[1] * ynf[1] + ynf[2] * ynf[2];
    if (rnew2 >= p.r_out * p.r_out) {
      // |x(th)| = r_out on the continuous extension: Illinois, as advance()
      const double ro2 = p.r_out * p.r_out;
      auto inside = [&](double th) {
        double xd[6];
        gather6(gm, base, y + th * (r2c + (1.0 - th) * (r3c + th * (r4c + (1.0 - th) * r5c))),
                xd);
        return ro2 - (xd[0] * xd[0] + xd[1] * xd[1] + xd[2] * xd[2]);
      };
      double flo = ro2 - (yfull[0] * yfull[0] + yfull[1] * yfull[1] + yfull[2] * yfull[2]);
      if (!(flo >= 0.0)) flo = 0.0;
      double fhi = ro2 - rnew2;
      if (!(fhi < 0.0)) fhi = -1e-300;
      double hi;
      const double lo = last_nonneg(inside, flo, fhi, &hi);
      const double th = 0.5 * (lo + hi);
      L.yc = y + th * (r2c + (1.0 - th) * (r3c + th * (r4c + (1.0 - th) * r5c)));
      L.lam += th * h;
      return RAY_ESCAPED;
    }
    L.yc = yn;
    L.f0c = K7;
    L.lam += h;
    if (rnew2 <= p.r_capture * p.r_capture) return RAY_CAPTURED;
    if (clipped) return RAY_LAMBDA_END;
    if (gj && L.c.sig * gj_side<double>(L.c.m0, L.c.m1, L.c.m2, ynf[0], ynf[1], ynf[2]) < 0.0) {
      L.c.sig = -L.c.sig;
      L.f0c = rhs_comp(L.c, ynf, cc, gm, base);
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

// Counts of one warp's finished rays (lane c == 0 of each group holds its own).
struct GroupCounts {
  long long acc = 0, rej = 0, traced = 0, esc = 0;
};

// Six-lane groups of the calling warp continue parked rays: records
// lo + e of recs (PARKREC doubles each: y[6], h, h_resume, sig, flags, na, nr,
// ray, lambda), e = 0, 1, ... claimed one per group with an atomic on *next,
// while lo + e < hi.  ngroups (1 to GROUPS_PER_WARP) groups of the warp take
// part: one group per warp keeps a ray's attempts free of the other groups'
// divergent branches.  Every lane of the warp must call it.
__device__ void tail_groups(const TraceParams& p, const double* recs, unsigned long long lo,
                            unsigned long long hi, unsigned long long* next, int ngroups,
                            GroupCounts& cnt) {
  const int lane = threadIdx.x & 31;
  const int g = lane / GROUP, cc = lane % GROUP;
  const bool in_group = g < ngroups && g < GROUPS_PER_WARP;
  const int base = g * GROUP;
  const unsigned gm = in_group ? (0x3Fu << base) : 0u;
  GLane L;
  bool have = false, done = !in_group;
  int na0 = 0, nr0 = 0;
  for (;;) {
    if (in_group && !have && !done) {
      unsigned long long e = 0;
      if (cc == 0) e = lo + atomicAdd(next, 1ull);
      e = __shfl_sync(gm, e, base);
      if (e >= hi) {
        done = true;
      } else {
        const double* pe = recs + e * PARKREC;
        L.yc = pe[cc];
        L.h = pe[6];
        L.h_resume = pe[7];
        const double sig = pe[8];
        const int fl = (int)pe[9];
        L.last_rej = (fl & 1) != 0;
        L.switching = (fl & 2) != 0;
        L.na = (int)pe[10];
        L.nr = (int)pe[11];
        L.ray = (int64_t)pe[12];
        L.lam = pe[13];
        L.star = find_star_t(p, L.ray);
        const StarDev& s = p.stars[L.star];
        const double om = 1.0 + p.state[6 * p.n + L.ray];
        double sp, cpsi;
        sincos(p.state[7 * p.n + L.ray], &sp, &cpsi);
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
        L.c.sig = sig;
        double yfull[6];
        gather6(gm, base, L.yc, yfull);
        L.f0c = rhs_comp(L.c, yfull, cc, gm, base);
        na0 = L.na;
        nr0 = L.nr;
        have = true;
      }
    }
    if (__ballot_sync(0xffffffffu, in_group && !done) == 0) break;
    if (have) {
      const int st = advance_group(p, L, cc, gm, base);
      if (st >= 0) {
        const StarDev& s = p.stars[L.star];
        const int64_t n = p.n;
        p.state[cc * n + L.ray] = (cc < 3) ? L.yc * s.R_km : L.yc * s.ma_eV;
        __syncwarp(gm);                 // the group's state writes before its status
        if (cc == 0) {
          status_after_state(p, L.ray, st);
          if (p.nacc) p.nacc[L.ray] = L.na;
          if (p.nrej) p.nrej[L.ray] = L.nr;
          if (p.ts) atomicMax(p.ts + 1 + L.star, global_ns());
          cnt.acc += L.na - na0;
          cnt.rej += L.nr - nr0;
          cnt.traced += 1;
          cnt.esc += (st == RAY_ESCAPED);
        }
        have = false;
      }
    }
  }
}

// Express SMs for K records: XRAYS_PER_SM per SM, at most an eighth of the
// device's SM identifiers.
__device__ __forceinline__ unsigned long long express_sms(unsigned long long K) {
  int nsm = 1;
  asm("mov.u32 %0, %%nsmid;" : "=r"(nsm));
  unsigned long long xs = (K + XRAYS_PER_SM - 1) / XRAYS_PER_SM;
  const unsigned long long cap = (unsigned long long)(nsm / 8 > 0 ? nsm / 8 : 1);
  return xs < cap ? xs : cap;
}

// The express records' split: the first S (two per express SM) are continued
// one group per warp, the rest (S to K) five groups per warp.
__device__ __forceinline__ unsigned long long express_solo(unsigned long long K) {
  const unsigned long long S = 2 * express_sms(K);
  return S < K ? S : K;
}

}  // namespace
}  // namespace rtk
