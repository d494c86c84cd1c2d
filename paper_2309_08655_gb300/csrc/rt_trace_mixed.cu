// Mixed-precision forward tracing: the Dormand-Prince stages (the analytic
// right-hand side and the stage combinations) run in FP32 with FP32
// accumulation of the increments; the ray state is kept in FP64 and receives
// each accepted increment in FP64.  FP32 rounding puts a noise floor under the
// embedded error estimate; when that floor reaches a quarter of the tolerance
// the estimate no longer steers the step size, and the ray is promoted: it is
// handed, from its current state, to the FP64 kernel (resume pass) for the
// rest of its path.  This happens where the controller demands steps too
// short for FP32 -- typically near the stellar surface or close to a turning
// point at the resonance.
#include <cuda_runtime.h>
#include <stdint.h>

#include "rt_device.cuh"
#include "rt_internal.h"

namespace rtk {

namespace {

constexpr unsigned FULL = 0xffffffffu;
constexpr float EPS32 = 5.9604645e-8f;     // unit roundoff 2^-24
constexpr float NOISE_C = 4.0f;             // rounding amplification allowed in a stage
constexpr float NOISE_LIMIT = 0.25f;

__device__ __forceinline__ void rhs32(const RayConst<float>& c, const float* y, float* f) {
  ham_rhs<float>(c, y[0], y[1], y[2], y[3], y[4], y[5], f[0], f[1], f[2], f[3], f[4], f[5]);
}

__device__ __forceinline__ float step_factor32(float err, bool accepted, bool last_rej) {
  float fac = (err > 0.0f) ? 0.9f * exp2f(-0.2f * log2f(err)) : 5.0f;
  fac = fminf(5.0f, fmaxf(0.2f, fac));
  if (!accepted || last_rej) fac = fminf(fac, 1.0f);
  return fac;
}

__device__ float initial_step32(const RayConst<float>& c, const float* y0, const float* f0,
                                float rtol, float atol, float hmax) {
  float dnf = 0.0f, dny = 0.0f;
#pragma unroll
  for (int i = 0; i < 6; ++i) {
    const float sk = atol + rtol * fabsf(y0[i]);
    dnf += (f0[i] / sk) * (f0[i] / sk);
    dny += (y0[i] / sk) * (y0[i] / sk);
  }
  float h = (dnf <= 1e-10f || dny <= 1e-10f) ? 1e-6f : sqrtf(dny / dnf) * 0.01f;
  h = fminf(h, hmax);
  float y1[6], f1[6];
#pragma unroll
  for (int i = 0; i < 6; ++i) y1[i] = y0[i] + h * f0[i];
  rhs32(c, y1, f1);
  float der2 = 0.0f;
#pragma unroll
  for (int i = 0; i < 6; ++i) {
    const float sk = atol + rtol * fabsf(y0[i]);
    der2 += ((f1[i] - f0[i]) / sk) * ((f1[i] - f0[i]) / sk);
  }
  der2 = sqrtf(der2) / h;
  const float der12 = fmaxf(fabsf(der2), sqrtf(dnf));
  const float h1 = (der12 <= 1e-15f) ? fmaxf(1e-6f, h * 1e-3f) : exp2f(0.2f * log2f(0.01f / der12));
  return fminf(fminf(100.0f * h, h1), hmax);
}

struct LaneM {
  RayConst<float> c;
  double y[6];
  float f0[6];
  float h;
  int na, nr;
  bool last_rej;
  bool switching;      // the current attempt ends just past a null-cone crossing
  float h_resume;
  double R_km, ma_eV;
};

// Side of the Goldreich-Julian null cone at an FP64 position (see rt_trace.cu
// for the switching scheme, which this kernel follows in FP32).
__device__ __forceinline__ float side_m(const RayConst<float>& c, double x0, double x1,
                                        double x2) {
  return (float)gj_side<double>((double)c.m0, (double)c.m1, (double)c.m2, x0, x1, x2);
}
constexpr float SWITCH_MIN_FRACTION_M = 1e-6f;
constexpr float SWITCH_OVERSHOOT_M = 1e-6f;

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
#pragma unroll
  for (int c = 0; c < 3; ++c) {
    L.y[c] = p.state[c * n + i] * iR;
    L.y[3 + c] = p.state[(3 + c) * n + i] * im;
  }
  const double om = 1.0 + p.state[6 * n + i];
  double sp, cpsi;
  sincos(p.state[7 * n + i], &sp, &cpsi);
  L.c.rs = (float)s.rs_prop;
  L.c.cp = (float)s.cp;
  L.c.pa = (float)s.plasma_a;
  L.c.W2 = (float)(om * om);
  L.c.iW2 = (float)(1.0 / (om * om));
  L.c.m0 = (float)(s.sin_tm * cpsi);
  L.c.m1 = (float)(s.sin_tm * sp);
  L.c.m2 = (float)s.cos_tm;
  L.c.disp = s.dispersion;
  L.c.plasma = s.plasma;
  L.c.sig = side_m(L.c, L.y[0], L.y[1], L.y[2]);
  L.switching = false;
  L.h_resume = 0.0f;
  float yf[6];
#pragma unroll
  for (int c = 0; c < 6; ++c) yf[c] = (float)L.y[c];
  rhs32(L.c, yf, L.f0);
  L.h = initial_step32(L.c, yf, L.f0, (float)p.rtol, (float)p.atol, 1e30f);
  L.na = p.nacc ? 0 : 0;
  L.nr = 0;
  L.last_rej = false;
}

__device__ void store_lane_m(const TraceParams& p, int64_t i, const LaneM& L, int st) {
  const int64_t n = p.n;
#pragma unroll
  for (int c = 0; c < 3; ++c) {
    p.state[c * n + i] = L.y[c] * L.R_km;
    p.state[(3 + c) * n + i] = L.y[3 + c] * L.ma_eV;
  }
  p.status[i] = (uint8_t)st;
  if (p.nacc) p.nacc[i] = L.na;
  if (p.nrej) p.nrej[i] = L.nr;
}

// One attempted FP32 step.  Returns -1 to continue, RAY_PROMOTED to hand the
// ray to the FP64 pass, else the final status.
__device__ int advance_m(const TraceParams& p, LaneM& L) {
  if (L.na >= p.max_steps || L.na + L.nr >= 4 * p.max_steps) return RAY_MAXSTEPS;
  const float h = L.h;
  const float rtol = (float)p.rtol, atol = (float)p.atol;
  float yf[6];
#pragma unroll
  for (int i = 0; i < 6; ++i) yf[i] = (float)L.y[i];
  const float* k1 = L.f0;
  float t[6], k2[6], k3[6], k4[6], k5[6], k6[6], k7[6], d5[6];
#pragma unroll
  for (int i = 0; i < 6; ++i) t[i] = yf[i] + h * ((float)DP::a21 * k1[i]);
  rhs32(L.c, t, k2);
#pragma unroll
  for (int i = 0; i < 6; ++i) t[i] = yf[i] + h * ((float)DP::a31 * k1[i] + (float)DP::a32 * k2[i]);
  rhs32(L.c, t, k3);
#pragma unroll
  for (int i = 0; i < 6; ++i)
    t[i] = yf[i] + h * ((float)DP::a41 * k1[i] + (float)DP::a42 * k2[i] + (float)DP::a43 * k3[i]);
  rhs32(L.c, t, k4);
#pragma unroll
  for (int i = 0; i < 6; ++i)
    t[i] = yf[i] + h * ((float)DP::a51 * k1[i] + (float)DP::a52 * k2[i] +
                        (float)DP::a53 * k3[i] + (float)DP::a54 * k4[i]);
  rhs32(L.c, t, k5);
#pragma unroll
  for (int i = 0; i < 6; ++i)
    t[i] = yf[i] + h * ((float)DP::a61 * k1[i] + (float)DP::a62 * k2[i] +
                        (float)DP::a63 * k3[i] + (float)DP::a64 * k4[i] +
                        (float)DP::a65 * k5[i]);
  rhs32(L.c, t, k6);
#pragma unroll
  for (int i = 0; i < 6; ++i) {
    d5[i] = h * ((float)DP::b1 * k1[i] + (float)DP::b3 * k3[i] + (float)DP::b4 * k4[i] +
                 (float)DP::b5 * k5[i] + (float)DP::b6 * k6[i]);
    t[i] = yf[i] + d5[i];
  }
  rhs32(L.c, t, k7);
  float s = 0.0f, sn = 0.0f;
  double yn[6];
#pragma unroll
  for (int i = 0; i < 6; ++i) {
    yn[i] = L.y[i] + (double)d5[i];
    const float a1 = (float)DP::e1 * k1[i], a3 = (float)DP::e3 * k3[i];
    const float a4 = (float)DP::e4 * k4[i], a5 = (float)DP::e5 * k5[i];
    const float a6 = (float)DP::e6 * k6[i], a7 = (float)DP::e7 * k7[i];
    const float e = h * (a1 + a3 + a4 + a5 + a6 + a7);
    const float nz = NOISE_C * EPS32 * fabsf(h) *
                     (fabsf(a1) + fabsf(a3) + fabsf(a4) + fabsf(a5) + fabsf(a6) + fabsf(a7));
    const float sc = atol + rtol * fmaxf(fabsf(yf[i]), fabsf((float)yn[i]));
    s += (e / sc) * (e / sc);
    sn += (nz / sc) * (nz / sc);
  }
  const float en = sqrtf(s / 6.0f);
  const float noise = sqrtf(sn / 6.0f);
  if (!isfinite(en)) {
    ++L.nr;
    L.h = h * 0.2f;
    L.last_rej = true;
    return (L.h < 1e-12f) ? RAY_NAN : -1;
  }
  // A rejection whose error estimate sits on the FP32 noise floor cannot be
  // trusted: the ray continues in FP64.  An accepted step on the noise floor
  // is kept, but may not grow the step.
  const bool noisy = noise > NOISE_LIMIT;
  if (noisy && !(en <= 1.0f)) return RAY_PROMOTED;
  const bool gj = (L.c.plasma == PLASMA_GJ);
  if (en <= 1.0f && gj && !L.switching && L.c.sig * side_m(L.c, yn[0], yn[1], yn[2]) < 0.0f) {
    // the step crossed the null cone: locate on the continuous extension and
    // redo the step to end just past the crossing
    float r3[3], r4[3], r5[3];
#pragma unroll
    for (int i = 0; i < 3; ++i) {
      r3[i] = h * k1[i] - d5[i];
      r4[i] = d5[i] - h * k7[i] - r3[i];
      r5[i] = h * ((float)DP::d1 * k1[i] + (float)DP::d3 * k3[i] + (float)DP::d4 * k4[i] +
                   (float)DP::d5 * k5[i] + (float)DP::d6 * k6[i] + (float)DP::d7 * k7[i]);
    }
    float lo = 0.0f, hi = 1.0f;
    for (int it = 0; it < 40; ++it) {
      const float mid = 0.5f * (lo + hi);
      if (mid <= lo || mid >= hi) break;
      double xd[3];
#pragma unroll
      for (int i = 0; i < 3; ++i)
        xd[i] = L.y[i] + (double)(mid * (d5[i] + (1.0f - mid) * (r3[i] + mid * (r4[i] +
                                                         (1.0f - mid) * r5[i]))));
      if (L.c.sig * side_m(L.c, xd[0], xd[1], xd[2]) >= 0.0f) lo = mid; else hi = mid;
    }
    ++L.nr;
    if (lo < SWITCH_MIN_FRACTION_M) {
      L.c.sig = -L.c.sig;
      rhs32(L.c, yf, L.f0);
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
    const double rnew = sqrt(yn[0] * yn[0] + yn[1] * yn[1] + yn[2] * yn[2]);
    if (rnew >= p.r_out) {
      // locate |x(th)| = r_out on the continuous extension (FP32 increments
      // added to the FP64 state)
      float r3[6], r4[6], r5[6];
#pragma unroll
      for (int i = 0; i < 6; ++i) {
        r3[i] = h * k1[i] - d5[i];
        r4[i] = d5[i] - h * k7[i] - r3[i];
        r5[i] = h * ((float)DP::d1 * k1[i] + (float)DP::d3 * k3[i] + (float)DP::d4 * k4[i] +
                     (float)DP::d5 * k5[i] + (float)DP::d6 * k6[i] + (float)DP::d7 * k7[i]);
      }
      double lo = 0.0, hi = 1.0;
      for (int it = 0; it < 60; ++it) {
        const double mid = 0.5 * (lo + hi);
        if (mid <= lo || mid >= hi) break;
        const float m = (float)mid;
        double xd[3];
#pragma unroll
        for (int i = 0; i < 3; ++i)
          xd[i] = L.y[i] +
                  (double)(m * (d5[i] + (1.0f - m) * (r3[i] + m * (r4[i] + (1.0f - m) * r5[i]))));
        const double rd = sqrt(xd[0] * xd[0] + xd[1] * xd[1] + xd[2] * xd[2]);
        if (rd < p.r_out) lo = mid; else hi = mid;
      }
      const float th = (float)(0.5 * (lo + hi));
#pragma unroll
      for (int i = 0; i < 6; ++i)
        L.y[i] += (double)(th * (d5[i] + (1.0f - th) * (r3[i] + th * (r4[i] + (1.0f - th) * r5[i]))));
      return RAY_ESCAPED;
    }
#pragma unroll
    for (int i = 0; i < 6; ++i) {
      L.y[i] = yn[i];
      L.f0[i] = k7[i];
    }
    if (rnew <= p.r_capture) return RAY_CAPTURED;
    if (gj && L.c.sig * side_m(L.c, L.y[0], L.y[1], L.y[2]) < 0.0f) {
      L.c.sig = -L.c.sig;             // past the cone: continue on the other side
      float yc[6];
#pragma unroll
      for (int i = 0; i < 6; ++i) yc[i] = (float)L.y[i];
      rhs32(L.c, yc, L.f0);
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
  ++L.nr;
  L.h = h * step_factor32(en, false, L.last_rej);
  L.last_rej = true;
  return (L.h < 1e-12f) ? RAY_STIFF : -1;
}

__global__ void __launch_bounds__(256) trace_mixed_kernel(TraceParams p) {
  const int lane = threadIdx.x & 31;
  int64_t ray = -1;
  LaneM L;
  long long acc = 0, rej = 0, traced = 0, esc = 0, promoted = 0;
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
        } else if (p.status[idx] != RAY_READY) {
          ray = -1;
        } else {
          ray = idx;
          load_lane_m(p, idx, L);
        }
      }
    }
    if (__ballot_sync(FULL, ray != -2) == 0) break;
    if (ray >= 0) {
      const int st = advance_m(p, L);
      if (st >= 0) {
        store_lane_m(p, ray, L, st);
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
      atomicAdd((unsigned long long*)&p.counters[0], (unsigned long long)acc);
      atomicAdd((unsigned long long*)&p.counters[1], (unsigned long long)rej);
      atomicAdd((unsigned long long*)&p.counters[2], (unsigned long long)traced);
      atomicAdd((unsigned long long*)&p.counters[3], (unsigned long long)esc);
      atomicAdd((unsigned long long*)&p.counters[4], (unsigned long long)promoted);
    }
  }
}

}  // namespace

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
