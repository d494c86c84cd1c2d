// Algorithmic operation counts of the integrator, for the roofline report.
// The analytic right-hand side (rt_device.cuh) is instantiated on the host
// with a counting scalar: every +, -, * counts one flop (a fused multiply-add
// therefore counts two), a division, square root, reciprocal or reciprocal
// square root counts one flop and is also tallied separately.  The
// Dormand-Prince stage combinations are counted from the tableau's sparsity.
#include <stdint.h>

#include "rt.h"

namespace {

struct Tally {
  double flops = 0, special = 0;
};
thread_local Tally g_t;

struct Cnt {
  double v;
  Cnt() : v(0) {}
  Cnt(double x) : v(x) {}  // NOLINT: constants are free
};
inline Cnt operator+(Cnt a, Cnt b) { g_t.flops += 1; return Cnt(a.v + b.v); }
inline Cnt operator-(Cnt a, Cnt b) { g_t.flops += 1; return Cnt(a.v - b.v); }
inline Cnt operator*(Cnt a, Cnt b) { g_t.flops += 1; return Cnt(a.v * b.v); }
inline Cnt operator-(Cnt a) { return Cnt(-a.v); }   // sign flips are free
inline Cnt& operator+=(Cnt& a, Cnt b) { a = a + b; return a; }
inline bool operator<(Cnt a, Cnt b) { return a.v < b.v; }
// found by argument-dependent lookup from the templates of rt_device.cuh
inline Cnt rt_rsqrt(Cnt v) { g_t.flops += 1; g_t.special += 1; return Cnt(1.0 / __builtin_sqrt(v.v)); }
inline Cnt rt_sqrt(Cnt v) { g_t.flops += 1; g_t.special += 1; return Cnt(__builtin_sqrt(v.v)); }
inline Cnt rt_rcp(Cnt v) { g_t.flops += 1; g_t.special += 1; return Cnt(1.0 / v.v); }

// The same right-hand side in double-float arithmetic (rt_df.cuh), counted in
// the FP32 operations its kernels execute: a double-float sum 11 (TwoSum 6,
// the low parts 2, Fast2Sum 3), a product 10 (1 multiply, 3 fused
// multiply-adds, Fast2Sum 3), a reciprocal square root 24 (the FP32 estimate,
// the residual's double-float product and the series correction).
constexpr double DF_ADD = 11, DF_MUL = 10, DF_RSQRT = 24, DF_MULF = 8, DF_ADDF = 10;
struct CntD {
  double v;
  CntD() : v(0) {}
  CntD(double x) : v(x) {}  // NOLINT: constants are free
};
inline CntD operator+(CntD a, CntD b) { g_t.flops += DF_ADD; return CntD(a.v + b.v); }
inline CntD operator-(CntD a, CntD b) { g_t.flops += DF_ADD; return CntD(a.v - b.v); }
inline CntD operator*(CntD a, CntD b) { g_t.flops += DF_MUL; return CntD(a.v * b.v); }
inline CntD operator-(CntD a) { return CntD(-a.v); }
inline CntD& operator+=(CntD& a, CntD b) { a = a + b; return a; }
inline bool operator<(CntD a, CntD b) { return a.v < b.v; }
inline CntD rt_rsqrt(CntD v) {
  g_t.flops += DF_RSQRT;
  g_t.special += 1;
  return CntD(1.0 / __builtin_sqrt(v.v));
}

}  // namespace

// the right-hand side template is __host__ __device__; its host instantiation
// here only ever calls the host overloads above
#pragma nv_diag_suppress 20011
#pragma nv_diag_suppress 20014
#pragma nv_diag_suppress 177
#include "rt_device.cuh"

extern "C" rt_status rt_flops_per_step(int32_t dispersion, int32_t plasma, double* out4) {
  if (!out4) return RT_EINVAL;
  if (dispersion < 0 || dispersion > 1 || plasma < 0 || plasma > 4) return RT_EINVAL;
  rtk::RayConst<Cnt> c;
  c.rs = 0.4; c.cp = 4000.0; c.pa = 0.1; c.W2 = 1.0; c.iW2 = 1.0;
  c.m0 = 0.3; c.m1 = 0.1; c.m2 = 0.9; c.sig = 1.0; c.disp = dispersion; c.plasma = plasma;
  g_t = Tally();
  Cnt d[6];
  rtk::ham_rhs<Cnt>(c, Cnt(20.0), Cnt(3.0), Cnt(-5.0), Cnt(0.3), Cnt(-0.4), Cnt(0.8), d[0], d[1],
                    d[2], d[3], d[4], d[5]);
  const double rhs = g_t.flops, rhs_special = g_t.special;
  // Stage inputs y + h * sum_j a_sj k_j for stages 2..6 with 1..5 nonzero
  // coefficients: (2 nnz + 1) flops per component; the 5th-order update uses
  // b_1, b_3..b_6 (nnz = 5); the error estimate h * sum e_j k_j uses 6 terms
  // (2 * 6); the scaled RMS norm per component: max, 2 flops for the scale,
  // 1 division, 2 for the square and sum, plus 1 division and 1 sqrt; the
  // controller: a power (counted as one special operation) and 4 flops.
  const int nnz_stage[5] = {1, 2, 3, 4, 5};
  double comb = 0;
  for (int s = 0; s < 5; ++s) comb += 6.0 * (2 * nnz_stage[s] + 1);
  comb += 6.0 * (2 * 5 + 1);
  comb += 6.0 * (2 * 6);
  comb += 6.0 * (2 + 1 + 2) + 2;
  comb += 5;
  out4[0] = rhs;                        // flops of one right-hand side evaluation
  out4[1] = 6.0 * rhs + comb;           // flops of one step attempt (FSAL: 6 evaluations)
  out4[2] = 2.0 * rhs + 60.0;           // flops of the initial step heuristic (2 evaluations)
  out4[3] = 6.0 * rhs_special + 6 + 3;  // divisions / square roots / powers per attempt
  return RT_OK;
}

extern "C" rt_status rt_flops_per_step_df(int32_t dispersion, int32_t plasma, double* out2) {
  if (!out2) return RT_EINVAL;
  if (dispersion < 0 || dispersion > 1 || plasma < 0 || plasma > 5) return RT_EINVAL;
  rtk::RayConst<CntD> c;
  c.rs = 0.4; c.cp = 4000.0; c.pa = 0.1; c.W2 = 1.0; c.iW2 = 1.0;
  c.m0 = 0.3; c.m1 = 0.1; c.m2 = 0.9; c.sig = 1.0; c.disp = dispersion; c.plasma = plasma;
  g_t = Tally();
  CntD d[6];
  rtk::ham_rhs<CntD>(c, CntD(20.0), CntD(3.0), CntD(-5.0), CntD(0.3), CntD(-0.4), CntD(0.8), d[0],
                     d[1], d[2], d[3], d[4], d[5]);
  const double rhs = g_t.flops;
  // stage inputs y + h (sum_j a_sj k_j): nnz products and nnz - 1 sums of
  // double-floats, one product by h and one sum, per component; the update
  // with nnz = 5; the error estimate h sum e_j k_j (6 products, 5 sums, one
  // product) and its FP32 scaled norm (6 per component, then 2); the step
  // reach (10) and the controller (6), FP32; the null-cone side at the new
  // point (F = 3 z (m.x) - m_z |x|^2: 8 products, 5 sums)
  const int nnz_stage[6] = {1, 2, 3, 4, 5, 5};
  double comb = 0;
  for (int s = 0; s < 6; ++s)
    comb += 6.0 * (nnz_stage[s] * DF_MUL + (nnz_stage[s] - 1) * DF_ADD + DF_MUL + DF_ADD);
  comb += 6.0 * (7 * DF_MUL + 5 * DF_ADD + 6) + 2;
  comb += 10 + 6;
  if (plasma == 0) comb += 8 * DF_MUL + 5 * DF_ADD;
  out2[0] = rhs;                       // FP32 flops of one right-hand side evaluation
  out2[1] = 6.0 * rhs + comb;          // FP32 flops of one step attempt
  return RT_OK;
}
