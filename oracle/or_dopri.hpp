// Oracle (test infrastructure only; never linked into the product path).
//
// Dormand-Prince 5(4) explicit Runge-Kutta pair (J. R. Dormand and P. J.
// Prince, J. Comput. Appl. Math. 6 (1980) 19), its published 4th-order
// continuous extension (Hairer, Norsett and Wanner, "Solving Ordinary
// Differential Equations I", Sec. II.6), the RMS error norm and the
// elementary step-size controller of Sec. II.4 of the same book, and the
// initial-step heuristic of Sec. II.4.  The paper asks for "high-precision
// ODE solvers" (Sec. 2.4 and Sec. 5) without naming one; this is the standard
// adaptive pair, written out plainly.
#pragma once
#include <cmath>

namespace orc {

struct DP5 {
  // nodes
  static constexpr double c[7] = {0.0, 1.0 / 5.0, 3.0 / 10.0, 4.0 / 5.0, 8.0 / 9.0, 1.0, 1.0};
  // Butcher matrix a[i][j], j < i
  static constexpr double a[7][6] = {
      {0, 0, 0, 0, 0, 0},
      {1.0 / 5.0, 0, 0, 0, 0, 0},
      {3.0 / 40.0, 9.0 / 40.0, 0, 0, 0, 0},
      {44.0 / 45.0, -56.0 / 15.0, 32.0 / 9.0, 0, 0, 0},
      {19372.0 / 6561.0, -25360.0 / 2187.0, 64448.0 / 6561.0, -212.0 / 729.0, 0, 0},
      {9017.0 / 3168.0, -355.0 / 33.0, 46732.0 / 5247.0, 49.0 / 176.0, -5103.0 / 18656.0, 0},
      {35.0 / 384.0, 0.0, 500.0 / 1113.0, 125.0 / 192.0, -2187.0 / 6784.0, 11.0 / 84.0}};
  // 5th-order weights (equal to the last row: first-same-as-last)
  static constexpr double b[7] = {35.0 / 384.0, 0.0, 500.0 / 1113.0, 125.0 / 192.0,
                                  -2187.0 / 6784.0, 11.0 / 84.0, 0.0};
  // 4th-order embedded weights
  static constexpr double bh[7] = {5179.0 / 57600.0, 0.0, 7571.0 / 16695.0, 393.0 / 640.0,
                                   -92097.0 / 339200.0, 187.0 / 2100.0, 1.0 / 40.0};
  // error weights e = b - bh as exact rationals (summing e_j K_j directly keeps
  // the error estimate free of the cancellation of acc5 - acc4)
  static constexpr double e[7] = {71.0 / 57600.0, 0.0, -71.0 / 16695.0, 71.0 / 1920.0,
                                  -17253.0 / 339200.0, 22.0 / 525.0, -1.0 / 40.0};
  // continuous extension coefficients (Shampine's d_i)
  static constexpr double d[7] = {-12715105075.0 / 11282082432.0, 0.0,
                                  87487479700.0 / 32700410799.0, -10690763975.0 / 1880347072.0,
                                  701980252875.0 / 199316789632.0, -1453857185.0 / 822651844.0,
                                  69997945.0 / 29380423.0};
};

// One trial step from (y, f0 = f(y)) with step h, for a state of N
// components (N = 6: x, k; N = 8: x, k, t, k_t).  Writes the 5th-order
// solution, the local error estimate (5th minus 4th order) and all stages
// (stage 7 is f(y_new), reused as the next step's first stage).
template <class F, int N>
inline void dp5_step(F& f, const double* y, const double* f0, double h, double* ynew,
                     double* err, double (*K)[N]) {
  for (int i = 0; i < N; ++i) K[0][i] = f0[i];
  double ys[N];
  for (int s = 1; s < 7; ++s) {
    for (int i = 0; i < N; ++i) {
      double acc = 0.0;
      for (int j = 0; j < s; ++j) acc += DP5::a[s][j] * K[j][i];
      ys[i] = y[i] + h * acc;
    }
    f(ys, K[s]);
  }
  // stage 7 was evaluated at the 5th-order solution (row 7 of a equals b)
  for (int i = 0; i < N; ++i) {
    double acc5 = 0.0, acce = 0.0;
    for (int j = 0; j < 7; ++j) {
      acc5 += DP5::b[j] * K[j][i];
      acce += DP5::e[j] * K[j][i];
    }
    ynew[i] = y[i] + h * acc5;
    err[i] = h * acce;
  }
}

// Dense output on [lambda_n, lambda_n + h] at fraction th in [0, 1].
template <int N>
inline void dp5_dense(const double* y, const double* ynew, const double (*K)[N], double h,
                      double th, double* out) {
  for (int i = 0; i < N; ++i) {
    double r1 = y[i];
    double r2 = ynew[i] - y[i];
    double r3 = h * K[0][i] - r2;
    double r4 = r2 - h * K[6][i] - r3;
    double dk = 0.0;
    for (int j = 0; j < 7; ++j) dk += DP5::d[j] * K[j][i];
    double r5 = h * dk;
    out[i] = r1 + th * (r2 + (1.0 - th) * (r3 + th * (r4 + (1.0 - th) * r5)));
  }
}

// RMS norm of the error, scaled by atol + rtol * max(|y|, |ynew|), over the
// six phase-space components x, k: with the eight-component state of a
// rotating magnetosphere the clock t and k_t follow the step sequence that
// x and k choose.
inline double dp5_error_norm(const double y[6], const double ynew[6], const double err[6],
                             double rtol, double atol) {
  double s = 0.0;
  for (int i = 0; i < 6; ++i) {
    double sc = atol + rtol * std::fmax(std::fabs(y[i]), std::fabs(ynew[i]));
    s += (err[i] / sc) * (err[i] / sc);
  }
  return std::sqrt(s / 6.0);
}

// Step-size factor of the elementary controller: 0.9 * err^(-1/5), clamped to
// [0.2, 5]; after a rejection the step may not grow.
inline double dp5_step_factor(double err, bool accepted, bool last_rejected) {
  double fac = (err > 0.0) ? 0.9 * std::pow(err, -0.2) : 5.0;
  fac = std::fmin(5.0, std::fmax(0.2, fac));
  if (!accepted || last_rejected) fac = std::fmin(fac, 1.0);
  return fac;
}

// Initial step: the two-evaluation heuristic (order 5) of Hairer et al.,
// with the norms over x, k (as the error norm).
template <int N = 6, class F>
inline double dp5_initial_step(F& f, const double* y0, const double* f0, double rtol,
                               double atol, double hmax) {
  double dnf = 0.0, dny = 0.0;
  for (int i = 0; i < 6; ++i) {
    double sk = atol + rtol * std::fabs(y0[i]);
    dnf += (f0[i] / sk) * (f0[i] / sk);
    dny += (y0[i] / sk) * (y0[i] / sk);
  }
  double h = (dnf <= 1e-10 || dny <= 1e-10) ? 1e-6 : std::sqrt(dny / dnf) * 0.01;
  h = std::fmin(h, hmax);
  double y1[N], f1[N];
  for (int i = 0; i < N; ++i) y1[i] = y0[i] + h * f0[i];
  f(y1, f1);
  double der2 = 0.0;
  for (int i = 0; i < 6; ++i) {
    double sk = atol + rtol * std::fabs(y0[i]);
    der2 += ((f1[i] - f0[i]) / sk) * ((f1[i] - f0[i]) / sk);
  }
  der2 = std::sqrt(der2) / h;
  double der12 = std::fmax(std::fabs(der2), std::sqrt(dnf));
  double h1 = (der12 <= 1e-15) ? std::fmax(1e-6, h * 1e-3) : std::pow(0.01 / der12, 0.2);
  return std::fmin(std::fmin(100.0 * h, h1), hmax);
}

}  // namespace orc
