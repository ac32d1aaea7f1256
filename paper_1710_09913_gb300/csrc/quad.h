// Collapsed Gauss-Jacobi quadrature on the reference simplex (host), for the
// sub-element integration of discontinuous coefficients in the A_T precompute.
//
// Gauss-Jacobi nodes: roots of the Jacobi polynomial P_n^(a,0) on [-1, 1], found by
// Newton's method with deflation of the roots already found, the polynomial and its
// derivative from the three-term recurrence; weights
//   w_k = 2^(a+1) G(n+a+1) G(n+1) / (n! G(n+a+1) (1 - x_k^2) P_n'(x_k)^2)
// (Szego, Orthogonal Polynomials, 15.3).  Mapped to t in [0, 1] with weight (1-t)^a.
// Simplex: x = s(1-t) [(1-r)], y = t [(1-r)], z = r with weights (1-t) [(1-t)(1-r)^2]
// (Duffy collapse); n points per direction integrate total degree 2n - 1 exactly.
#pragma once

#include <cmath>
#include <vector>

namespace dogip {

inline void jacobi_eval(int n, double a, double x, double* p, double* dp) {
  // P_0 = 1, P_1 = ((a+2) x + a) / 2 for b = 0, then the standard recurrence
  double p0 = 1.0, p1 = 0.5 * ((a + 2.0) * x + a);
  if (n == 0) {
    *p = 1.0;
    *dp = 0.0;
    return;
  }
  for (int k = 2; k <= n; ++k) {
    const double c = 2.0 * k + a;
    const double a1 = 2.0 * k * (k + a) * (c - 2.0);
    const double a2 = (c - 1.0) * a * a;
    const double a3 = (c - 2.0) * (c - 1.0) * c;
    const double a4 = 2.0 * (k + a - 1.0) * (k - 1.0) * c;
    const double p2 = ((a2 + a3 * x) * p1 - a4 * p0) / a1;
    p0 = p1;
    p1 = p2;
  }
  *p = p1;
  // derivative: (1-x^2) P_n' = n (a - (2n+a) x) / (2n+a) P_n + 2 (n+a) n / (2n+a) P_{n-1}
  const double c = 2.0 * n + a;
  *dp = (n * (a - c * x) / c * p1 + 2.0 * (n + a) * n / c * p0) / (1.0 - x * x);
}

// n-point rule on [0, 1] for the weight (1-t)^a (a = 0, 1, 2).
inline void gauss_jacobi01(int n, double a, std::vector<double>& t, std::vector<double>& w) {
  std::vector<double> x(n);
  for (int k = 0; k < n; ++k) {
    double r = -std::cos((2.0 * k + 1.0) * M_PI / (2.0 * n));  // Chebyshev guess
    if (k > 0) r = std::max(r, 0.5 * (r + x[k - 1]));
    for (int it = 0; it < 100; ++it) {
      double p, dp;
      jacobi_eval(n, a, r, &p, &dp);
      double s = 0.0;
      for (int j = 0; j < k; ++j) s += 1.0 / (r - x[j]);
      const double dr = p / (dp - s * p);
      r -= dr;
      if (std::fabs(dr) < 1e-16) break;
    }
    x[k] = r;
  }
  const double lg = std::lgamma(n + a + 1.0) + std::lgamma(n + 1.0) - std::lgamma(n + 1.0) -
                    std::lgamma(n + a + 1.0);
  t.resize(n);
  w.resize(n);
  for (int k = 0; k < n; ++k) {
    double p, dp;
    jacobi_eval(n, a, x[k], &p, &dp);
    const double wk = std::pow(2.0, a + 1.0) * std::exp(lg) / ((1.0 - x[k] * x[k]) * dp * dp);
    t[k] = 0.5 * (x[k] + 1.0);
    w[k] = wk / std::pow(2.0, a + 1.0);
  }
}

// Points [nq x d] (reference coordinates) and weights of the collapsed rule.
inline void simplex_rule(int d, int n, std::vector<double>& pts, std::vector<double>& wts) {
  std::vector<double> s, ws, t, wt, r, wr;
  gauss_jacobi01(n, 0.0, s, ws);
  gauss_jacobi01(n, 1.0, t, wt);
  pts.clear();
  wts.clear();
  if (d == 2) {
    for (int i = 0; i < n; ++i)
      for (int j = 0; j < n; ++j) {
        pts.push_back(s[i] * (1.0 - t[j]));
        pts.push_back(t[j]);
        wts.push_back(ws[i] * wt[j]);
      }
  } else {
    gauss_jacobi01(n, 2.0, r, wr);
    for (int i = 0; i < n; ++i)
      for (int j = 0; j < n; ++j)
        for (int k = 0; k < n; ++k) {
          pts.push_back(s[i] * (1.0 - t[j]) * (1.0 - r[k]));
          pts.push_back(t[j] * (1.0 - r[k]));
          pts.push_back(r[k]);
          wts.push_back(ws[i] * wt[j] * wr[k]);
        }
  }
}

}  // namespace dogip
