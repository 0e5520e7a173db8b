// Laplace quadrature for the MP2 energy denominator (Eq. SCHLT of
// arXiv:1611.06797; the paper uses a minimax grid, Sec. II C and Sec. III A,
// without printing its nodes):
//     1/x ~= sum_k w_k exp(-x tau_k),   x in [xmin, xmax] = [2 gap, 2 width].
// The relative error eta(x) = 1 - x sum_k w_k exp(-x tau_k) is driven towards the
// minimax solution by Lawson reweighting of a least-squares fit; each weighted
// fit is a Levenberg-Marquardt solve in (w_k, ln tau_k) with the analytic
// Jacobian.  The problem is scale invariant, so it is solved on y = x / xmin in
// [1, R] and rescaled (tau = tau'/xmin, w = w'/xmin).  Two starts are refined and
// the better kept: a trapezoid rule in t = ln(tau) with balanced truncation, and
// log-spaced nodes with least-squares weights.
#include <algorithm>
#include <cmath>
#ifndef M_PI
#define M_PI 3.14159265358979323846
#endif
#include <vector>

#include "../../include/ltmp2.h"

namespace {

struct Fit {
  std::vector<double> w, a;  // weights and log-nodes (tau = exp(a))
};

// max |eta| on m log-spaced points of [1, R]
double max_rel_error(const Fit &f, double R, int m) {
  double worst = 0.0;
  const int n = (int)f.w.size();
  for (int s = 0; s < m; ++s) {
    const double y = std::exp(std::log(R) * s / (m - 1));
    double sum = 0.0;
    for (int k = 0; k < n; ++k) sum += f.w[k] * std::exp(-y * std::exp(f.a[k]));
    worst = std::max(worst, std::fabs(1.0 - y * sum));
  }
  return worst;
}

// Solve (A + lambda diag(A)) x = b for symmetric positive A (Cholesky).  false if singular.
bool solve_spd(std::vector<double> A, std::vector<double> b, int n, std::vector<double> &x) {
  for (int j = 0; j < n; ++j) {
    double d = A[j * n + j];
    for (int k = 0; k < j; ++k) d -= A[j * n + k] * A[j * n + k];
    if (!(d > 0.0)) return false;
    d = std::sqrt(d);
    A[j * n + j] = d;
    for (int i = j + 1; i < n; ++i) {
      double s = A[i * n + j];
      for (int k = 0; k < j; ++k) s -= A[i * n + k] * A[j * n + k];
      A[i * n + j] = s / d;
    }
  }
  x.assign(n, 0.0);
  for (int i = 0; i < n; ++i) {
    double s = b[i];
    for (int k = 0; k < i; ++k) s -= A[i * n + k] * x[k];
    x[i] = s / A[i * n + i];
  }
  for (int i = n - 1; i >= 0; --i) {
    double s = x[i];
    for (int k = i + 1; k < n; ++k) s -= A[k * n + i] * x[k];
    x[i] = s / A[i * n + i];
  }
  return true;
}

// weighted residuals r_s = sqrt(rho_s) eta(y_s)
double residuals(const Fit &f, const std::vector<double> &y, const std::vector<double> &sr,
                 std::vector<double> &r) {
  const int n = (int)f.w.size(), S = (int)y.size();
  double ss = 0.0;
  r.resize(S);
  for (int s = 0; s < S; ++s) {
    double sum = 0.0;
    for (int k = 0; k < n; ++k) sum += f.w[k] * std::exp(-y[s] * std::exp(f.a[k]));
    r[s] = sr[s] * (1.0 - y[s] * sum);
    ss += r[s] * r[s];
  }
  return ss;
}

// Levenberg-Marquardt on the weighted least-squares problem, parameters (w, a).
void lm_fit(Fit &f, const std::vector<double> &y, const std::vector<double> &sr, int iters) {
  const int n = (int)f.w.size(), S = (int)y.size(), P = 2 * n;
  std::vector<double> r, rn, J((size_t)S * P), JtJ(P * P), Jtr(P), step;
  double lambda = 1e-3;
  double cost = residuals(f, y, sr, r);
  for (int it = 0; it < iters; ++it) {
    for (int s = 0; s < S; ++s) {
      for (int k = 0; k < n; ++k) {
        const double tau = std::exp(f.a[k]);
        const double e = std::exp(-y[s] * tau);
        J[(size_t)s * P + k] = -sr[s] * y[s] * e;                               // d r / d w_k
        J[(size_t)s * P + n + k] = sr[s] * y[s] * f.w[k] * y[s] * tau * e;      // d r / d a_k
      }
    }
    std::fill(JtJ.begin(), JtJ.end(), 0.0);
    std::fill(Jtr.begin(), Jtr.end(), 0.0);
    for (int s = 0; s < S; ++s) {
      const double *row = &J[(size_t)s * P];
      for (int i = 0; i < P; ++i) {
        Jtr[i] += row[i] * r[s];
        for (int j = 0; j <= i; ++j) JtJ[i * P + j] += row[i] * row[j];
      }
    }
    for (int i = 0; i < P; ++i)
      for (int j = 0; j < i; ++j) JtJ[j * P + i] = JtJ[i * P + j];
    bool improved = false;
    for (int tries = 0; tries < 12; ++tries) {
      std::vector<double> A = JtJ, b(P);
      for (int i = 0; i < P; ++i) {
        A[i * P + i] += lambda * (JtJ[i * P + i] + 1e-300);
        b[i] = -Jtr[i];
      }
      if (!solve_spd(A, b, P, step)) { lambda *= 10.0; continue; }
      Fit g = f;
      for (int k = 0; k < n; ++k) {
        g.w[k] += step[k];
        g.a[k] += std::max(-1.0, std::min(1.0, step[n + k]));
      }
      const double c2 = residuals(g, y, sr, rn);
      if (std::isfinite(c2) && c2 < cost) {
        f = g;
        r.swap(rn);
        cost = c2;
        lambda = std::max(1e-12, lambda * 0.3);
        improved = true;
        break;
      }
      lambda *= 10.0;
    }
    if (!improved) break;
  }
}

// linear least squares for w at fixed nodes (unit weights)
void fit_weights(Fit &f, const std::vector<double> &y) {
  const int n = (int)f.a.size(), S = (int)y.size();
  std::vector<double> A(n * n, 0.0), b(n, 0.0), x;
  for (int s = 0; s < S; ++s) {
    std::vector<double> row(n);
    for (int k = 0; k < n; ++k) row[k] = y[s] * std::exp(-y[s] * std::exp(f.a[k]));
    for (int i = 0; i < n; ++i) {
      b[i] += row[i];
      for (int j = 0; j < n; ++j) A[i * n + j] += row[i] * row[j];
    }
  }
  for (int i = 0; i < n; ++i) A[i * n + i] *= 1.0 + 1e-10;
  if (solve_spd(A, b, n, x)) f.w = x;
}

Fit solve_interval(Fit f, double R, int outer) {
  const int S = 240;
  std::vector<double> y(S), rho(S, 1.0 / S), sr(S);
  for (int s = 0; s < S; ++s) y[s] = std::exp(std::log(R) * s / (S - 1));
  Fit best = f;
  double best_err = max_rel_error(f, R, 4000);
  for (int o = 0; o < outer; ++o) {
    for (int s = 0; s < S; ++s) sr[s] = std::sqrt(rho[s]);
    lm_fit(f, y, sr, 25);
    // Lawson update towards the minimax weights
    std::vector<double> r;
    std::vector<double> ones(S, 1.0);
    residuals(f, y, ones, r);
    double tot = 0.0;
    for (int s = 0; s < S; ++s) {
      rho[s] *= std::sqrt(std::fabs(r[s]) + 1e-300);
      tot += rho[s];
    }
    for (int s = 0; s < S; ++s) rho[s] /= tot;
    const double err = max_rel_error(f, R, 4000);
    if (std::isfinite(err) && err < best_err) { best_err = err; best = f; }
  }
  return best;
}

}  // namespace

extern "C" int ltmp2_laplace_grid(double gap, double width, int n_tau, double *tau, double *w,
                                  double *max_err) {
  if (!tau || !w || n_tau < 1 || n_tau > 24) return LTMP2_ERR_INVALID_ARG;
  if (!(gap > 0.0) || !(width >= gap) || !std::isfinite(width)) return LTMP2_ERR_INVALID_ARG;
  const double xmin = 2.0 * gap, xmax = 2.0 * width;
  const double R = std::max(xmax / xmin, 1.0 + 1e-12);
  const int n = n_tau;
  // Start 1: trapezoid rule for 1/y = int exp(-y e^t) e^t dt (analytic in |Im t| < pi/2,
  // so step h costs ~exp(-pi^2/h)); the range [t_lo, t_hi] drops tails of the same size.
  Fit f1;
  f1.a.resize(n);
  f1.w.resize(n);
  {
    double h = 1.0;
    for (int it = 0; it < 200; ++it) {
      const double C = M_PI * M_PI / h;
      const double L = std::log(C * R) + C;
      h = 0.5 * (h + L / n);
    }
    const double C = M_PI * M_PI / h;
    const double t_lo = -C - std::log(R);
    for (int k = 0; k < n; ++k) {
      f1.a[k] = t_lo + h * (k + 0.5);
      f1.w[k] = h * std::exp(f1.a[k]);
    }
  }
  // Start 2: log-spaced nodes with least-squares weights
  Fit f2;
  f2.a.resize(n);
  f2.w.resize(n);
  for (int k = 0; k < n; ++k) {
    const double t = (n == 1) ? 0.5 : (double)k / (n - 1);
    f2.a[k] = std::log(0.3 / R) + t * (std::log(2.0 + 0.5 * n) - std::log(0.3 / R));
  }
  {
    std::vector<double> y(400);
    for (int s = 0; s < 400; ++s) y[s] = std::exp(std::log(R) * s / 399.0);
    fit_weights(f2, y);
  }
  Fit g1 = solve_interval(f1, R, 40);
  Fit g2 = solve_interval(f2, R, 40);
  Fit f = (max_rel_error(g1, R, 4000) <= max_rel_error(g2, R, 4000)) ? g1 : g2;
  const double err = max_rel_error(f, R, 20000);
  if (!std::isfinite(err) || err >= 1.0) return LTMP2_ERR_NO_CONVERGENCE;
  std::vector<int> order(n);
  for (int k = 0; k < n; ++k) order[k] = k;
  std::sort(order.begin(), order.end(), [&](int x, int y) { return f.a[x] < f.a[y]; });
  for (int k = 0; k < n; ++k) {
    tau[k] = std::exp(f.a[order[k]]) / xmin;
    w[k] = f.w[order[k]] / xmin;
  }
  if (max_err) *max_err = err;
  return LTMP2_OK;
}
