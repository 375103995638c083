// Least-squares refit of the rational approximation of the Gaussian
// (arXiv 2008.11607, Section 2.1 Step 2, host FP64).
//
// R(x) = a_0 mu / (x^2 + mu^2)
//      + sum_{l=1}^{L} [2 mu Re(a_l) (mu^2 + l^2 + x^2) + 2 l Im(a_l) (mu^2 + l^2 - x^2)]
//                      / [x^4 + 2 (mu^2 - l^2) x^2 + (mu^2 + l^2)^2]
// (eq. A(x,mu), the conjugate-symmetric form a_{-l} = conj(a_l)) is linear in
// y = [a_0, Re a_1..Re a_L, Im a_1..Im a_L]; y minimises
// sum_k (psi_1(x_k) - R(x_k))^2 (eq. minl2approx), psi_1(x) = exp(-x^2/4)/sqrt(4 pi),
// on K points chosen one at a time like Leja points: x_1 = 0, and each next
// point is the candidate (n_candidates equally spaced values of [0, xmax];
// R is even, so the half line suffices) that maximises the product of its
// distances to the points already chosen.  The paper leaves K, the interval
// and mu open; mu is a parameter here (Table tab:coef_al's mu by default in
// the bindings).  The system is solved by Householder QR on the column-scaled
// design matrix (its condition number is of order 1e12 for L = 24, where
// the normal equations would lose every digit).
#include <math.h>

#include <algorithm>
#include <vector>

#include "internal.h"

namespace rexi {
namespace {

constexpr int kCols = 2 * kL + 1;

double psi1(double x) { return exp(-0.25 * x * x) / sqrt(4.0 * M_PI); }

void design_row(double x, double mu, double* row) {
  const double x2 = x * x, m2 = mu * mu;
  row[0] = mu / (x2 + m2);
  for (int l = 1; l <= kL; ++l) {
    const double l2 = (double)l * l;
    const double den = x2 * x2 + 2.0 * (m2 - l2) * x2 + (m2 + l2) * (m2 + l2);
    row[l] = 2.0 * mu * (m2 + l2 + x2) / den;
    row[kL + l] = 2.0 * l * (m2 + l2 - x2) / den;
  }
}

double eval_fit(double x, const GaussFit& f) {
  double row[kCols];
  design_row(x, f.mu, row);
  double r = row[0] * f.are[0];
  for (int l = 1; l <= kL; ++l) r += row[l] * f.are[l] + row[kL + l] * f.aim[l];
  return r;
}

std::vector<double> leja(int K, double xmax, int ncand) {
  std::vector<double> cand(ncand), logd(ncand), pts;
  for (int i = 0; i < ncand; ++i) cand[i] = xmax * (double)i / (double)(ncand - 1);
  pts.push_back(0.0);
  for (int i = 0; i < ncand; ++i) logd[i] = log(fabs(cand[i]) + 1e-300);
  while ((int)pts.size() < K) {
    int best = 0;
    for (int i = 1; i < ncand; ++i)
      if (logd[i] > logd[best]) best = i;
    const double p = cand[best];
    pts.push_back(p);
    for (int i = 0; i < ncand; ++i) logd[i] += log(fabs(cand[i] - p) + 1e-300);
  }
  return pts;
}

// Householder QR of A (m x n, column-major, m >= n): the reflectors are kept
// below the diagonal (their first entries in v0), R on and above it.
struct QR {
  int m = 0, n = 0;
  std::vector<double> a, v0, vv;
  bool factor(int m_, int n_, const std::vector<double>& A0) {
    m = m_;
    n = n_;
    a = A0;
    v0.assign(n, 0.0);
    vv.assign(n, 0.0);
    for (int j = 0; j < n; ++j) {
      double nrm = 0.0;
      for (int i = j; i < m; ++i) nrm += at(i, j) * at(i, j);
      nrm = sqrt(nrm);
      if (nrm == 0.0) return false;
      const double alpha = at(j, j) > 0 ? -nrm : nrm;
      v0[j] = at(j, j) - alpha;  // v = x - alpha e_1
      double s = v0[j] * v0[j];
      for (int i = j + 1; i < m; ++i) s += at(i, j) * at(i, j);
      vv[j] = s;
      for (int c = j + 1; c < n; ++c) {
        double d = v0[j] * at(j, c);
        for (int i = j + 1; i < m; ++i) d += at(i, j) * at(i, c);
        const double t = 2.0 * d / s;
        at(j, c) -= t * v0[j];
        for (int i = j + 1; i < m; ++i) at(i, c) -= t * at(i, j);
      }
      at(j, j) = alpha;
    }
    return true;
  }
  double& at(int i, int j) { return a[(size_t)j * m + i]; }
  // y = argmin ||A y - b||: Q^T b, then back substitution with R
  void solve(std::vector<double> b, std::vector<double>& y) {
    for (int j = 0; j < n; ++j) {
      double d = v0[j] * b[j];
      for (int i = j + 1; i < m; ++i) d += at(i, j) * b[i];
      const double t = 2.0 * d / vv[j];
      b[j] -= t * v0[j];
      for (int i = j + 1; i < m; ++i) b[i] -= t * at(i, j);
    }
    y.assign(n, 0.0);
    for (int j = n - 1; j >= 0; --j) {
      double s = b[j];
      for (int c = j + 1; c < n; ++c) s -= at(j, c) * y[c];
      y[j] = s / at(j, j);
    }
  }
};

// min ||A y - b|| by Householder QR, then refinement steps on the residual
// (y += argmin ||A d - (b - A y)||, the residual formed in doubled
// precision), which recover digits the QR solve loses to the design matrix's
// condition number.
bool lstsq_qr(int m, int n, const std::vector<double>& A0, const std::vector<double>& b, std::vector<double>& y) {
  QR qr;
  if (!qr.factor(m, n, A0)) return false;
  qr.solve(b, y);
  std::vector<double> r(m), d;
  for (int it = 0; it < 4; ++it) {
    // residual in twice the working precision (Ogita, Rump and Oishi's Dot2:
    // each product split exactly by an FMA, the sum carried with TwoSum)
    for (int i = 0; i < m; ++i) {
      double s = b[i], c = 0.0;
      for (int j = 0; j < n; ++j) {
        const double p = -A0[(size_t)j * m + i] * y[j];
        const double pe = fma(-A0[(size_t)j * m + i], y[j], -p);
        const double t = s + p;
        const double z = t - s;
        c += ((s - (t - z)) + (p - z)) + pe;
        s = t;
      }
      r[i] = s + c;
    }
    qr.solve(r, d);
    for (int j = 0; j < n; ++j) y[j] += d[j];
  }
  return true;
}

}  // namespace

bool gauss_refit(double mu, int K, double xmax, int n_candidates, GaussFit* out, double* max_err) {
  // the Leja selection costs K x n_candidates logarithms: keep a call to seconds
  if (!(mu < 0.0) || !isfinite(mu) || K < kCols || K > 20000 || !(xmax > 0.0) || !isfinite(xmax) ||
      n_candidates < K || n_candidates > 1000000 || (double)K * (double)n_candidates > 5e8)
    return false;
  const std::vector<double> x = leja(K, xmax, n_candidates);
  std::vector<double> a((size_t)K * kCols), b(K), scale(kCols, 0.0), y;
  double row[kCols];
  for (int k = 0; k < K; ++k) {
    design_row(x[k], mu, row);
    for (int j = 0; j < kCols; ++j) {
      a[(size_t)j * K + k] = row[j];
      scale[j] = std::max(scale[j], fabs(row[j]));
    }
    b[k] = psi1(x[k]);
  }
  for (int j = 0; j < kCols; ++j)
    for (int k = 0; k < K; ++k) a[(size_t)j * K + k] /= scale[j];
  if (!lstsq_qr(K, kCols, a, b, y)) return false;
  GaussFit f;
  f.mu = mu;
  f.are[0] = y[0] / scale[0];
  f.aim[0] = 0.0;
  for (int l = 1; l <= kL; ++l) {
    f.are[l] = y[l] / scale[l];
    f.aim[l] = y[kL + l] / scale[kL + l];
  }
  if (max_err) {
    // on [-1.5 xmax, 1.5 xmax], 0.005-spaced (R and psi_1 are even)
    double worst = 0.0;
    const int np = (int)ceil(1.5 * xmax / 0.005);
    for (int i = 0; i <= np; ++i) {
      const double xx = 1.5 * xmax * (double)i / (double)np;
      worst = std::max(worst, fabs(psi1(xx) - eval_fit(xx, f)));
    }
    *max_err = worst;
  }
  *out = f;
  return true;
}

}  // namespace rexi
