// Host FP64 generation of the REXII coefficients (arXiv 2008.11607, Section 2.1
// and Appendices A, B).  The device kernels consume tables built from these.
#include <math.h>

#include "internal.h"

namespace rexi {

// Appendix A, Table tab:coef_al: mu and a_l for l = 0..24 (a_{-l} = conj(a_l)).
// The table prints a separate sign column; it is the sign of the real part
// (with the other reading the Gaussian fit error is O(1) instead of < 8e-15).
static const double kMu = -5.133333333333333;
static const double kARe[kL + 1] = {
    -6.520430828919864e+01, 4.261818064131437e+01,  -9.801650304425239e+00, -1.054225194693395e+00,
    7.950505668209775e-01,  -1.218558380859130e-01, 7.365401806949337e-03,  -2.801087265991056e-04,
    1.254835436432561e-04,  2.295472292491263e-04,  1.858484460459430e-04,  4.068056518449676e-05,
    -8.341508001647741e-05, -9.970528169841103e-05, -3.499639858693093e-05, 2.295021920298455e-05,
    2.931048772724314e-05,  7.502088478301169e-06,  -5.815291167450100e-06, -4.069948458364005e-06,
    7.932524475429588e-08,  6.120984882186265e-07,  5.531365159161319e-08,  -2.867805871375946e-08,
    -1.143081277095316e-09};
static const double kAIm[kL + 1] = {
    0.0,                    2.761406741120911e+01,  -2.189295463610722e+01, 6.791786454153551e+00,
    -8.904997258367445e-01, 3.321241563407446e-02,  2.212802103193251e-03,  -5.566945197754387e-04,
    -2.467200513365371e-04, -8.494118951459107e-05, 9.242889460185034e-05,  1.653479957565515e-04,
    1.045331460447588e-04,  -5.856228484297677e-06, -6.129059473910835e-05, -4.099832469456381e-05,
    1.708815129697846e-07,  1.525082051744077e-05,  6.919604247338349e-06,  -1.440010113050771e-06,
    -1.794169428574330e-06, -1.131894636585849e-07, 1.585749903175946e-07,  1.239499740327838e-08,
    -2.763239274253499e-09};

double table_mu() { return kMu; }

GaussFit table_fit() {
  GaussFit g;
  g.mu = kMu;
  for (int l = 0; l <= kL; ++l) {
    g.are[l] = kARe[l];
    g.aim[l] = kAIm[l];
  }
  return g;
}

void table_a(double re[kL + 1], double im[kL + 1]) {
  for (int l = 0; l <= kL; ++l) {
    re[l] = kARe[l];
    im[l] = kAIm[l];
  }
}

bool valid_h(double h) { return h > 0.0 && h < M_PI && isfinite(h); }
bool valid_tol(double tol) { return tol >= 1e-16 && tol <= 0.1 && isfinite(tol); }

// Appendix B: psi_h(z) <= tol for |z| >= c h with c = 2 sqrt(-ln(sqrt(4 pi) tol));
// the two Gaussians beyond the truncation must be below tol, which leaves
// m0 = c - 1 (rounded up here).  eq. matrixAccuracyBound: tau rho <= (M - m0) h.
int pole_count(double tau_rho, double h, double tol) {
  if (!(tau_rho >= 0.0) || !isfinite(tau_rho) || !valid_h(h) || !valid_tol(tol)) return -1;
  const double c = 2.0 * sqrt(-log(sqrt(4.0 * M_PI) * tol));
  const double m0 = ceil(c - 1.0);
  const double Mf = ceil(tau_rho / h) + m0;
  if (Mf > 50000000.0) return -1;
  return (int)Mf;
}

// c1_n = h sum_{k=L1(n)}^{L2(n)} Re(a_k) b_{n-k}, c2_n = h sum Im(a_k) b_{n-k},
// b_m = e^{-i m h} e^{h^2}, L1 = max(-L, n-M), L2 = min(L, n+M), n = -N..N,
// for the fit (mu, a_l) of Step 2 (a_{-l} = conj(a_l)).
// bre/bim: 2M + 1 values of scratch (b_m at m + M); c*: 2N + 1 values each.
void rexii_terms_into_fit(int M, double h, const GaussFit& fit, double* bre, double* bim, double* c1re,
                          double* c1im, double* c2re, double* c2im) {
  const int N = M + kL;
  const double eh2 = exp(h * h);
  for (int m = -M; m <= M; ++m) {
    const double ang = (double)m * h;
    bre[m + M] = eh2 * cos(ang);
    bim[m + M] = -eh2 * sin(ang);
  }
  for (int n = -N; n <= N; ++n) {
    const int k0 = (n - M > -kL) ? n - M : -kL;
    const int k1 = (n + M < kL) ? n + M : kL;
    double s1r = 0.0, s1i = 0.0, s2r = 0.0, s2i = 0.0;
    for (int k = k0; k <= k1; ++k) {
      const int kk = k < 0 ? -k : k;
      const double are = fit.are[kk];
      const double aim = k < 0 ? -fit.aim[kk] : fit.aim[kk];  // a_{-k} = conj(a_k)
      const double br = bre[n - k + M], bi = bim[n - k + M];
      s1r += are * br;
      s1i += are * bi;
      s2r += aim * br;
      s2i += aim * bi;
    }
    c1re[n + N] = h * s1r;
    c1im[n + N] = h * s1i;
    c2re[n + N] = h * s2r;
    c2im[n + N] = h * s2i;
  }
}

void rexii_terms_into(int M, double h, double* bre, double* bim, double* c1re, double* c1im, double* c2re,
                      double* c2im) {
  static const GaussFit tab = table_fit();
  rexii_terms_into_fit(M, h, tab, bre, bim, c1re, c1im, c2re, c2im);
}

void rexii_terms_fit(int M, double h, const GaussFit& fit, TermSet* ts) {
  const int N = M + kL;
  ts->M = M;
  ts->N = N;
  ts->h = h;
  ts->mu = fit.mu;
  const int nt = 2 * N + 1;
  ts->c1re.assign(nt, 0.0);
  ts->c1im.assign(nt, 0.0);
  ts->c2re.assign(nt, 0.0);
  ts->c2im.assign(nt, 0.0);
  std::vector<double> bre(2 * M + 1), bim(2 * M + 1);
  rexii_terms_into_fit(M, h, fit, bre.data(), bim.data(), ts->c1re.data(), ts->c1im.data(), ts->c2re.data(),
                       ts->c2im.data());
}

void rexii_terms(int M, double h, TermSet* ts) { rexii_terms_fit(M, h, table_fit(), ts); }

}  // namespace rexi
