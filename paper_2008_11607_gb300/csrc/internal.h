// Internal declarations shared by the librexi translation units.
// Nothing here is part of the public ABI (see include/rexi.h).
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include <vector>

#include "rexi.h"

namespace rexi {

constexpr int kL = 24;             // conjugate pairs of the rational Gaussian fit (Appendix A)
constexpr int kMaxStages = 40;     // FFT stages (radix >= 2, n <= 8192)
constexpr int kMaxRadix = 127;     // largest prime factor accepted for FFT lengths

// ---- host coefficient generation (coeffs.cpp) ----------------------------
struct TermSet {
  int M = 0, N = 0;
  double h = 0.0, mu = 0.0;
  std::vector<double> c1re, c1im, c2re, c2im;  // n = -N..N at index n + N
};
int pole_count(double tau_rho, double h, double tol);  // -1 on bad arguments
bool valid_h(double h);
bool valid_tol(double tol);
double table_mu();
void table_a(double re[kL + 1], double im[kL + 1]);
// A rational fit of the Gaussian (Section 2.1 Step 2): mu and a_l, l = 0..L
// (a_{-l} = conj(a_l)).  table_fit() is Table tab:coef_al.
struct GaussFit {
  double mu = 0.0;
  double are[kL + 1] = {0.0}, aim[kL + 1] = {0.0};
};
GaussFit table_fit();
void rexii_terms(int M, double h, TermSet* ts);
void rexii_terms_fit(int M, double h, const GaussFit& fit, TermSet* ts);
void rexii_terms_into_fit(int M, double h, const GaussFit& fit, double* bre, double* bim, double* c1re,
                          double* c1im, double* c2re, double* c2im);
// Least-squares refit on Leja points (refit.cpp); false on bad arguments.
bool gauss_refit(double mu, int K, double xmax, int n_candidates, GaussFit* out, double* max_err);
// The same sums into caller arrays (no allocation): bre/bim hold 2M + 1
// values of scratch, c1re..c2im receive 2N + 1 values each (index n + N).
void rexii_terms_into(int M, double h, double* bre, double* bim, double* c1re, double* c1im, double* c2re,
                      double* c2im);

// Host: a double as a double-float pair (hi = nearest float, lo = the rest).
inline float2 df_split_host(double v) {
  const float h = (float)v;
  return make_float2(h, (float)(v - (double)h));
}

// Records the text returned by rexi_last_error_message() (api.cu).
void set_last_error(const char* msg);

// ---- FFT (fft.cu) ---------------------------------------------------------
struct FftPlan1D {
  int n = 0;
  int nstages = 0;
  int radix[kMaxStages] = {0};
  const double2* tw = nullptr;  // device table w[t] = exp(-2 pi i t / n), t < n
  const float4* twf = nullptr;  // the same as double-float pairs (re_hi, re_lo, im_hi, im_lo), then the
                                // per-stage grouping of df_twiddles (2n entries), or null
};
bool fft_factor(int n, FftPlan1D* p);  // fills n, nstages, radix; false if unsupported
// Forward (sign -1) or inverse (sign +1, scaled by `scale`) 2-D transform of
// `nfields` fields of ny x nx complex128, from `in` to `out` (may alias).
// zero_imag_in: treat the input as real; real_out: write Re, imaginary 0.
cudaError_t fft2d(const double2* in, double2* out, int nfields, const FftPlan1D& px,
                  const FftPlan1D& py, int sign, double scale, int zero_imag_in, int real_out,
                  cudaStream_t s);
// The same in double-float arithmetic (FP32 pipes, about 48 significant bits)
// when both plans carry double-float twiddles; FP64 otherwise.
cudaError_t fft2d_df(const double2* in, double2* out, int nfields, const FftPlan1D& px,
                     const FftPlan1D& py, int sign, double scale, int zero_imag_in, int real_out,
                     cudaStream_t s);
void split_twiddles(const double2* tw, int n, float4* out);  // host: FP64 table -> double-float
// host: the double-float twiddle table of a transform (2 p.n entries: w[t], then grouped per stage)
void df_twiddles(const double2* tw, const FftPlan1D& p, float4* out);
// Real input (nx = 2 m even): forward transform of the real parts of `in`
// into the half spectrum, ny x (m + 1) complex128 per field (field stride
// ny (m + 1)), through an m-point transform per row (pxh: plan of length m);
// inverse from the half spectrum (overwritten) to real fields (imaginary 0),
// scaled.  df: 0 FP64; 1 double-float arithmetic (when every plan carries
// double-float twiddles) with an FP64 half spectrum; 2 the same with the half
// spectrum kept as double-float pairs (float4 per value, 16 bytes like FP64)
// for a double-float combine pass.
bool fft_df_ready(const FftPlan1D& px, const FftPlan1D& pxh, const FftPlan1D& py);
cudaError_t fft2d_r2c(const double2* in, double2* spec, int nfields, const FftPlan1D& px, const FftPlan1D& pxh,
                      const FftPlan1D& py, int df, cudaStream_t s);
cudaError_t fft2d_c2r(double2* spec, double2* out, int nfields, const FftPlan1D& px, const FftPlan1D& pxh,
                      const FftPlan1D& py, double scale, int df, cudaStream_t s);

// ---- Fourier-path pole kernels (pole_fft.cu) ------------------------------
struct SymbolParams {
  int nx, ny;
  double inv_dx, inv_dy, g, f, H;
  const double2* half_x;  // (cos(pi k/nx), sin(pi k/nx)), k < nx
  const double2* half_y;
  int spectral = 0;       // 1: spectral derivatives on a collocated grid (no averaging);
                          // 2: the scalar operator i (d_xx + d_yy) acting on each field
  double shift = 0.0;     // spectral == 2: sigma of the shift nu = i sigma (omega = lambda - sigma)
};
struct FusedScalars {
  double tau, q, R0re, R0im;  // q = (h mu)^2, R0 = r(0) over the selected terms
  int nterms;                 // scalar terms in the table
  int adjoint;                // apply r(tau B)^H instead of r(tau B)
  int exact_hn = 1;           // mixed table: every h n lies on the split grid (no low part)
};
cudaError_t pole_fused_fp64(double2* spec, const SymbolParams& sp, const double* table,
                            const FusedScalars& fs, cudaStream_t s);
// Orbits of the wavenumber grid under the symmetries of omega(k): k -> -k
// separately in x and y (|sin|, |cos| of the half angles are even), and
// kx <-> ky when the grid is square with equal spacing.  One pole sum per
// orbit, then a combine pass over every wavenumber with its own symbol.
struct OrbitParams {
  int ax, ay;  // nx/2 + 1, ny/2 + 1 (folded index ranges)
  int sym;     // 1: swap-symmetric (representatives a <= b, triangular index)
  int norb;    // number of orbits
};
OrbitParams orbit_params(const SymbolParams& sp);
int orbit_slice_cap(int norb);  // most term slices a workspace holds partial sums for
// Term slices for the orbit kernels: the count that minimises the modelled
// run time (waves of resident blocks x terms per block), at most `cap`.
int pole_orbit_slices(int form, int norb, int nterms, int cap);
// part[s * norb + o] = sum of the table's terms in slice s at x = tau omega(rep(o)).
cudaError_t pole_orbits_fp64(double2* part, int slices, const SymbolParams& sp, const OrbitParams& op,
                             const double* table, const FusedScalars& fs, cudaStream_t s);
cudaError_t pole_orbits_mixed(double2* part, int slices, const SymbolParams& sp, const OrbitParams& op,
                              const float* table, const FusedScalars& fs, double grid, cudaStream_t s);
// spec <- r(tau B) spec at every wavenumber, R+ = sum over slices of part:
// a per-orbit pass writes the combine scalars to `fin`
// (orbit_scalars_bytes(norb) bytes, 32-byte aligned), then a pass over the
// wavenumbers applies them.  row_len: nx (full spectrum, rows of nx values)
// or nx/2 + 1 (half spectrum of real input, wavenumbers kx = 0..nx/2 only).
cudaError_t pole_orbit_combine(double2* spec, const double2* part, int slices, void* fin, const SymbolParams& sp,
                               const OrbitParams& op, const FusedScalars& fs, int row_len, cudaStream_t s);
size_t orbit_scalars_bytes(int norb);
// The same on a half spectrum kept as double-float pairs (float4 per value),
// in double-float arithmetic; C-grid symbol and real R0 (real input) only,
// cudaErrorInvalidValue otherwise.  half_x_df, half_y_df: (cos, sin) of
// pi k / n as double-float pairs.
// Complex input in the mixed form (C grid): the combine of pole_orbit_combine
// (full spectrum, FP64 storage) in double-float arithmetic.
cudaError_t pole_orbit_combine_dfc(double2* spec, const double2* part, int slices, void* fin, const SymbolParams& sp,
                                   const float4* half_x_df, const float4* half_y_df, const OrbitParams& op,
                                   const FusedScalars& fs, cudaStream_t s);
// Scalar operators (SymbolParams::spectral == 2): spec <- phase R(k) spec on
// every field of the full spectrum (rows of nx values), R the sum over slices
// of the orbit's partial sums; conj(phase R) for the adjoint.
cudaError_t pole_orbit_combine_scalar(double2* spec, const double2* part, int slices, const SymbolParams& sp,
                                      const OrbitParams& op, double2 phase, int adjoint, cudaStream_t s);
cudaError_t pole_orbit_combine_df(void* spec_df, const double2* part, int slices, void* fin, const SymbolParams& sp,
                                  const float4* half_x_df, const float4* half_y_df, const OrbitParams& op,
                                  const FusedScalars& fs, int row_len, cudaStream_t s);
struct PlainScalars {
  double tau;
  int nterms;   // terms in this chunk
  int adjoint;
};
cudaError_t pole_plain_terms(const double2* spec, double2* chunk, const SymbolParams& sp,
                             const double2* table, const PlainScalars& ps, cudaStream_t s);
cudaError_t pole_plain_reduce(const double2* chunk, double2* acc, long long nk3, int nterms,
                              int first, cudaStream_t s);

}  // namespace rexi
