/*
 * rexi.h -- C ABI of librexi, a GB300 (sm_103a) implementation of one REXII
 * time step  out = r(dt A) f  ~  e^{dt A} f  for the linear rotating
 * shallow-water (LRSW) operator A on a doubly periodic staggered (C) grid.
 *
 * Method: Caliari, Einkemmer, Moriggl, Ostermann, "An accurate and
 * time-parallel rational exponential integrator for hyperbolic and oscillatory
 * PDEs" (arXiv 2008.11607).  r is the REXII rational approximation of
 * Section 2.1 (eq. modifiedRexi) with the L = 24 conjugate-symmetric
 * coefficients of Appendix A (Table tab:coef_al); the matrix form is
 * eq. REXI_Modified_matrix, reduced for real data by
 * eq. modifiedRexiMatrixReducedSum; the pole count follows
 * eq. matrixAccuracyBound with the tolerance constant of Appendix B.
 *
 * Operator (Section 4, with depth H, gravity g, Coriolis f):
 *   eta_t = -H(x,y) (u_x + v_y),  u_t = -g eta_x + f v,  v_t = -g eta_y - f u,
 * second-order centred differences on the C grid: eta_{i,j} at cell centres
 * ((i+1/2)dx, (j+1/2)dy), u_{i,j} at ((i+1)dx, (j+1/2)dy), v_{i,j} at
 * ((i+1/2)dx, (j+1)dy); Coriolis by the four-point average (v to u) and its
 * transpose (u to v).
 *
 * Conventions shared by every entry point
 * ---------------------------------------
 * - State layout: 3 fields (eta, u, v), each ny rows of nx complex128 values
 *   (interleaved re, im doubles), x fastest:  element (field, j, i) at
 *   ((field * ny + j) * nx + i).  Device pointers unless stated otherwise;
 *   they must be 16-byte aligned.
 * - Memory ownership: the caller owns every buffer passed in.  The library
 *   never frees caller memory.  A plan owns only small tables (twiddles,
 *   half angles, and up to eight coefficient tables of the FP64 and mixed
 *   Fourier forms, one per pole count and term range, allocated by the first
 *   step that needs one); rexi_plan_create allocates the fixed tables and
 *   rexi_plan_destroy frees them all.
 * - A plan is used by one host thread at a time; its steps may be enqueued on
 *   different streams.
 *   rexi_step allocates nothing: its scratch is the caller's workspace.
 * - Streams: `stream` is a cudaStream_t passed as void* (NULL = legacy
 *   default stream).  Calls are asynchronous on that stream; inputs must stay
 *   valid and unmodified until the stream reaches the call.
 * - Errors: every call returns a rexi_status; nothing aborts, traps or waits
 *   without bound.  Invalid arguments give REXI_EINVAL and launch nothing.
 * - Precision: coefficients (host) and all accumulation over poles are FP64.
 */
#ifndef REXI_H
#define REXI_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct rexi_plan_s* rexi_plan_t; /* opaque, library-owned */

typedef enum {
  REXI_OK = 0,
  REXI_EINVAL = -1,      /* bad argument, size, alignment or unsupported combination */
  REXI_ENOMEM = -2,      /* a plan table could not be allocated, or the workspace is too small */
  REXI_ECUDA = -3,       /* a CUDA runtime call or kernel launch failed */
  REXI_ENOCONV = -4,     /* Krylov iteration cap reached before the residual target */
  REXI_ETIMEOUT = -5,    /* a bounded device-side wait gave up */
  REXI_EUNSUPPORTED = -6 /* the requested form is not available for this plan */
} rexi_status;

/* Arithmetic form of the pole loop (plan creation). */
enum {
  REXI_FORM_FP64 = 0,  /* fused: all solves of a wavenumber in FP64 registers (once per
                          orbit of omega's symmetries), FP64 transforms and combine */
  REXI_FORM_MIXED = 1, /* fused: solves in FP32 pairs (double-float); transforms and, for
                          real input, the half spectrum and combine in double-float;
                          FP64 at the state boundary */
  REXI_FORM_PLAIN = 2  /* paper-style: per-term solve pairs materialised, then a
                          separate reduction pass (Section 4.1, GPU algorithm) */
};

/* Per-call diagnostics; filled after an internal stream synchronisation only
   when the pointer passed to rexi_step is non-NULL. */
typedef struct {
  int32_t M;          /* Gaussian-sum half width from the pole-count rule */
  int32_t N;          /* M + L, L = 24 */
  int32_t n_terms;    /* REXII terms evaluated: N + 1 (real input) or 2N + 1 */
  int32_t n_poles;    /* single-shift poles J: 2(N + 1) or 2(2N + 1) */
  double tau_rho;     /* dt * rho(A) */
  double rho;         /* spectral radius used */
  int32_t krylov_iters;        /* Krylov path: largest iteration count over terms
                                  (shared method: Lanczos steps of the basis) */
  int32_t krylov_unconverged;  /* Krylov path: terms that hit the iteration cap */
  double krylov_max_rel_res;   /* Krylov path: largest final relative residual
                                  (shared method: the step's error bound) */
  int64_t krylov_term_iters;   /* Krylov path: CG iterations summed over all terms
                                  (shared method: Lanczos steps run in the first
                                  pass, a multiple of the check interval) */
} rexi_step_info;

/* ------------------------------------------------------------------------ */
/* Coefficients (host, FP64).                                               */
/* ------------------------------------------------------------------------ */

/* Pole count M for a given tau*rho, parameter h and tolerance.
 * M = ceil(tau_rho / h) + ceil(c(tol) - 1),  c(tol) = 2 sqrt(-ln(sqrt(4 pi) tol))
 * (eq. matrixAccuracyBound; Appendix B: c ~ 12 and m0 = c - 1 ~ 11 at
 * tol = 1e-16, so this is the paper's M = ceil(rho/h) + 11 there).
 * EINVAL unless tau_rho >= 0, 0 < h < pi and 1e-16 <= tol <= 0.1. */
rexi_status rexi_pole_count(double tau_rho, double h, double tol, int32_t* M_out);

/* REXII term coefficients of eq. modifiedRexi (Section 2.1, Step 3):
 *   c1_n = h sum_{k=L1(n)}^{L2(n)} Re(a_k) b_{n-k},  c2_n = h sum Im(a_k) b_{n-k},
 *   b_m = e^{-imh} e^{h^2} (eq. bm), L1 = max(-L, n-M), L2 = min(L, n+M),
 * for n = -N..N (N = M + 24), written as interleaved (re, im) doubles:
 * c1_re_im[2*(n+N)], c1_re_im[2*(n+N)+1].  Pass NULL arrays to query the
 * count (*n_terms = 2N+1); otherwise cap >= 2N+1 is required (EINVAL).
 * Also returns mu (Table tab:coef_al) so that alpha_n = h(mu + i n). */
rexi_status rexi_rexii_terms(int32_t M, double h, double* mu_out, int32_t* n_terms,
                             double* c1_re_im, double* c2_re_im, int32_t cap);

/* Single-shift partial-fraction form of the same rational function:
 *   r(z) = sum_j beta_j / (z - z_j),  z = dt * (eigenvalue of A),
 * obtained from each term (C1 - C2 z)/((alpha_{-n} - z)(alpha_n + z)) of
 * eq. REXI_Modified_matrix (C1 = c1 h mu + c2 h n, C2 = i c2) by partial
 * fractions.  real_input = 1 gives the reduced set n = 0..N with
 * Gamma_0 = 1, Gamma_n = 2 folded into beta (the result is then Re of the
 * sum, eq. modifiedRexiMatrixReducedSum): J = 2(N+1); real_input = 0 gives
 * n = -N..N: J = 2(2N+1).  Arrays are interleaved (re, im), host memory;
 * NULL arrays query *n_poles; otherwise cap >= J (EINVAL). */
rexi_status rexi_coeffs(double tau_rho, double tol, double h, int32_t real_input, int32_t* M_out,
                        int32_t* n_poles, double* poles_re_im, double* weights_re_im, int32_t cap);

/* The rational approximation of the Gaussian psi_1 (Section 2.1 Step 2),
 * R(x) = Re sum_{l=-L}^{L} a_l / (ix + mu + il), L = 24, a_{-l} = conj(a_l).
 * Coefficient arrays hold a_l for l = -L..L as interleaved (re, im) doubles
 * (2 (2L + 1) = 98 values, a_l at index 2 (l + L)); host memory, caller-owned.
 *
 * rexi_gaussian_fit_table: Table tab:coef_al (Appendix A) and its mu.
 *
 * rexi_gaussian_refit: the least-squares fit of eq. minl2approx, written in
 * the real form of eq. A(x,mu) (unknowns a_0, Re a_l, Im a_l), on K points
 * chosen like Leja points: x_1 = 0, then each next point is the one of
 * n_candidates equally spaced candidates in [0, xmax] that maximises the
 * product of distances to the points chosen so far (R is even).  Solved by
 * Householder QR of the column-scaled design matrix in FP64.  The paper leaves
 * K, the interval and the choice of mu open; e.g. mu from the table, K = 200,
 * xmax = 40, 20001 candidates reach max |psi_1 - R| ~ 5e-14 on [-60, 60]
 * (the table: 8.1e-15).  max_err (nullable): max |psi_1 - R| on
 * [-1.5 xmax, 1.5 xmax] at spacing 0.005.  EINVAL unless mu < 0,
 * 2L + 1 <= K <= 20000, xmax > 0, K <= n_candidates <= 1e6 and
 * K n_candidates <= 5e8 (the point selection costs K n_candidates steps).
 *
 * rexi_plan_set_gaussian_fit: the plan's constant-depth steps use (mu, a)
 * instead of the table in every REXII/REXI coefficient (a_re_im NULL restores
 * the table).  EINVAL unless mu < 0, the values are finite and
 * a_{-l} = conj(a_l) to 1e-14 of the largest |a|.  Frees the plan's cached
 * coefficient tables (waiting for the device).  The variable-depth path
 * keeps the table: its steps return REXI_EUNSUPPORTED while a custom fit is
 * set. */
rexi_status rexi_gaussian_fit_table(double* mu, double* a_re_im);
rexi_status rexi_gaussian_refit(double mu, int32_t K, double xmax, int32_t n_candidates, double* a_re_im,
                                double* max_err);
rexi_status rexi_plan_set_gaussian_fit(rexi_plan_t plan, double mu, const double* a_re_im);

/* ------------------------------------------------------------------------ */
/* Plans.                                                                   */
/* ------------------------------------------------------------------------ */

/* Create a plan for an nx x ny grid on [0, Lx) x [0, Ly).
 * depth_dev == NULL: constant depth H_const, Fourier (FFT) path.
 * depth_dev != NULL: variable depth, ny*nx FP64 values at eta points
 *   (device memory, must stay valid for the plan's lifetime): Krylov path.
 * form: REXI_FORM_FP64 / REXI_FORM_MIXED / REXI_FORM_PLAIN.
 * h: REXII parameter (0 < h < pi; the paper's best range is 0.3..0.6).
 * Sizes: 2 <= nx, ny <= 4096, every prime factor of nx and ny <= 127
 * (constant-depth path; the variable-depth path accepts 3 <= nx, ny <= 16384).
 * g > 0, H_const > 0 (and depth values > 0), Lx, Ly > 0.
 * Allocates device tables (cudaMalloc) on the current device. */
rexi_status rexi_plan_create(rexi_plan_t* plan, int32_t nx, int32_t ny, double Lx, double Ly,
                             double g, double f, double H_const, const double* depth_dev,
                             int32_t form, double h);

void rexi_plan_destroy(rexi_plan_t plan);

/* Spectral radius of A used for the pole count: the exact maximum over the
 * discrete wavenumbers for constant depth, and the bound
 * sqrt(g Hmax (4/dx^2 + 4/dy^2)) + |f| for variable depth (Hmax taken from
 * depth_dev at plan creation). */
rexi_status rexi_spectral_radius(rexi_plan_t plan, double* rho_out);

/* Spatial symbol of the constant-depth (Fourier) path:
 * REXI_SYMBOL_CGRID (default): the staggered second-order operator above;
 * REXI_SYMBOL_SPECTRAL: spectral derivatives on a collocated grid
 *   (d/dx -> i k', k' = 2 pi k / Lx with the signed wavenumber, Nyquist as
 *   +n/2, no Coriolis averaging), the discretisation behind eq. lswRoh
 *   (rho = sqrt(2 pi^2 D^2 + 1) for D x D on the unit square, H = g = f = 1).
 * Recomputes rho.  Variable-depth plans accept only the C grid. */
/* REXI_SYMBOL_SCHRODINGER: the scalar operator A = i (d_xx + d_yy) by
 *   second-order centred differences (periodic), applied to each of the three
 *   fields independently (so a single wavefunction goes in field 0 with the
 *   others zero).  Its eigenvalues are i lambda(k) with
 *   lambda = -(4/dx^2) sin^2(pi kx/nx) - (4/dy^2) sin^2(pi ky/ny) in
 *   [-(4/dx^2 + 4/dy^2), 0]; with ny = 2 and data constant in y it is the
 *   one-dimensional free Schroedinger operator A_2 of Section 3.2.  Needs
 *   complex input (real_input = 0) and the FP64 or mixed form; rho is the
 *   largest |lambda - sigma| (sigma: rexi_plan_set_shift). */
enum { REXI_SYMBOL_CGRID = 0, REXI_SYMBOL_SPECTRAL = 1, REXI_SYMBOL_SCHRODINGER = 2 };
rexi_status rexi_plan_set_symbol(rexi_plan_t plan, int32_t symbol);

/* Rational approximation used by the constant-depth path (Section 2):
 * REXI_COEF_REXII (default): eq. modifiedRexi / REXI_Modified_matrix.
 * REXI_COEF_REXI: the original REXI in its matrix form for real operators,
 *   eq. originalREXImatrix, sum_n Re(beta^Re_n (tau A + alpha_n I)^{-1}) f,
 *   with beta^Re of Section 2.1 Step 3 (shallow-water symbols only; for a real
 *   operator and real data it is the rational function
 *   sum_n gamma_n (tau A + alpha_n I)^{-1}, gamma_n = (beta^Re_n + conj(beta^Re_{-n}))/2,
 *   which is what is applied to complex data too).  It is not the scalar REXI
 *   applied to the eigenvalues, so Theorem 1 and the pole-count rule do not
 *   hold for it: M is the rule's value for the plan's rho, or choose rho
 *   (rexi_plan_set_rho) to reach the M wanted.
 * REXI_COEF_REXIE: REXI Extended, eq. REXIE, for operators i B with B real
 *   (the scalar symbol only).  Per eigenvalue it is the scalar eq. originalRexi,
 *   which equals eq. modifiedRexi for real arguments (beta^Re = Re c1 + i Re c2,
 *   beta^Im = Im c1 + i Im c2), so the Fourier path evaluates it with the same
 *   term table as REXII.
 * The variable-depth path and the plain form accept REXI_COEF_REXII only
 * (REXI_EUNSUPPORTED at the step otherwise). */
enum { REXI_COEF_REXII = 0, REXI_COEF_REXI = 1, REXI_COEF_REXIE = 2 };
rexi_status rexi_plan_set_coefficients(rexi_plan_t plan, int32_t set);

/* Spectral shift of the remark in Section 2.2: e^{tau A} = e^{tau nu} e^{tau (A - nu I)}
 * with nu = i sigma, so that the pole count follows rho(A - nu I).
 * REXI_SHIFT_NONE (default): sigma = 0; REXI_SHIFT_MIDPOINT: sigma = the midpoint
 * of the operator's eigenvalue range (zeta_1 + zeta_2)/2; REXI_SHIFT_VALUE: the
 * given sigma.  A non-zero sigma needs the scalar symbol (the shallow-water
 * spectra are symmetric about 0, where the midpoint is 0): REXI_EUNSUPPORTED
 * otherwise.  Recomputes rho; rexi_plan_get_shift returns the sigma in effect. */
enum { REXI_SHIFT_NONE = 0, REXI_SHIFT_MIDPOINT = 1, REXI_SHIFT_VALUE = 2 };
rexi_status rexi_plan_set_shift(rexi_plan_t plan, int32_t mode, double sigma);
rexi_status rexi_plan_get_shift(rexi_plan_t plan, double* sigma);

/* Override the spectral radius used by the pole-count rule (rho > 0), or
 * restore the plan's own value (rho = 0).  The paper's wave scenarios take
 * rho from the highest active Fourier mode instead of the grid (Section 4,
 * text after eq. WAVESCENARIO1; Table tab:W8_M). */
rexi_status rexi_plan_set_rho(rexi_plan_t plan, double rho);

/* Krylov path settings (ignored by the FFT path): relative residual target
 * per term, iteration cap per term, number of terms solved together. */
rexi_status rexi_plan_set_krylov(rexi_plan_t plan, double rtol, int32_t max_iters, int32_t term_batch);

/* Solver of the variable-depth path (REXI_EUNSUPPORTED on constant-depth
 * plans):
 * REXI_KRYLOV_CG (default): one pole-pair CG solve per REXII term, terms
 *   batched (pair operator (alpha_{-n} - dt A)(alpha_n + dt A), Section 3's
 *   reduced sum); computes in the plan's form.
 * REXI_KRYLOV_SHARED: one Lanczos basis of K = -i dt A (self-adjoint in the
 *   energy inner product) shared by every single-shift pole z_j of the step:
 *   (dt A - z_j)^{-1} f = -i (K + i z_j)^{-1} f, and the Krylov space of a
 *   shifted system does not depend on the shift.  Every pole's residual is a
 *   multiple of the next Lanczos vector, so the error of the whole step is
 *   ||f|| b_k phi(K) v_k for a rational function phi known from the Lanczos
 *   scalars; the solver stops when b_k max |phi| over [-dt rho, dt rho]
 *   (sampled, rho the plan's spectral radius) is <= rtol (from
 *   rexi_plan_set_krylov, relative to ||f|| in the energy norm; max_iters
 *   caps the Lanczos steps), then forms sum_j beta_j x_j = V_k c.  Lanczos
 *   vectors that fit in workspace bytes beyond rexi_workspace_size (3 nx ny
 *   complex values, or 3 nx ny real values for real input, rounded up to 256
 *   bytes, each) are kept from the first pass; the rest are regenerated from
 *   the stored scalars.  Real input runs the real form of the recurrence
 *   (the vectors alternate between real and imaginary, a_j = 0); in the
 *   mixed form its vectors and stencil arithmetic are double-float (pairs of
 *   FP32 values, about 48 significant bits) with FP64 scalars and inner
 *   products.  FP64 otherwise.  Applies to rexi_step and rexi_step_adjoint,
 *   and, for real input, to rexi_step_grad_depth: two Lanczos runs (on the
 *   input and on W^{-1} grad_out), every vector kept, and the gradient as a
 *   two-sided Galerkin form over the two bases (FP64; workspace from
 *   rexi_workspace_size_grad_depth, about 2 (3 tau rho + 100) state-sized
 *   real vectors).  Complex input keeps per-term CG for the gradient. */
enum { REXI_KRYLOV_CG = 0, REXI_KRYLOV_SHARED = 1 };
rexi_status rexi_plan_set_krylov_method(rexi_plan_t plan, int32_t method);

/* Bytes of device workspace rexi_step and rexi_step_adjoint need for this
 * plan, dt and tol. */
rexi_status rexi_workspace_size(rexi_plan_t plan, double dt, double tol, int32_t real_input,
                                size_t* bytes);

/* Bytes of device workspace rexi_step_grad_depth needs (variable-depth plans;
 * REXI_EUNSUPPORTED otherwise). */
rexi_status rexi_workspace_size_grad_depth(rexi_plan_t plan, double dt, double tol, int32_t real_input,
                                           size_t* bytes);

/* ------------------------------------------------------------------------ */
/* The time step.                                                           */
/* ------------------------------------------------------------------------ */

/* out = r(dt A) in, r the REXII approximation with M from the pole-count rule
 * for dt * rho(A) and tol (eq. modifiedRexiMatrixReducedSum for real input,
 * eq. REXI_Modified_matrix otherwise).
 * real_input = 1: the imaginary parts of `in` are ignored and `out` is real
 *   (imaginary parts written as 0).  real_input = 0: complex state.
 * term_begin/term_end: evaluate only the REXII terms n with |n| in
 *   [term_begin, term_end) (0 <= term_begin <= term_end <= N + 1), so that
 *   several devices can each take a slice of the terms and sum their outputs
 *   (the step is linear in the terms); pass 0, -1 for all terms.
 * `in` and `out` may be the same buffer on the FFT path; on the Krylov path
 * they must not overlap (EINVAL).  workspace_dev: >= rexi_workspace_size
 * bytes, 256-byte aligned.  info: NULL, or filled after a stream sync. */
rexi_status rexi_step(rexi_plan_t plan, const void* in_dev, void* out_dev, double dt, double tol,
                      int32_t real_input, int32_t term_begin, int32_t term_end, void* workspace_dev,
                      size_t workspace_bytes, void* stream, rexi_step_info* info);

/* Adjoint of rexi_step with respect to the Euclidean inner product of the
 * state vector (sum of conj(a) b over all 3 nx ny entries):
 *   grad_in = r(dt A)^H grad_out,
 * i.e. the gradient of a real loss with respect to the (complex) input state
 * given its gradient with respect to the output.  Same layouts and rules as
 * rexi_step. */
rexi_status rexi_step_adjoint(rexi_plan_t plan, const void* grad_out_dev, void* grad_in_dev,
                              double dt, double tol, int32_t real_input, void* workspace_dev,
                              size_t workspace_bytes, void* stream);

/* Gradient with respect to the depth field (variable-depth plans only;
 * REXI_EUNSUPPORTED otherwise).  For out = r(dt A(H)) in and a real loss L
 * with grad_out = dL/d out (complex convention dL/dRe + i dL/dIm), ADDS dL/dH
 * to grad_depth_dev (ny * nx FP64 values at eta points, device).  With the
 * single-shift form r(dt A) = sum_j beta_j (dt A - z_j)^{-1} and H entering A
 * only through the eta row, (A v)_eta = -H div v:
 *   dL/dH_k = dt Re sum_j beta_j conj(y_j,eta,k) (div x_j)_k,
 *   x_j = (dt A - z_j)^{-1} in,  y_j = (dt A - z_j)^{-H} grad_out;
 * both are recovered per REXII term from two CG solves with the pair
 * operator (with the shared-Krylov method and real input: from two Lanczos
 * bases, see rexi_plan_set_krylov_method).  Workspace:
 * rexi_workspace_size_grad_depth bytes; info as for
 * rexi_step. */
rexi_status rexi_step_grad_depth(rexi_plan_t plan, const void* in_dev, const void* grad_out_dev,
                                 double* grad_depth_dev, double dt, double tol, int32_t real_input,
                                 void* workspace_dev, size_t workspace_bytes, void* stream, rexi_step_info* info);

/* out = r(dt A) in with HOST buffers: copies `in_host` to the device
 * workspace, runs rexi_step there and copies the result back into
 * `out_host`, all on `stream`, then synchronises the stream so that
 * `out_host` is ready on return.  Pinned host memory gives asynchronous,
 * full-bandwidth copies; pageable memory works but is staged by the driver.
 * The workspace must hold rexi_workspace_size() plus two states
 * (2 * 3 * nx * ny * 16 bytes): see rexi_workspace_size_host. */
rexi_status rexi_step_host(rexi_plan_t plan, const void* in_host, void* out_host, double dt, double tol,
                           int32_t real_input, void* workspace_dev, size_t workspace_bytes, void* stream,
                           rexi_step_info* info);

/* Workspace bytes for rexi_step_host. */
rexi_status rexi_workspace_size_host(rexi_plan_t plan, double dt, double tol, int32_t real_input,
                                     size_t* bytes);

/* rexi_step_host without the final synchronisation: the copy in, the step
 * and the copy out are enqueued on `stream` and the call returns.
 * `out_host` holds the result, and `in_host` and the workspace may be reused,
 * only once the stream has reached the end of this call's work (synchronise
 * the stream or an event recorded on it).  With pinned host memory the
 * copies run on the copy engines, so consecutive steps enqueued on two
 * streams, each with its own workspace, overlap one step's copies with the
 * other's kernels.  Steps on different streams may share the plan; the
 * kernels of a plan's host-buffer steps run in call order (each call's
 * kernels wait, after its copy in, for those of the previous call), so that
 * the GPU is never left waiting on copies of steps that finished together.
 * No per-call information is returned (use rexi_step_host for that). */
rexi_status rexi_step_host_async(rexi_plan_t plan, const void* in_host, void* out_host, double dt, double tol,
                                 int32_t real_input, void* workspace_dev, size_t workspace_bytes, void* stream);

/* Device-side phase timing of rexi_step calls: with profiling enabled, each
 * call records CUDA events on its own stream around its phases.
 * rexi_plan_read_profile waits for the recorded events, fills ms5 (5
 * doubles) with the summed milliseconds per phase since the last read
 * (ms[0] forward transform or Krylov set-up, ms[1] the pole loop over all
 * terms including the combine pass (Krylov: the CG iterations), ms[2]
 * inverse transform or final accumulation, ms[3] table upload, ms[4] the
 * part of ms[1] spent in the per-wavenumber combine pass of the FP64 and
 * mixed Fourier forms, 0 elsewhere), returns the number of profiled phase
 * sets (one per call on the Fourier path, one per term batch on the Krylov
 * path) and of kernels launched, then resets the sums. */
rexi_status rexi_plan_set_profiling(rexi_plan_t plan, int32_t enable);
rexi_status rexi_plan_read_profile(rexi_plan_t plan, double* ms5, int32_t* n_calls, int64_t* n_launches);

/* Constant-depth step that allocates nothing, for callers that may not
 * allocate device memory (code running inside another allocator's hooks or
 * memory pool, a loop with a fixed memory budget, a process whose device
 * memory is reserved up front).  It needs no plan and no workspace: its
 * scratch is one fixed static device array (about 3.4 MiB, held by every GPU
 * that loads the library until the process exits).  The paper has no
 * counterpart; this is a deployment convenience.
 * Arguments as for rexi_plan_create (constant depth H, parameter h) and
 * rexi_step (all terms, fused FP64 form).  Limits: 2 <= nx, ny <= 1024,
 * nx * ny <= 65536, prime factors <= 127, at most 8193 scalar terms
 * (dt * rho up to about 2030 at h = 0.5, tol = 1e-10); larger requests return
 * REXI_EINVAL with the reason in rexi_last_error_message().
 * The first call on each device looks up the array's device address
 * (cudaGetSymbolAddress) and caches it for the life of the process; the
 * cache does not survive cudaDeviceReset, so make no call after one.  Each
 * call copies its tables from static pageable host buffers, which the next
 * call overwrites, so the entry point cannot be captured in a CUDA graph: a
 * call on a capturing stream returns REXI_EINVAL before any copy or launch.
 * All calls share the array: calls whose GPU work overlaps
 * (different streams, several host threads) race and give wrong results;
 * order them on one stream.  Every region is written before it is read, so
 * nothing needs clearing between calls. */
rexi_status rexi_step_noalloc(int32_t nx, int32_t ny, double Lx, double Ly, double g, double f, double H,
                              double h, const void* in_dev, void* out_dev, double dt, double tol,
                              int32_t real_input, void* stream);

/* ------------------------------------------------------------------------ */
/* Batched serving launch.                                                  */
/* ------------------------------------------------------------------------ */

/* Many independent constant-depth instances advanced together, each with its
 * own grid (nx[i] x ny[i]) and time step dt[i] (so its own pole count), with
 * shared Lx, Ly, g, f, H, tol, h and form (REXI_FORM_FP64 or REXI_FORM_MIXED).
 * Each instance computes exactly what rexi_step computes for it.
 * States are packed in one device buffer: instance i occupies
 * 3 * nx[i] * ny[i] complex128 values from element offsets[i]
 * (rexi_batch_layout); instances of equal size are packed next to each other.
 * rexi_batch_create allocates device tables (coefficients, work list). */
typedef struct rexi_batch_s* rexi_batch_t;

enum {
  REXI_BATCH_PERSISTENT = 0,  /* one persistent pole kernel over all instances, one combine launch, whole step
                                 replayed from a CUDA graph */
  REXI_BATCH_PER_INSTANCE = 1 /* FFT, pole and inverse-FFT launches instance by instance */
};

rexi_status rexi_batch_create(rexi_batch_t* batch, int32_t n, const int32_t* nx, const int32_t* ny,
                              const double* dt, double Lx, double Ly, double g, double f, double H, double tol,
                              int32_t form, double h);
void rexi_batch_destroy(rexi_batch_t batch);

/* offsets: NULL or n + 1 entries (element offsets, last = total); M_out: NULL
 * or n pole counts; workspace_bytes: device workspace rexi_batch_step needs. */
rexi_status rexi_batch_layout(rexi_batch_t batch, int64_t* offsets, int32_t* M_out, size_t* workspace_bytes);

/* One step of every instance: out = r(dt_i A_i) in for each i.  The
 * persistent mode captures its launch sequence in a CUDA graph on the first
 * call for given buffers and replays it afterwards (on a stream owned by the
 * batch, ordered after `stream` and before later work on `stream` by events);
 * the buffers must not move between calls that should reuse the graph.
 * `in` and `out` may be the same buffer. */
rexi_status rexi_batch_step(rexi_batch_t batch, const void* in_dev, void* out_dev, int32_t real_input,
                            void* workspace_dev, size_t workspace_bytes, int32_t mode, void* stream);

/* Times the persistent mode for CTA sizes {64, 128, 256} x orbits per
 * thread {1, 2} on the given buffers (a few steps each; results are
 * overwritten) and keeps the fastest.  An orbit is the set of wavenumbers
 * (+-kx, +-ky), and (+-ky, +-kx) on square grids with equal spacing, which
 * share omega(k) and hence the pole sum.  Outputs (each nullable): the chosen
 * configuration and its time per step in milliseconds. */
rexi_status rexi_batch_autotune(rexi_batch_t batch, const void* in_dev, void* out_dev, int32_t real_input,
                                void* workspace_dev, size_t workspace_bytes, void* stream, int32_t* threads,
                                int32_t* orbits_per_thread, double* best_ms);

/* Current configuration and counters (each nullable): CTA size, orbits per
 * thread, persistent CTAs launched, work items, sum over instances of
 * wavenumber orbits x scalar terms (the pole-sum evaluations of one step),
 * kernels launched so far. */
rexi_status rexi_batch_info(rexi_batch_t batch, int32_t* threads, int32_t* orbits_per_thread, int32_t* ctas,
                            int32_t* n_items, int64_t* terms_orbits, int64_t* launches);

/* ------------------------------------------------------------------------ */
/* Measurement utility.                                                     */
/* ------------------------------------------------------------------------ */

/* Fused multiply-add throughput probe (no counterpart in the paper; it
 * measures the ALU rates that bound the pole-sum kernels).  kind 0: FP32,
 * kind 1: FP64, kind 2: packed FP32 (fma.rn.f32x2, two multiply-adds per
 * instruction).  Launches `blocks` blocks of 256 threads; every thread does
 * 256 * iters multiply-add instructions in 16 independent chains (2 flops per
 * instruction for kinds 0 and 1, 4 for kind 2, so 256 * blocks * 256 * iters
 * * 2 flops per call, twice that for kind 2).  out_dev: device memory for
 * blocks * 256 values of the kind's type, written only in an impossible
 * sentinel case.  Asynchronous on `stream`; the caller times it.  EINVAL on
 * a bad kind, blocks or iters < 1, or NULL out_dev. */
rexi_status rexi_alu_probe(int32_t kind, int32_t blocks, int32_t iters, void* out_dev, void* stream);

/* Human-readable name of a status code (static string). */
const char* rexi_status_string(rexi_status status);

/* Library version string (static). */
const char* rexi_version(void);

/* Text of the last error recorded by a failing call on this host thread
 * (static per-thread buffer; empty when the last call succeeded). */
const char* rexi_last_error_message(void);

#ifdef __cplusplus
}
#endif

#endif /* REXI_H */
