// C ABI of librexi (declared in include/rexi.h): argument checking, plans,
// workspace layout and the step driver for the Fourier path.
#include <math.h>
#include <stdarg.h>
#include <stdio.h>
#include <string.h>

#include <algorithm>
#include <vector>

#include "internal.h"
#include "krylov.h"

using namespace rexi;

namespace {

thread_local char g_err[512];

rexi_status fail(rexi_status st, const char* fmt, ...) {
  va_list ap;
  va_start(ap, fmt);
  vsnprintf(g_err, sizeof(g_err), fmt, ap);
  va_end(ap);
  return st;
}
rexi_status cuda_fail(cudaError_t e, const char* where) {
  return fail(REXI_ECUDA, "%s: %s", where, cudaGetErrorString(e));
}

#define CUDA_TRY(expr, where)                   \
  do {                                          \
    cudaError_t _e = (expr);                    \
    if (_e != cudaSuccess) return cuda_fail(_e, where); \
  } while (0)

size_t align_up(size_t v, size_t a) { return (v + a - 1) / a * a; }

}  // namespace

void rexi::set_last_error(const char* msg) {
  snprintf(g_err, sizeof(g_err), "%s", msg);
}

struct rexi_plan_s {
  int nx = 0, ny = 0;
  double Lx = 1, Ly = 1, g = 1, f = 1, H = 1, h = 0.5;
  const double* depth = nullptr;
  int form = REXI_FORM_FP64;
  double rho = 0.0;
  double rho_natural = 0.0;  // rho of the discretisation (rho may be overridden)
  int spectral = 0;  // symbol: 0 C grid, 1 spectral LRSW, 2 scalar i (d_xx + d_yy)
  int coef_set = REXI_COEF_REXII;
  GaussFit fit = table_fit();  // rational fit of the Gaussian (Table tab:coef_al unless replaced)
  bool fit_custom = false;
  int fit_gen = 0;             // bumped when the fit changes (coefficient-table cache key)
  int shift_mode = REXI_SHIFT_NONE;
  double shift_value = 0.0;  // sigma requested with REXI_SHIFT_VALUE
  double sigma = 0.0;        // sigma in effect (scalar operator only)
  double Hmax = 0.0, Hmean = 0.0;
  // Fourier path tables (device)
  FftPlan1D fx, fy;
  double2* tw_x = nullptr;
  double2* tw_y = nullptr;
  float4* twf_x = nullptr;  // double-float twiddles (mixed form)
  float4* twf_y = nullptr;
  // half-length x plan for real input (nx = 2 m even, m >= 2)
  FftPlan1D fxh;
  bool r2c = false;
  double2* tw_xh = nullptr;
  float4* twf_xh = nullptr;
  // half angles as double-float pairs (cos hi, cos lo, sin hi, sin lo) for
  // the double-float combine pass
  float4* halfdf_x = nullptr;
  float4* halfdf_y = nullptr;
  double2* half_x = nullptr;
  double2* half_y = nullptr;
  // device coefficient tables of the FP64 and mixed Fourier forms, one per
  // (form, M, term range, split grid); immutable once uploaded
  struct CoefTable {
    int M = 0, tb = 0, te = 0, nterms = 0, coef_set = 0, fit_gen = 0;
    int exact_hn = 1;  // mixed form: every h n of the table on the split grid G
    double G = 0.0, R0re = 0.0, R0im = 0.0;
    void* dev = nullptr;
    cudaEvent_t ready = nullptr;
    uint64_t last_use = 0;
  };
  std::vector<CoefTable> coef;
  uint64_t coef_clock = 0;
  // host-buffer steps: kernels of consecutive calls run in call order (each
  // waits for the previous call's kernels), their copies overlap
  cudaEvent_t host_kernels_done = nullptr;
  bool host_kernels_recorded = false;
  // coefficient staging (pinned host) guarded by an event
  void* staging = nullptr;
  size_t staging_bytes = 0;
  cudaEvent_t staging_done = nullptr;
  bool staging_pending = false;
  // Krylov path
  KrylovSettings kry;
  // profiling: per call 6 events (start, after upload, after forward, after
  // poles, end, and between the pole sum and the combine pass)
  bool prof_on = false;
  bool prof_mid = false;
  std::vector<std::vector<cudaEvent_t>> prof_pool;
  size_t prof_used = 0;
  int64_t launches = 0;
  int64_t prof_launch_base = 0;
};

namespace {
void prof_mark(rexi_plan_s* p, int i, cudaStream_t s) {
  if (!p->prof_on) return;
  if (i == 0) {
    if (p->prof_used == p->prof_pool.size()) {
      std::vector<cudaEvent_t> set(6, nullptr);
      for (auto& e : set) cudaEventCreate(&e);
      p->prof_pool.push_back(set);
    }
    ++p->prof_used;
    p->prof_mid = false;
  }
  if (i == 5) p->prof_mid = true;
  // paths without a separate combine pass: the combine phase is empty
  if (i == 3 && !p->prof_mid) cudaEventRecord(p->prof_pool[p->prof_used - 1][5], s);
  cudaEventRecord(p->prof_pool[p->prof_used - 1][i], s);
}
}  // namespace

extern "C" {

const char* rexi_status_string(rexi_status s) {
  switch (s) {
    case REXI_OK: return "REXI_OK";
    case REXI_EINVAL: return "REXI_EINVAL";
    case REXI_ENOMEM: return "REXI_ENOMEM";
    case REXI_ECUDA: return "REXI_ECUDA";
    case REXI_ENOCONV: return "REXI_ENOCONV";
    case REXI_ETIMEOUT: return "REXI_ETIMEOUT";
    case REXI_EUNSUPPORTED: return "REXI_EUNSUPPORTED";
  }
  return "REXI_UNKNOWN";
}

const char* rexi_version(void) { return "librexi 0.1 (sm_103a)"; }

const char* rexi_last_error_message(void) { return g_err; }

rexi_status rexi_pole_count(double tau_rho, double h, double tol, int32_t* M_out) {
  g_err[0] = 0;
  if (!M_out) return fail(REXI_EINVAL, "M_out is NULL");
  const int M = pole_count(tau_rho, h, tol);
  if (M < 0) return fail(REXI_EINVAL, "bad tau_rho/h/tol (%g, %g, %g)", tau_rho, h, tol);
  *M_out = M;
  return REXI_OK;
}

rexi_status rexi_rexii_terms(int32_t M, double h, double* mu_out, int32_t* n_terms, double* c1,
                             double* c2, int32_t cap) {
  g_err[0] = 0;
  if (M < 0 || M > 50000000 || !valid_h(h) || !n_terms) return fail(REXI_EINVAL, "bad M/h");
  const int N = M + kL;
  *n_terms = 2 * N + 1;
  if (mu_out) *mu_out = table_mu();
  if (!c1 && !c2) return REXI_OK;
  if (!c1 || !c2 || cap < 2 * N + 1) return fail(REXI_EINVAL, "arrays NULL or cap < 2N+1");
  TermSet ts;
  rexii_terms(M, h, &ts);
  for (int i = 0; i < 2 * N + 1; ++i) {
    c1[2 * i] = ts.c1re[i];
    c1[2 * i + 1] = ts.c1im[i];
    c2[2 * i] = ts.c2re[i];
    c2[2 * i + 1] = ts.c2im[i];
  }
  return REXI_OK;
}

rexi_status rexi_coeffs(double tau_rho, double tol, double h, int32_t real_input, int32_t* M_out,
                        int32_t* n_poles, double* poles, double* weights, int32_t cap) {
  g_err[0] = 0;
  if (!M_out || !n_poles) return fail(REXI_EINVAL, "M_out/n_poles NULL");
  const int M = pole_count(tau_rho, h, tol);
  if (M < 0) return fail(REXI_EINVAL, "bad tau_rho/h/tol");
  const int N = M + kL;
  const int J = real_input ? 2 * (N + 1) : 2 * (2 * N + 1);
  *M_out = M;
  *n_poles = J;
  if (!poles && !weights) return REXI_OK;
  if (!poles || !weights || cap < J) return fail(REXI_EINVAL, "arrays NULL or cap < J");
  TermSet ts;
  rexii_terms(M, h, &ts);
  const double hmu = h * ts.mu;
  int j = 0;
  for (int n = real_input ? 0 : -N; n <= N; ++n) {
    const double gam = (real_input && n > 0) ? 2.0 : 1.0;
    const int i = n + N;
    // C1 = c1 h mu + c2 h n, C2 = i c2, alpha_{+-n} = h (mu +- i n)
    const double C1r = ts.c1re[i] * hmu + ts.c2re[i] * h * n;
    const double C1i = ts.c1im[i] * hmu + ts.c2im[i] * h * n;
    const double C2r = -ts.c2im[i], C2i = ts.c2re[i];
    const double apr = hmu, api = h * n;    // alpha_n
    const double amr = hmu, ami = -h * n;   // alpha_{-n}
    const double inv2 = 1.0 / (2.0 * hmu);  // 1 / (alpha_n + alpha_{-n})
    // P = (C1 - C2 alpha_{-n}) / (2 h mu),  Q = (C1 + C2 alpha_n) / (2 h mu)
    const double Pr = (C1r - (C2r * amr - C2i * ami)) * inv2;
    const double Pi = (C1i - (C2r * ami + C2i * amr)) * inv2;
    const double Qr = (C1r + (C2r * apr - C2i * api)) * inv2;
    const double Qi = (C1i + (C2r * api + C2i * apr)) * inv2;
    // pole alpha_{-n}, weight -Gamma P;  pole -alpha_n, weight Gamma Q
    poles[2 * j] = amr;
    poles[2 * j + 1] = ami;
    weights[2 * j] = -gam * Pr;
    weights[2 * j + 1] = -gam * Pi;
    ++j;
    poles[2 * j] = -apr;
    poles[2 * j + 1] = -api;
    weights[2 * j] = gam * Qr;
    weights[2 * j + 1] = gam * Qi;
    ++j;
  }
  return REXI_OK;
}

void rexi_plan_destroy(rexi_plan_t p) {
  if (!p) return;
  if (p->staging_done) {
    cudaEventSynchronize(p->staging_done);
    cudaEventDestroy(p->staging_done);
  }
  cudaFree(p->tw_x);
  cudaFree(p->tw_y);
  cudaFree(p->twf_x);
  cudaFree(p->twf_y);
  cudaFree(p->tw_xh);
  cudaFree(p->twf_xh);
  cudaFree(p->halfdf_x);
  cudaFree(p->halfdf_y);
  cudaFree(p->half_x);
  cudaFree(p->half_y);
  if (p->staging) cudaFreeHost(p->staging);
  for (auto& c : p->coef) {
    cudaFree(c.dev);
    if (c.ready) cudaEventDestroy(c.ready);
  }
  if (p->host_kernels_done) cudaEventDestroy(p->host_kernels_done);
  krylov_destroy(&p->kry);
  for (auto& set : p->prof_pool)
    for (auto e : set) cudaEventDestroy(e);
  delete p;
}

static bool upload_table(const std::vector<double2>& host, double2** dev, rexi_status* st) {
  if (cudaMalloc(dev, host.size() * sizeof(double2)) != cudaSuccess) {
    *st = fail(REXI_ENOMEM, "cudaMalloc of a plan table failed");
    return false;
  }
  if (cudaMemcpy(*dev, host.data(), host.size() * sizeof(double2), cudaMemcpyHostToDevice) != cudaSuccess) {
    *st = fail(REXI_ECUDA, "upload of a plan table failed");
    return false;
  }
  return true;
}

rexi_status rexi_plan_create(rexi_plan_t* out, int32_t nx, int32_t ny, double Lx, double Ly, double g,
                             double f, double H, const double* depth, int32_t form, double h) {
  g_err[0] = 0;
  if (!out) return fail(REXI_EINVAL, "plan pointer NULL");
  *out = nullptr;
  if (!(Lx > 0 && Ly > 0 && g > 0 && isfinite(f) && isfinite(Lx) && isfinite(Ly) && isfinite(g)))
    return fail(REXI_EINVAL, "bad Lx/Ly/g/f");
  if (!valid_h(h)) return fail(REXI_EINVAL, "h must lie in (0, pi)");
  if (form != REXI_FORM_FP64 && form != REXI_FORM_MIXED && form != REXI_FORM_PLAIN)
    return fail(REXI_EINVAL, "unknown form %d", form);
  rexi_plan_s* p = new rexi_plan_s();
  p->nx = nx; p->ny = ny; p->Lx = Lx; p->Ly = Ly; p->g = g; p->f = f; p->H = H; p->h = h;
  p->depth = depth; p->form = form;
  rexi_status st = REXI_OK;
  const double dx = Lx / nx, dy = Ly / ny;
  if (!depth) {
    if (!(H > 0 && isfinite(H))) { delete p; return fail(REXI_EINVAL, "H_const must be > 0"); }
    if (!fft_factor(nx, &p->fx) || !fft_factor(ny, &p->fy)) {
      delete p;
      return fail(REXI_EINVAL, "grid %dx%d: need 2..4096 with prime factors <= %d", nx, ny, kMaxRadix);
    }
    // twiddles w[t] = exp(-2 pi i t / n) and half angles (cos(pi k/n), sin(pi k/n))
    auto make = [](int n, std::vector<double2>& tw, std::vector<double2>& half) {
      tw.resize(n);
      half.resize(n);
      for (int t = 0; t < n; ++t) {
        const double a = 2.0 * M_PI * (double)t / (double)n;
        tw[t] = make_double2(cos(a), -sin(a));
        const double b = M_PI * (double)t / (double)n;
        half[t] = make_double2(cos(b), sin(b));
      }
    };
    std::vector<double2> twx, hx, twy, hy;
    make(nx, twx, hx);
    make(ny, twy, hy);
    if (!upload_table(twx, &p->tw_x, &st) || !upload_table(twy, &p->tw_y, &st) ||
        !upload_table(hx, &p->half_x, &st) || !upload_table(hy, &p->half_y, &st)) {
      rexi_plan_destroy(p);
      return st;
    }
    p->fx.tw = p->tw_x;
    p->fy.tw = p->tw_y;
    {  // double-float twiddles for the mixed form's transforms
      std::vector<double2> fx4(2 * nx), fy4(2 * ny);
      df_twiddles(twx.data(), p->fx, reinterpret_cast<float4*>(fx4.data()));
      df_twiddles(twy.data(), p->fy, reinterpret_cast<float4*>(fy4.data()));
      if (!upload_table(fx4, reinterpret_cast<double2**>(&p->twf_x), &st) ||
          !upload_table(fy4, reinterpret_cast<double2**>(&p->twf_y), &st)) {
        rexi_plan_destroy(p);
        return st;
      }
      p->fx.twf = p->twf_x;
      p->fy.twf = p->twf_y;
      std::vector<double2> hx4(nx), hy4(ny);
      split_twiddles(hx.data(), nx, reinterpret_cast<float4*>(hx4.data()));
      split_twiddles(hy.data(), ny, reinterpret_cast<float4*>(hy4.data()));
      if (!upload_table(hx4, reinterpret_cast<double2**>(&p->halfdf_x), &st) ||
          !upload_table(hy4, reinterpret_cast<double2**>(&p->halfdf_y), &st)) {
        rexi_plan_destroy(p);
        return st;
      }
    }
    if (nx % 2 == 0 && fft_factor(nx / 2, &p->fxh)) {  // real-input transforms along x
      const int m = nx / 2;
      std::vector<double2> twh(m), twh4(2 * m);
      for (int t = 0; t < m; ++t) {
        const double a = 2.0 * M_PI * (double)t / (double)m;
        twh[t] = make_double2(cos(a), -sin(a));
      }
      df_twiddles(twh.data(), p->fxh, reinterpret_cast<float4*>(twh4.data()));
      if (!upload_table(twh, &p->tw_xh, &st) || !upload_table(twh4, reinterpret_cast<double2**>(&p->twf_xh), &st)) {
        rexi_plan_destroy(p);
        return st;
      }
      p->fxh.tw = p->tw_xh;
      p->fxh.twf = p->twf_xh;
      p->r2c = true;
    }
    // rho(A): largest omega over the discrete wavenumbers (exact for constant depth)
    std::vector<double> sx2(nx), cx2(nx);
    for (int k = 0; k < nx; ++k) { sx2[k] = hx[k].y * hx[k].y; cx2[k] = hx[k].x * hx[k].x; }
    double best = 0.0;
    for (int ky = 0; ky < ny; ++ky) {
      const double sy2 = hy[ky].y * hy[ky].y, cy2 = hy[ky].x * hy[ky].x;
      const double wy = 4.0 * sy2 / (dy * dy);
      for (int kx = 0; kx < nx; ++kx) {
        const double w2 = g * H * (4.0 * sx2[kx] / (dx * dx) + wy) + f * f * cx2[kx] * cy2;
        best = std::max(best, w2);
      }
    }
    p->rho = sqrt(best);
    p->rho_natural = p->rho;
    p->Hmax = H;
    p->Hmean = H;
  } else {
    if (nx < 3 || ny < 3 || nx > 16384 || ny > 16384) {
      delete p;
      return fail(REXI_EINVAL, "variable-depth grid %dx%d outside 3..16384", nx, ny);
    }
    if (form == REXI_FORM_PLAIN) { delete p; return fail(REXI_EUNSUPPORTED, "plain form is Fourier-path only"); }
    std::vector<double> Hh((size_t)nx * ny);
    if (cudaMemcpy(Hh.data(), depth, Hh.size() * sizeof(double), cudaMemcpyDeviceToHost) != cudaSuccess) {
      delete p;
      return fail(REXI_EINVAL, "depth_dev is not readable device memory");
    }
    double hmax = 0.0, hsum = 0.0, hmin = 1e300;
    for (double v : Hh) { hmax = std::max(hmax, v); hmin = std::min(hmin, v); hsum += v; }
    if (!(hmin > 0.0) || !isfinite(hmax)) { delete p; return fail(REXI_EINVAL, "depth must be > 0 and finite"); }
    p->Hmax = hmax;
    p->Hmean = hsum / (double)Hh.size();
    p->rho = sqrt(g * hmax * (4.0 / (dx * dx) + 4.0 / (dy * dy))) + fabs(f);
    p->rho_natural = p->rho;
    st = krylov_init(&p->kry, nx, ny, Lx, Ly, g, f, depth, p->Hmean);
    if (st != REXI_OK) { rexi_plan_destroy(p); return st; }
    p->kry.rho_bound = p->rho_natural;
  }
  if (cudaEventCreateWithFlags(&p->staging_done, cudaEventDisableTiming) != cudaSuccess) {
    rexi_plan_destroy(p);
    return fail(REXI_ECUDA, "event creation failed");
  }
  *out = p;
  return REXI_OK;
}

rexi_status rexi_spectral_radius(rexi_plan_t p, double* rho) {
  g_err[0] = 0;
  if (!p || !rho) return fail(REXI_EINVAL, "NULL argument");
  *rho = p->rho;
  return REXI_OK;
}

rexi_status rexi_plan_set_krylov_method(rexi_plan_t p, int32_t method) {
  g_err[0] = 0;
  if (!p || (method != REXI_KRYLOV_CG && method != REXI_KRYLOV_SHARED)) return fail(REXI_EINVAL, "bad Krylov method");
  if (!p->depth) return fail(REXI_EUNSUPPORTED, "Krylov method needs a variable-depth plan");
  p->kry.method = method;
  return REXI_OK;
}

rexi_status rexi_plan_set_krylov(rexi_plan_t p, double rtol, int32_t max_iters, int32_t term_batch) {
  g_err[0] = 0;
  if (!p || !(rtol > 0.0 && rtol < 1.0) || max_iters < 1 || term_batch < 1)
    return fail(REXI_EINVAL, "bad Krylov settings");
  p->kry.rtol = rtol;
  p->kry.max_iters = max_iters;
  p->kry.term_batch = term_batch;
  return REXI_OK;
}

}  // extern "C"

// ---------------------------------------------------------------------------
// Workspace layout (Fourier path), every region 256-byte aligned:
//   [table][spectrum 3 nx ny double2][plain form: accumulator + chunk of terms]
namespace {

struct FourierLayout {
  int M, N, nterms_scalar, nterms_plain, slice_cap;
  size_t table_off, table_bytes, spec_off, acc_off, chunk_off, chunk_terms, part_off, fin_off, total;
};

SymbolParams symbol_params(const rexi_plan_s* p);

constexpr size_t kPlainChunkBudget = size_t(8) << 30;  // bytes of materialised terms per chunk

FourierLayout fourier_layout(const rexi_plan_s* p, int M, int real_input) {
  FourierLayout L{};
  L.M = M;
  L.N = M + kL;
  L.nterms_scalar = 2 * L.N + 1;
  L.nterms_plain = real_input ? L.N + 1 : 2 * L.N + 1;
  const size_t nk3 = 3 * (size_t)p->nx * p->ny;
  size_t tb = 0;  // the FP64 and mixed forms keep their tables in the plan
  if (p->form == REXI_FORM_PLAIN) tb = (size_t)L.nterms_plain * 4 * sizeof(double2);
  L.table_off = 0;
  L.table_bytes = tb;
  L.spec_off = align_up(tb, 256);
  size_t end = L.spec_off + align_up(nk3 * sizeof(double2), 256);
  L.acc_off = end;
  L.chunk_off = end;
  L.chunk_terms = 0;
  L.part_off = end;
  L.fin_off = end;
  L.slice_cap = 0;
  if (p->form != REXI_FORM_PLAIN) {
    // per-orbit partial sums of the pole loop, one row per term slice, then
    // the per-orbit combine scalars
    const OrbitParams op = orbit_params(symbol_params(p));
    L.slice_cap = orbit_slice_cap(op.norb);
    end += align_up((size_t)L.slice_cap * op.norb * sizeof(double2), 256);
    L.fin_off = end;
    end += align_up(orbit_scalars_bytes(op.norb), 256);
  }
  if (p->form == REXI_FORM_PLAIN) {
    L.acc_off = end;
    end += align_up(nk3 * sizeof(double2), 256);
    L.chunk_off = end;
    size_t per = nk3 * sizeof(double2);
    size_t ct = std::max<size_t>(1, kPlainChunkBudget / per);
    ct = std::min<size_t>(ct, (size_t)L.nterms_plain);
    ct = std::min<size_t>(ct, 65535);
    L.chunk_terms = ct;
    end += align_up(ct * per, 256);
  }
  L.total = end;
  return L;
}

rexi_status check_step_args(rexi_plan_s* p, const void* in, void* out, double dt, double tol,
                            void* ws, int* M) {
  if (!p) return fail(REXI_EINVAL, "plan NULL");
  if (!in || !out || !ws) return fail(REXI_EINVAL, "NULL buffer");
  if (((uintptr_t)in | (uintptr_t)out) & 15) return fail(REXI_EINVAL, "state buffers must be 16-byte aligned");
  if ((uintptr_t)ws & 255) return fail(REXI_EINVAL, "workspace must be 256-byte aligned");
  if (!(dt >= 0.0) || !isfinite(dt)) return fail(REXI_EINVAL, "dt must be finite and >= 0");
  *M = pole_count(dt * p->rho, p->h, tol);
  if (*M < 0) return fail(REXI_EINVAL, "pole count rule rejected dt*rho=%g h=%g tol=%g", dt * p->rho, p->h, tol);
  return REXI_OK;
}

rexi_status stage_upload(rexi_plan_s* p, const void* src, size_t bytes, void* dst, cudaStream_t s) {
  if (p->staging_pending) {
    CUDA_TRY(cudaEventSynchronize(p->staging_done), "staging wait");
    p->staging_pending = false;
  }
  if (bytes > p->staging_bytes) {
    if (p->staging) cudaFreeHost(p->staging);
    p->staging = nullptr;
    p->staging_bytes = 0;
    size_t nb = std::max<size_t>(bytes, 1 << 16);
    if (cudaHostAlloc(&p->staging, nb, cudaHostAllocDefault) != cudaSuccess)
      return fail(REXI_ENOMEM, "pinned staging allocation failed");
    p->staging_bytes = nb;
  }
  memcpy(p->staging, src, bytes);
  CUDA_TRY(cudaMemcpyAsync(dst, p->staging, bytes, cudaMemcpyHostToDevice, s), "table upload");
  CUDA_TRY(cudaEventRecord(p->staging_done, s), "staging event");
  p->staging_pending = true;
  return REXI_OK;
}

SymbolParams symbol_params(const rexi_plan_s* p) {
  SymbolParams sp;
  sp.nx = p->nx;
  sp.ny = p->ny;
  sp.inv_dx = p->nx / p->Lx;
  sp.inv_dy = p->ny / p->Ly;
  sp.g = p->g;
  sp.f = p->f;
  sp.H = p->H;
  sp.half_x = p->half_x;
  sp.half_y = p->half_y;
  sp.spectral = p->spectral;
  sp.shift = p->sigma;
  return sp;
}

bool term_selected(int n, int tb, int te) {
  const int a = n < 0 ? -n : n;
  return a >= tb && a < te;
}

// The scalar-term table of the FP64 (G = 0) or mixed form for M and the
// term range [tb, te): found in the plan's cache or built on the host and
// uploaded on stream s.  A table is never rewritten, so calls on other streams
// only wait for its upload.  At most kCoefTables are kept; evicting one waits
// for the device to go idle (it may still be read).
constexpr size_t kCoefTables = 8;

rexi_status fused_table(rexi_plan_s* p, int M, int tb, int te, double G, cudaStream_t s,
                        const rexi_plan_s::CoefTable** out) {
  for (auto& c : p->coef) {
    if (c.M == M && c.tb == tb && c.te == te && c.G == G && c.coef_set == p->coef_set && c.fit_gen == p->fit_gen) {
      c.last_use = ++p->coef_clock;
      // an upload still in flight (on another stream): order this stream after
      // it; a finished one needs no wait (and none is recorded, so a step can be
      // captured in a graph once its table exists)
      if (cudaEventQuery(c.ready) == cudaErrorNotReady) {
        if (cudaPeekAtLastError() == cudaErrorNotReady) cudaGetLastError();  // a status, not an error
        CUDA_TRY(cudaStreamWaitEvent(s, c.ready, 0), "table wait");
      }
      *out = &c;
      return REXI_OK;
    }
  }
  TermSet ts;
  rexii_terms_fit(M, p->h, p->fit, &ts);
  const int N = ts.N;
  const double h = p->h, hmu = h * ts.mu, q = hmu * hmu;
  // scalar terms n = -N..N restricted to |n| in [tb, te)
  std::vector<int> sel;
  for (int n = -N; n <= N; ++n)
    if (term_selected(n, tb, te)) sel.push_back(n);
  rexi_plan_s::CoefTable c;
  c.M = M;
  c.tb = tb;
  c.te = te;
  c.G = G;
  c.coef_set = p->coef_set;
  c.fit_gen = p->fit_gen;
  c.nterms = (int)sel.size();
  // Every scalar term is (A_n + B_n y) / ((h mu)^2 + y^2), y = x + h n.
  // REXII (eq. modifiedRexi): A = c1 h mu, B = c2.
  // REXIE (eq. REXIE) on a scalar operator i B with B real: per eigenvalue it
  //   is eq. originalRexi, Re(beta^Re / (ix + alpha_n)) + i Re(beta^Im / (ix + alpha_n)),
  //   whose A = h mu (Re beta^Re + i Re beta^Im), B = Im beta^Re + i Im beta^Im;
  //   with beta^Re = Re c1 + i Re c2 and beta^Im = Im c1 + i Im c2 (both are
  //   h sum a_k b_{n-k} split by parts) these are again c1 h mu and c2.
  // Original REXI, eq. originalREXImatrix, for a real operator and real data:
  //   Re(beta (tau A + alpha_n)^{-1}) = (beta (tau A + alpha_n)^{-1}
  //   + conj(beta) (tau A + alpha_{-n})^{-1}) / 2, so the scalar function is
  //   sum_n gamma_n / (z + alpha_n), gamma_n = (beta^Re_n + conj(beta^Re_{-n})) / 2,
  //   i.e. A = gamma h mu, B = -i gamma at z = ix.
  std::vector<double> Are(2 * N + 1), Aim(2 * N + 1), Bre(2 * N + 1), Bim(2 * N + 1);
  for (int n = -N; n <= N; ++n) {
    const int i = n + N, j = -n + N;
    if (p->coef_set == REXI_COEF_REXI) {
      const double gr = 0.5 * (ts.c1re[i] + ts.c1re[j]), gi = 0.5 * (ts.c2re[i] - ts.c2re[j]);
      Are[i] = gr * hmu;
      Aim[i] = gi * hmu;
      Bre[i] = gi;
      Bim[i] = -gr;
    } else {
      Are[i] = ts.c1re[i] * hmu;
      Aim[i] = ts.c1im[i] * hmu;
      Bre[i] = ts.c2re[i];
      Bim[i] = ts.c2im[i];
    }
  }
  for (int n : sel) {
    const int i = n + N;
    const double hn = h * n, d = q + hn * hn;
    c.R0re += (Are[i] + Bre[i] * hn) / d;
    c.R0im += (Aim[i] + Bim[i] * hn) / d;
  }
  // 48 bytes per term in both forms
  std::vector<double> tab(6 * std::max<size_t>(sel.size(), 1), 0.0);
  if (G == 0.0) {  // FP64: h n, A_re, A_im, B_re, B_im, 0 with A = c1 h mu, B = c2
    for (size_t t = 0; t < sel.size(); ++t) {
      const int n = sel[t], i = n + N;
      double* e = &tab[6 * t];
      e[0] = h * n;
      e[1] = Are[i];
      e[2] = Aim[i];
      e[3] = Bre[i];
      e[4] = Bim[i];
      e[5] = 0.0;
    }
  } else {  // double-float: see pole_orbit_mixed_kernel
    auto split = [](double v, float& hi, float& lo) {
      hi = (float)v;
      lo = (float)(v - (double)hi);
    };
    float* tf = reinterpret_cast<float*>(tab.data());
    for (size_t t = 0; t < sel.size(); ++t) {
      const int n = sel[t], i = n + N;
      float* e = tf + 12 * t;
      const double hn = h * n;
      const double hn_g = rint(hn / G) * G;
      float Arh, Arl, Aih, Ail, Brh, Brl, Bih, Bil;
      split(Are[i], Arh, Arl);
      split(Aim[i], Aih, Ail);
      split(Bre[i], Brh, Brl);
      split(Bim[i], Bih, Bil);
      e[0] = (float)hn_g; e[1] = Arh; e[2] = Aih; e[3] = Brh;
      e[4] = Bih; e[5] = Arl; e[6] = Ail; e[7] = Brl;
      e[8] = Bil; e[9] = (float)(hn - hn_g); e[10] = (float)((hn - hn_g) - (double)e[9]); e[11] = 0.f;
      if (hn != hn_g) c.exact_hn = 0;
    }
  }
  if (p->coef.size() >= kCoefTables) {
    auto lru = std::min_element(p->coef.begin(), p->coef.end(),
                                [](const rexi_plan_s::CoefTable& a, const rexi_plan_s::CoefTable& b) {
                                  return a.last_use < b.last_use;
                                });
    CUDA_TRY(cudaDeviceSynchronize(), "table eviction");
    cudaFree(lru->dev);
    cudaEventDestroy(lru->ready);
    p->coef.erase(lru);
  }
  const size_t bytes = tab.size() * sizeof(double);
  if (cudaMalloc(&c.dev, bytes) != cudaSuccess) return fail(REXI_ENOMEM, "coefficient table allocation failed");
  if (cudaEventCreateWithFlags(&c.ready, cudaEventDisableTiming) != cudaSuccess) {
    cudaFree(c.dev);
    return fail(REXI_ECUDA, "event creation failed");
  }
  rexi_status st = stage_upload(p, tab.data(), bytes, c.dev, s);
  if (st == REXI_OK && cudaEventRecord(c.ready, s) != cudaSuccess) st = fail(REXI_ECUDA, "table event");
  if (st != REXI_OK) {
    cudaStreamSynchronize(s);
    cudaFree(c.dev);
    cudaEventDestroy(c.ready);
    return st;
  }
  c.last_use = ++p->coef_clock;
  p->coef.push_back(c);
  *out = &p->coef.back();
  return REXI_OK;
}

rexi_status fourier_step(rexi_plan_s* p, const void* in, void* out, double dt, int M, int real_input,
                         int tb, int te, void* ws, size_t ws_bytes, cudaStream_t s, bool adjoint) {
  const FourierLayout L = fourier_layout(p, M, real_input);
  if (ws_bytes < L.total) return fail(REXI_ENOMEM, "workspace %zu < %zu bytes", ws_bytes, L.total);
  char* base = static_cast<char*>(ws);
  double2* spec = reinterpret_cast<double2*>(base + L.spec_off);
  const int N = L.N;
  if (te < 0 || te > N + 1) te = N + 1;
  if (tb < 0 || tb > te) return fail(REXI_EINVAL, "bad term range [%d, %d)", tb, te);
  if (p->spectral == 2) {
    if (real_input) return fail(REXI_EINVAL, "the scalar operator i(d_xx + d_yy) needs complex input (real_input = 0)");
    if (p->form == REXI_FORM_PLAIN) return fail(REXI_EUNSUPPORTED, "plain form: shallow-water symbols only");
    if (p->coef_set == REXI_COEF_REXI)
      return fail(REXI_EUNSUPPORTED, "original REXI (eq. originalREXImatrix) needs a real operator");
  } else {
    if (p->coef_set == REXI_COEF_REXIE)
      return fail(REXI_EUNSUPPORTED, "REXIE (eq. REXIE) needs an operator i B with B real (the scalar symbol)");
    if (p->coef_set != REXI_COEF_REXII && p->form == REXI_FORM_PLAIN)
      return fail(REXI_EUNSUPPORTED, "plain form: REXII coefficients only");
  }
  const double h = p->h, hmu = h * p->fit.mu, q = hmu * hmu;
  const double tau = dt;
  const SymbolParams sp = symbol_params(p);
  const size_t nk = (size_t)p->nx * p->ny;
  rexi_status st;

  // real input on the C-grid: half spectrum (kx = 0..nx/2) through real
  // transforms along x; the pole step there is the Hermitian part of the
  // full-spectrum step (the real part the full path takes at the end)
  const bool half = real_input && p->r2c && !p->spectral && p->form != REXI_FORM_PLAIN;
  // mixed form on the half spectrum: the spectrum stays in double-float from
  // the forward transform through the combine pass to the inverse transform
  const bool df_spec = half && p->form == REXI_FORM_MIXED && fft_df_ready(p->fx, p->fxh, p->fy);
  const int df = p->form == REXI_FORM_MIXED ? (df_spec ? 2 : 1) : 0;
  prof_mark(p, 0, s);
  const double2* in2 = static_cast<const double2*>(in);
  auto forward = [&]() -> rexi_status {
    prof_mark(p, 1, s);
    // forward transform (imaginary parts dropped for real input)
    CUDA_TRY(half ? fft2d_r2c(in2, spec, 3, p->fx, p->fxh, p->fy, df, s)
             : df ? fft2d_df(in2, spec, 3, p->fx, p->fy, -1, 1.0, real_input, 0, s)
                  : fft2d(in2, spec, 3, p->fx, p->fy, -1, 1.0, real_input, 0, s),
             "forward FFT");
    p->launches += 2;
    prof_mark(p, 2, s);
    return REXI_OK;
  };

  if (p->form == REXI_FORM_FP64 || p->form == REXI_FORM_MIXED) {
    double G = 0.0;
    if (p->form == REXI_FORM_MIXED) {
      // grid G = 2^-g so that |x| + h N < 2^24 G for every x the pole kernel
      // evaluates: all wavenumbers of the grid, so x <= tau max(rho, rho of the
      // discretisation) (an override of rho below the grid's own can only
      // shrink the pole count, not the range of x)
      const double span = dt * std::max(p->rho, p->rho_natural) + h * N + 4.0;
      if (span > 4.0e6) return fail(REXI_EINVAL, "mixed form needs dt*rho + h*N < 4e6 (got %g)", span);
      int gexp = 0;
      while (ldexp(1.0, 23 - gexp) > span && gexp < 60) ++gexp;  // largest g with span < 2^(23-g)
      G = ldexp(1.0, -(gexp - 1));
    }
    const rexi_plan_s::CoefTable* ct = nullptr;
    if ((st = fused_table(p, M, tb, te, G, s, &ct)) != REXI_OK) return st;
    FusedScalars fs;
    fs.tau = tau;
    fs.q = q;
    fs.R0re = ct->R0re;
    fs.R0im = ct->R0im;
    fs.nterms = ct->nterms;
    fs.adjoint = adjoint ? 1 : 0;
    fs.exact_hn = ct->exact_hn;
    // With the real part of the step taken (real input), r(0) enters through
    // its real part: Re r(tau B) = Re(R0) I + Im(R+) Bt + (Re R0 - Re R+) Bt^2
    // on the C-grid, where B(-k) = conj B(k).
    if (half) fs.R0im = 0.0;
    const int row_len = half ? p->nx / 2 + 1 : p->nx;
    const OrbitParams op = orbit_params(sp);
    const int slices = pole_orbit_slices(p->form, op.norb, fs.nterms, L.slice_cap);
    double2* part = reinterpret_cast<double2*>(base + L.part_off);
    if ((st = forward()) != REXI_OK) return st;
    if (p->form == REXI_FORM_FP64)
      CUDA_TRY(pole_orbits_fp64(part, slices, sp, op, static_cast<const double*>(ct->dev), fs, s),
               "pole_orbits_fp64");
    else
      CUDA_TRY(pole_orbits_mixed(part, slices, sp, op, static_cast<const float*>(ct->dev), fs, G, s),
               "pole_orbits_mixed");
    prof_mark(p, 5, s);
    if (p->spectral == 2) {
      // e^{tau A} = e^{i tau sigma} e^{tau (A - i sigma I)}
      const double2 phase = make_double2(cos(tau * p->sigma), sin(tau * p->sigma));
      CUDA_TRY(pole_orbit_combine_scalar(spec, part, slices, sp, op, phase, adjoint ? 1 : 0, s),
               "pole_orbit_combine_scalar");
    } else if (p->form == REXI_FORM_MIXED && !half && !p->spectral) {
      // complex input (or real input without the half-length transform): the
      // combine in double-float arithmetic on the FP64 spectrum
      CUDA_TRY(pole_orbit_combine_dfc(spec, part, slices, base + L.fin_off, sp, p->halfdf_x, p->halfdf_y, op, fs,
                                      s),
               "pole_orbit_combine_dfc");
    } else if (df_spec)
      CUDA_TRY(pole_orbit_combine_df(spec, part, slices, base + L.fin_off, sp, p->halfdf_x, p->halfdf_y, op, fs,
                                     row_len, s),
               "pole_orbit_combine_df");
    else
      CUDA_TRY(pole_orbit_combine(spec, part, slices, base + L.fin_off, sp, op, fs, row_len, s),
               "pole_orbit_combine");
    p->launches += 3;
  } else {
    // plain form: terms n = 0..N (real) or -N..N (complex), |n| in [tb, te)
    TermSet ts;
    rexii_terms_fit(M, p->h, p->fit, &ts);
    std::vector<double2> tab;
    for (int n = real_input ? 0 : -N; n <= N; ++n) {
      if (!term_selected(n, tb, te)) continue;
      const int i = n + N;
      const double gam = (real_input && n > 0) ? 2.0 : 1.0;
      const double C1r = ts.c1re[i] * hmu + ts.c2re[i] * h * n;
      const double C1i = ts.c1im[i] * hmu + ts.c2im[i] * h * n;
      const double C2r = -ts.c2im[i], C2i = ts.c2re[i];
      const double amr = hmu, ami = -h * n;
      // K = C1 - C2 alpha_{-n}
      const double Kr = C1r - (C2r * amr - C2i * ami);
      const double Ki = C1i - (C2r * ami + C2i * amr);
      tab.push_back(make_double2(hmu, h * n));
      tab.push_back(make_double2(amr, ami));
      tab.push_back(make_double2(gam * C2r, gam * C2i));
      tab.push_back(make_double2(gam * Kr, gam * Ki));
    }
    const int nt = (int)(tab.size() / 4);
    double2* acc = reinterpret_cast<double2*>(base + L.acc_off);
    double2* chunk = reinterpret_cast<double2*>(base + L.chunk_off);
    if (nt == 0) {
      if ((st = forward()) != REXI_OK) return st;
      CUDA_TRY(cudaMemsetAsync(acc, 0, 3 * nk * sizeof(double2), s), "zero accumulator");
    } else {
      if ((st = stage_upload(p, tab.data(), tab.size() * sizeof(double2), base + L.table_off, s)) != REXI_OK) return st;
      if ((st = forward()) != REXI_OK) return st;
      const double2* dtab = reinterpret_cast<const double2*>(base + L.table_off);
      for (int t0 = 0; t0 < nt; t0 += (int)L.chunk_terms) {
        PlainScalars ps;
        ps.tau = tau;
        ps.nterms = std::min<int>((int)L.chunk_terms, nt - t0);
        ps.adjoint = adjoint ? 1 : 0;
        CUDA_TRY(pole_plain_terms(spec, chunk, sp, dtab + 4 * t0, ps, s), "pole_plain_terms");
        CUDA_TRY(pole_plain_reduce(chunk, acc, (long long)(3 * nk), ps.nterms, t0 == 0 ? 1 : 0, s),
                 "pole_plain_reduce");
        p->launches += 2;
      }
    }
    spec = acc;
  }
  prof_mark(p, 3, s);
  // inverse transform, 1/(nx ny), real part for real input
  CUDA_TRY(half ? fft2d_c2r(spec, static_cast<double2*>(out), 3, p->fx, p->fxh, p->fy, 1.0 / (double)nk, df, s)
           : df ? fft2d_df(spec, static_cast<double2*>(out), 3, p->fx, p->fy, +1, 1.0 / (double)nk, 0, real_input, s)
                : fft2d(spec, static_cast<double2*>(out), 3, p->fx, p->fy, +1, 1.0 / (double)nk, 0, real_input, s),
           "inverse FFT");
  p->launches += 2;
  prof_mark(p, 4, s);
  return REXI_OK;
}

void fill_info(const rexi_plan_s* p, int M, int real_input, double dt, rexi_step_info* info) {
  if (!info) return;
  memset(info, 0, sizeof(*info));
  info->M = M;
  info->N = M + kL;
  info->n_terms = real_input ? info->N + 1 : 2 * info->N + 1;
  info->n_poles = real_input ? 2 * (info->N + 1) : 2 * (2 * info->N + 1);
  info->tau_rho = dt * p->rho;
  info->rho = p->rho;
}

}  // namespace

extern "C" {

rexi_status rexi_workspace_size(rexi_plan_t p, double dt, double tol, int32_t real_input, size_t* bytes) {
  g_err[0] = 0;
  if (!p || !bytes) return fail(REXI_EINVAL, "NULL argument");
  if (!(dt >= 0.0) || !isfinite(dt)) return fail(REXI_EINVAL, "dt must be finite and >= 0");
  const int M = pole_count(dt * p->rho, p->h, tol);
  if (M < 0) return fail(REXI_EINVAL, "pole count rule rejected the arguments");
  if (p->depth) {
    *bytes = krylov_workspace_bytes(&p->kry, M, real_input, p->form);
  } else {
    *bytes = fourier_layout(p, M, real_input).total;
  }
  return REXI_OK;
}

rexi_status rexi_workspace_size_grad_depth(rexi_plan_t p, double dt, double tol, int32_t real_input, size_t* bytes) {
  g_err[0] = 0;
  if (!p || !bytes) return fail(REXI_EINVAL, "NULL argument");
  if (!p->depth) return fail(REXI_EUNSUPPORTED, "depth gradient needs a variable-depth plan");
  if (!(dt >= 0.0) || !isfinite(dt)) return fail(REXI_EINVAL, "dt must be finite and >= 0");
  const int M = pole_count(dt * p->rho, p->h, tol);
  if (M < 0) return fail(REXI_EINVAL, "pole count rule rejected the arguments");
  *bytes = krylov_grad_workspace_bytes(&p->kry, M, real_input, p->form, p->h);
  return REXI_OK;
}

rexi_status rexi_step(rexi_plan_t p, const void* in, void* out, double dt, double tol, int32_t real_input,
                      int32_t term_begin, int32_t term_end, void* ws, size_t ws_bytes, void* stream,
                      rexi_step_info* info) {
  g_err[0] = 0;
  int M = 0;
  rexi_status st = check_step_args(p, in, out, dt, tol, ws, &M);
  if (st != REXI_OK) return st;
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  if (p->depth && (p->coef_set != REXI_COEF_REXII || p->fit_custom))
    return fail(REXI_EUNSUPPORTED, "the variable-depth path uses REXII with Table tab:coef_al only");
  if (p->depth) {
    KrylovHooks hooks;
    hooks.mark = [](void* ctx, int i, cudaStream_t st) { prof_mark(static_cast<rexi_plan_s*>(ctx), i, st); };
    hooks.ctx = p;
    hooks.launches = &p->launches;
    st = krylov_step(&p->kry, p->form, p->h, M, in, out, dt, real_input, term_begin, term_end, ws, ws_bytes,
                     s, info, false, hooks);
    if (info) { info->M = M; info->N = M + kL; info->tau_rho = dt * p->rho; info->rho = p->rho; }
    return st;
  }
  st = fourier_step(p, in, out, dt, M, real_input, term_begin, term_end, ws, ws_bytes, s, false);
  if (st == REXI_OK) fill_info(p, M, real_input, dt, info);
  return st;
}

rexi_status rexi_step_adjoint(rexi_plan_t p, const void* gout, void* gin, double dt, double tol,
                              int32_t real_input, void* ws, size_t ws_bytes, void* stream) {
  g_err[0] = 0;
  int M = 0;
  rexi_status st = check_step_args(p, gout, gin, dt, tol, ws, &M);
  if (st != REXI_OK) return st;
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  if (p->depth && (p->coef_set != REXI_COEF_REXII || p->fit_custom))
    return fail(REXI_EUNSUPPORTED, "the variable-depth path uses REXII with Table tab:coef_al only");
  if (p->depth)
    return krylov_step(&p->kry, p->form, p->h, M, gout, gin, dt, real_input, 0, -1, ws, ws_bytes, s, nullptr,
                       true, KrylovHooks());
  return fourier_step(p, gout, gin, dt, M, real_input, 0, -1, ws, ws_bytes, s, true);
}

}  // extern "C"

extern "C" {

rexi_status rexi_workspace_size_host(rexi_plan_t p, double dt, double tol, int32_t real_input, size_t* bytes) {
  size_t b = 0;
  rexi_status st = rexi_workspace_size(p, dt, tol, real_input, &b);
  if (st != REXI_OK) return st;
  const size_t state = align_up(3 * (size_t)p->nx * p->ny * sizeof(double2), 256);
  *bytes = 2 * state + b;
  return REXI_OK;
}

namespace {
rexi_status step_host_enqueue(rexi_plan_t p, const void* in_host, void* out_host, double dt, double tol,
                              int32_t real_input, void* ws, size_t ws_bytes, void* stream, rexi_step_info* info) {
  if (!p || !in_host || !out_host || !ws) return fail(REXI_EINVAL, "NULL argument");
  if ((uintptr_t)ws & 255) return fail(REXI_EINVAL, "workspace must be 256-byte aligned");
  const size_t bytes = 3 * (size_t)p->nx * p->ny * sizeof(double2);
  const size_t state = align_up(bytes, 256);
  if (ws_bytes < 2 * state) return fail(REXI_ENOMEM, "workspace too small for the host-buffer step");
  char* base = static_cast<char*>(ws);
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  if (!p->host_kernels_done)
    CUDA_TRY(cudaEventCreateWithFlags(&p->host_kernels_done, cudaEventDisableTiming), "event creation");
  CUDA_TRY(cudaMemcpyAsync(base, in_host, bytes, cudaMemcpyHostToDevice, s), "host-to-device copy");
  // the kernels of the previous host-buffer step of this plan (on any stream)
  // first: concurrent steps would finish together and leave the copy engines
  // and the SMs idle in turn
  if (p->host_kernels_recorded) CUDA_TRY(cudaStreamWaitEvent(s, p->host_kernels_done, 0), "kernel order");
  rexi_status st = rexi_step(p, base, base + state, dt, tol, real_input, 0, -1, base + 2 * state,
                             ws_bytes - 2 * state, stream, info);
  if (st != REXI_OK) return st;
  CUDA_TRY(cudaEventRecord(p->host_kernels_done, s), "kernel order");
  p->host_kernels_recorded = true;
  CUDA_TRY(cudaMemcpyAsync(out_host, base + state, bytes, cudaMemcpyDeviceToHost, s), "device-to-host copy");
  return REXI_OK;
}
}  // namespace

rexi_status rexi_step_host(rexi_plan_t p, const void* in_host, void* out_host, double dt, double tol,
                           int32_t real_input, void* ws, size_t ws_bytes, void* stream, rexi_step_info* info) {
  g_err[0] = 0;
  rexi_status st = step_host_enqueue(p, in_host, out_host, dt, tol, real_input, ws, ws_bytes, stream, info);
  if (st != REXI_OK) return st;
  CUDA_TRY(cudaStreamSynchronize(static_cast<cudaStream_t>(stream)), "stream synchronise");
  return REXI_OK;
}

rexi_status rexi_step_host_async(rexi_plan_t p, const void* in_host, void* out_host, double dt, double tol,
                                 int32_t real_input, void* ws, size_t ws_bytes, void* stream) {
  g_err[0] = 0;
  return step_host_enqueue(p, in_host, out_host, dt, tol, real_input, ws, ws_bytes, stream, nullptr);
}

rexi_status rexi_plan_set_profiling(rexi_plan_t p, int32_t enable) {
  g_err[0] = 0;
  if (!p) return fail(REXI_EINVAL, "plan NULL");
  p->prof_on = enable != 0;
  p->prof_used = 0;
  p->prof_launch_base = p->launches;
  return REXI_OK;
}

rexi_status rexi_plan_read_profile(rexi_plan_t p, double* ms5, int32_t* n_calls, int64_t* n_launches) {
  g_err[0] = 0;
  if (!p || !ms5) return fail(REXI_EINVAL, "NULL argument");
  for (int i = 0; i < 5; ++i) ms5[i] = 0.0;
  for (size_t k = 0; k < p->prof_used; ++k) {
    auto& e = p->prof_pool[k];
    CUDA_TRY(cudaEventSynchronize(e[4]), "profile event");
    float t;
    const int map[5][2] = {{1, 2}, {2, 3}, {3, 4}, {0, 1}, {5, 3}};
    for (int ph = 0; ph < 5; ++ph) {
      CUDA_TRY(cudaEventElapsedTime(&t, e[map[ph][0]], e[map[ph][1]]), "profile elapsed");
      ms5[ph] += t;
    }
  }
  if (n_calls) *n_calls = (int32_t)p->prof_used;
  if (n_launches) *n_launches = p->launches - p->prof_launch_base;
  p->prof_used = 0;
  p->prof_launch_base = p->launches;
  return REXI_OK;
}

}  // extern "C"

extern "C" rexi_status rexi_step_grad_depth(rexi_plan_t p, const void* in, const void* gout, double* grad_depth,
                                           double dt, double tol, int32_t real_input, void* ws, size_t ws_bytes,
                                           void* stream, rexi_step_info* info) {
  g_err[0] = 0;
  int M = 0;
  rexi_status st = check_step_args(p, in, const_cast<void*>(gout), dt, tol, ws, &M);
  if (st != REXI_OK) return st;
  if (!p->depth) return fail(REXI_EUNSUPPORTED, "depth gradient needs a variable-depth plan");
  if (!grad_depth || ((uintptr_t)grad_depth & 7)) return fail(REXI_EINVAL, "grad_depth must be 8-byte aligned");
  KrylovHooks hooks;
  hooks.mark = [](void* ctx, int i, cudaStream_t s) { prof_mark(static_cast<rexi_plan_s*>(ctx), i, s); };
  hooks.ctx = p;
  hooks.launches = &p->launches;
  st = krylov_grad_depth(&p->kry, p->form, p->h, M, in, gout, grad_depth, dt, real_input, ws, ws_bytes,
                         static_cast<cudaStream_t>(stream), info, hooks);
  if (info) {
    info->M = M;
    info->tau_rho = dt * p->rho;
    info->rho = p->rho;
  }
  return st;
}

namespace {
// rho of the constant-depth symbol in use: the largest |eigenvalue| over the
// discrete wavenumbers (for the scalar operator, of the shifted operator
// A - i sigma I, sigma from the plan's shift mode); resets any override.
void update_rho(rexi_plan_s* p) {
  double best = 0.0, lmin = 0.0, lmax = -1e300;
  const double dx = p->Lx / p->nx, dy = p->Ly / p->ny;
  for (int ky = 0; ky < p->ny; ++ky) {
    for (int kx = 0; kx < p->nx; ++kx) {
      if (p->spectral == 2) {
        const double sx = sin(M_PI * kx / p->nx), sy = sin(M_PI * ky / p->ny);
        const double lam = -(4.0 * sx * sx / (dx * dx) + 4.0 * sy * sy / (dy * dy));
        lmin = std::min(lmin, lam);
        lmax = std::max(lmax, lam);
        continue;
      }
      double w2;
      if (p->spectral) {
        const int sx = 2 * kx <= p->nx ? kx : kx - p->nx, sy = 2 * ky <= p->ny ? ky : ky - p->ny;
        const double a = 2.0 * M_PI * sx / p->Lx, b = 2.0 * M_PI * sy / p->Ly;
        w2 = p->g * p->H * (a * a + b * b) + p->f * p->f;
      } else {
        const double sx = sin(M_PI * kx / p->nx), cx = cos(M_PI * kx / p->nx);
        const double sy = sin(M_PI * ky / p->ny), cy = cos(M_PI * ky / p->ny);
        w2 = p->g * p->H * (4 * sx * sx / (dx * dx) + 4 * sy * sy / (dy * dy)) + p->f * p->f * cx * cx * cy * cy;
      }
      best = std::max(best, w2);
    }
  }
  if (p->spectral == 2) {
    p->sigma = p->shift_mode == REXI_SHIFT_MIDPOINT ? 0.5 * (lmin + lmax)
               : p->shift_mode == REXI_SHIFT_VALUE  ? p->shift_value
                                                    : 0.0;
    p->rho = p->rho_natural = std::max(fabs(lmin - p->sigma), fabs(lmax - p->sigma));
  } else {
    p->sigma = 0.0;
    p->rho = p->rho_natural = sqrt(best);
  }
}
}  // namespace

extern "C" rexi_status rexi_plan_set_symbol(rexi_plan_t p, int32_t symbol) {
  g_err[0] = 0;
  if (!p || (symbol != REXI_SYMBOL_CGRID && symbol != REXI_SYMBOL_SPECTRAL && symbol != REXI_SYMBOL_SCHRODINGER))
    return fail(REXI_EINVAL, "bad symbol");
  if (p->depth && symbol != REXI_SYMBOL_CGRID) return fail(REXI_EUNSUPPORTED, "this symbol needs constant depth");
  p->spectral = symbol;
  if (p->depth) return REXI_OK;
  update_rho(p);
  return REXI_OK;
}

extern "C" rexi_status rexi_plan_set_shift(rexi_plan_t p, int32_t mode, double sigma) {
  g_err[0] = 0;
  if (!p || mode < REXI_SHIFT_NONE || mode > REXI_SHIFT_VALUE || !isfinite(sigma))
    return fail(REXI_EINVAL, "bad shift mode or value");
  if (mode == REXI_SHIFT_VALUE && sigma != 0.0 && p->spectral != 2)
    return fail(REXI_EUNSUPPORTED,
                "a non-zero shift needs the scalar operator (the shallow-water spectrum is symmetric about 0)");
  p->shift_mode = mode;
  p->shift_value = sigma;
  if (!p->depth) update_rho(p);
  return REXI_OK;
}

extern "C" rexi_status rexi_plan_set_coefficients(rexi_plan_t p, int32_t set) {
  g_err[0] = 0;
  if (!p || set < REXI_COEF_REXII || set > REXI_COEF_REXIE) return fail(REXI_EINVAL, "bad coefficient set");
  p->coef_set = set;
  return REXI_OK;
}

namespace {
void fit_to_array(const GaussFit& f, double* a) {
  for (int l = -kL; l <= kL; ++l) {
    const int k = l < 0 ? -l : l;
    a[2 * (l + kL)] = f.are[k];
    a[2 * (l + kL) + 1] = l < 0 ? -f.aim[k] : f.aim[k];
  }
}
}  // namespace

extern "C" rexi_status rexi_gaussian_fit_table(double* mu, double* a_re_im) {
  g_err[0] = 0;
  if (!mu || !a_re_im) return fail(REXI_EINVAL, "NULL argument");
  const GaussFit f = table_fit();
  *mu = f.mu;
  fit_to_array(f, a_re_im);
  return REXI_OK;
}

extern "C" rexi_status rexi_gaussian_refit(double mu, int32_t K, double xmax, int32_t n_candidates,
                                           double* a_re_im, double* max_err) {
  g_err[0] = 0;
  if (!a_re_im) return fail(REXI_EINVAL, "NULL coefficient array");
  GaussFit f;
  if (!gauss_refit(mu, K, xmax, n_candidates, &f, max_err))
    return fail(REXI_EINVAL,
                "refit needs mu < 0, 2L+1 <= K <= 20000, xmax > 0, K <= n_candidates <= 1e6, K n_candidates <= 5e8");
  fit_to_array(f, a_re_im);
  return REXI_OK;
}

extern "C" rexi_status rexi_plan_set_gaussian_fit(rexi_plan_t p, double mu, const double* a_re_im) {
  g_err[0] = 0;
  if (!p) return fail(REXI_EINVAL, "plan NULL");
  GaussFit f = table_fit();
  bool custom = false;
  if (a_re_im) {
    if (!(mu < 0.0) || !isfinite(mu)) return fail(REXI_EINVAL, "mu must be finite and < 0");
    double amax = 0.0;
    for (int i = 0; i < 2 * (2 * kL + 1); ++i) {
      if (!isfinite(a_re_im[i])) return fail(REXI_EINVAL, "non-finite coefficient");
      amax = std::max(amax, fabs(a_re_im[i]));
    }
    // a_{-l} = conj(a_l) (the symmetric form of eq. A(x,mu)); a_0 real
    for (int l = 0; l <= kL; ++l) {
      const double* pl = a_re_im + 2 * (kL + l);
      const double* ml = a_re_im + 2 * (kL - l);
      if (fabs(pl[0] - ml[0]) > 1e-14 * amax || fabs(pl[1] + ml[1]) > 1e-14 * amax)
        return fail(REXI_EINVAL, "coefficients must satisfy a_{-l} = conj(a_l)");
      f.are[l] = pl[0];
      f.aim[l] = l == 0 ? 0.0 : pl[1];
    }
    f.mu = mu;
    custom = true;
  }
  // tables built from the old fit may still be read by queued work
  if (!p->coef.empty()) {
    CUDA_TRY(cudaDeviceSynchronize(), "fit change");
    for (auto& c : p->coef) {
      cudaFree(c.dev);
      cudaEventDestroy(c.ready);
    }
    p->coef.clear();
  }
  p->fit = f;
  p->fit_custom = custom;
  ++p->fit_gen;
  return REXI_OK;
}

extern "C" rexi_status rexi_plan_get_shift(rexi_plan_t p, double* sigma) {
  g_err[0] = 0;
  if (!p || !sigma) return fail(REXI_EINVAL, "NULL argument");
  *sigma = p->sigma;
  return REXI_OK;
}

extern "C" rexi_status rexi_plan_set_rho(rexi_plan_t p, double rho) {
  g_err[0] = 0;
  if (!p || !(rho >= 0.0) || !isfinite(rho)) return fail(REXI_EINVAL, "bad rho");
  p->rho = rho > 0.0 ? rho : p->rho_natural;
  p->kry.rho_bound = p->rho;  // interval of the shared-Krylov error bound
  return REXI_OK;
}
