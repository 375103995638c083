// rexi_step_noalloc: the constant-depth REXII step for callers that may not
// allocate device memory.
//
// Some callers cannot call cudaMalloc or any allocating routine: code that
// runs where allocation is forbidden or unsafe (inside another library's
// memory-pool or allocator hooks, a real-time loop with a fixed memory
// budget, a process whose device memory is fully reserved up front), or a
// host without access to torch's caching allocator.  rexi_plan_create
// allocates plan tables and rexi_step wants a caller workspace; this entry
// point needs neither.  Its scratch (FFT twiddles, half-angle tables, the
// coefficient table and the spectrum) lives in one file-scope static device
// array of fixed size, which every GPU that loads the library keeps until
// the process exits.
//
// Limits: 2 <= nx, ny <= 1024 and nx * ny <= 65536 (a 256 x 256 grid), every
// prime factor of nx and ny <= 127, and at most 8193 scalar REXII terms
// (2N + 1 with N = M + 24; with h = 0.5 and tol = 1e-10 that is
// dt * rho(A) up to about 2030).  Larger requests return REXI_EINVAL and
// launch nothing.  Arithmetic is the fused FP64 form of rexi_step.
//
// Sharing: every call uses the same device array, which keeps the contents of
// the last call; each call writes every region before reading it, so nothing
// has to start at zero.  Calls whose GPU work overlaps (on different streams,
// or from several host threads) race on that array and give wrong results:
// order them on one stream.  The host-side tables are static too; a mutex
// serialises the host part of concurrent calls.
//
// Set-up: the first call on each device asks the runtime for the device
// address of the array (cudaGetSymbolAddress, with that device current) and
// caches it for the life of the process.  The cache does not survive
// cudaDeviceReset (or any other teardown of the device's primary context):
// after one, the cached address is stale, so do not call this entry point
// again in that process.
//
// Tables: each call fills host-side static tables (twiddles, half angles, the
// coefficient table) under a mutex and copies them into the device array with
// cudaMemcpyAsync from that pageable memory; the driver stages such copies
// before the call returns, so the next call may overwrite the host tables.
// For the same reason the entry point cannot be captured in a CUDA graph (a
// captured copy would read host tables that later calls overwrite): a call on
// a capturing stream returns REXI_EINVAL before any copy or launch.
#include <math.h>
#include <stdint.h>

#include <mutex>

#include "internal.h"

namespace {

using namespace rexi;

constexpr int kMaxSide = 1024;
constexpr int kMaxPoints = 65536;
constexpr int kMaxTerms = 8193;  // 2N + 1
constexpr int kMaxM = (kMaxTerms - 1) / 2 - kL;
constexpr int kMaxDevices = 64;

// Region offsets inside the static array (all multiples of 256 bytes).
constexpr size_t kTwX = 0;
constexpr size_t kTwY = kTwX + kMaxSide * sizeof(double2);
constexpr size_t kHalfX = kTwY + kMaxSide * sizeof(double2);
constexpr size_t kHalfY = kHalfX + kMaxSide * sizeof(double2);
constexpr size_t kTable = kHalfY + kMaxSide * sizeof(double2);
constexpr size_t kTableBytes = ((size_t)kMaxTerms * 6 * sizeof(double) + 255) / 256 * 256;
constexpr size_t kSpec = kTable + kTableBytes;
constexpr size_t kScratchBytes = kSpec + 3 * (size_t)kMaxPoints * sizeof(double2);  // ~3.4 MiB

static __device__ __align__(256) unsigned char g_scratch[kScratchBytes];

std::mutex g_mutex;
void* g_scratch_addr[kMaxDevices] = {};

// Host-side staging, reused by every call under g_mutex.
double2 h_tw_x[kMaxSide], h_tw_y[kMaxSide], h_half_x[kMaxSide], h_half_y[kMaxSide];
double h_table[kMaxTerms * 6];
double h_bre[2 * kMaxM + 1], h_bim[2 * kMaxM + 1];
double h_c1re[kMaxTerms], h_c1im[kMaxTerms], h_c2re[kMaxTerms], h_c2im[kMaxTerms];

// errors are reported through rexi_last_error_message()
rexi_status fail(rexi_status st, const char* msg) {
  set_last_error(msg);
  return st;
}

void fill_axis(int n, double2* tw, double2* half) {
  for (int t = 0; t < n; ++t) {
    const double a = 2.0 * M_PI * (double)t / (double)n;
    tw[t] = make_double2(cos(a), -sin(a));
    const double b = M_PI * (double)t / (double)n;
    half[t] = make_double2(cos(b), sin(b));
  }
}

}  // namespace

extern "C" rexi_status rexi_step_noalloc(int32_t nx, int32_t ny, double Lx, double Ly, double g, double f,
                                         double H, double h, const void* in_dev, void* out_dev, double dt,
                                         double tol, int32_t real_input, void* stream) {
  set_last_error("");
  if (!in_dev || !out_dev) return fail(REXI_EINVAL, "rexi_step_noalloc: NULL state pointer");
  if (((uintptr_t)in_dev | (uintptr_t)out_dev) & 15)
    return fail(REXI_EINVAL, "rexi_step_noalloc: state pointers must be 16-byte aligned");
  if (nx < 2 || ny < 2 || nx > kMaxSide || ny > kMaxSide || (long long)nx * ny > kMaxPoints)
    return fail(REXI_EINVAL,
                "rexi_step_noalloc: grid exceeds the fixed scratch (need 2 <= nx, ny <= 1024, nx*ny <= 65536)");
  if (!(Lx > 0 && Ly > 0 && g > 0 && H > 0 && isfinite(f) && isfinite(Lx) && isfinite(Ly) && isfinite(g) &&
        isfinite(H)))
    return fail(REXI_EINVAL, "rexi_step_noalloc: bad Lx/Ly/g/f/H");
  if (!valid_h(h)) return fail(REXI_EINVAL, "rexi_step_noalloc: h must lie in (0, pi)");
  if (!(dt >= 0.0) || !isfinite(dt)) return fail(REXI_EINVAL, "rexi_step_noalloc: dt must be finite and >= 0");
  FftPlan1D fx, fy;
  if (!fft_factor(nx, &fx) || !fft_factor(ny, &fy))
    return fail(REXI_EINVAL, "rexi_step_noalloc: grid sizes need prime factors <= 127");

  const double dx = Lx / nx, dy = Ly / ny;
  // rho(A): largest omega over the discrete wavenumbers (constant depth)
  double best = 0.0;
  for (int ky = 0; ky < ny; ++ky) {
    const double sy = sin(M_PI * ky / ny), cy = cos(M_PI * ky / ny);
    for (int kx = 0; kx < nx; ++kx) {
      const double sx = sin(M_PI * kx / nx), cx = cos(M_PI * kx / nx);
      const double w2 = g * H * (4.0 * sx * sx / (dx * dx) + 4.0 * sy * sy / (dy * dy)) + f * f * cx * cx * cy * cy;
      if (w2 > best) best = w2;
    }
  }
  const double rho = sqrt(best);
  const int M = pole_count(dt * rho, h, tol);
  if (M < 0) return fail(REXI_EINVAL, "rexi_step_noalloc: pole-count rule rejected dt*rho, h or tol");
  const int N = M + kL;
  const int nterms = 2 * N + 1;
  if (nterms > kMaxTerms)
    return fail(REXI_EINVAL, "rexi_step_noalloc: more than 8193 REXII terms (dt*rho too large for the fixed scratch)");

  cudaStream_t s = static_cast<cudaStream_t>(stream);
  cudaStreamCaptureStatus cap = cudaStreamCaptureStatusNone;
  if (cudaStreamIsCapturing(s, &cap) != cudaSuccess)
    return fail(REXI_ECUDA, "rexi_step_noalloc: cudaStreamIsCapturing failed");
  if (cap != cudaStreamCaptureStatusNone)
    return fail(REXI_EINVAL,
                "rexi_step_noalloc: the stream is capturing a CUDA graph; this entry point copies from "
                "host tables that later calls overwrite and cannot be captured");

  std::lock_guard<std::mutex> lock(g_mutex);
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= kMaxDevices)
    return fail(REXI_ECUDA, "rexi_step_noalloc: no current CUDA device");
  if (!g_scratch_addr[dev]) {
    void* ptr = nullptr;
    if (cudaGetSymbolAddress(&ptr, g_scratch) != cudaSuccess || !ptr)
      return fail(REXI_ECUDA, "rexi_step_noalloc: cudaGetSymbolAddress of the static scratch failed");
    g_scratch_addr[dev] = ptr;
  }
  char* base = static_cast<char*>(g_scratch_addr[dev]);

  // tables on the host, then copied into the static device array
  fill_axis(nx, h_tw_x, h_half_x);
  fill_axis(ny, h_tw_y, h_half_y);
  rexii_terms_into(M, h, h_bre, h_bim, h_c1re, h_c1im, h_c2re, h_c2im);
  const double mu = table_mu(), hmu = h * mu, q = hmu * hmu;
  double R0r = 0.0, R0i = 0.0;
  for (int n = -N; n <= N; ++n) {
    const double c1r = h_c1re[n + N], c1i = h_c1im[n + N], c2r = h_c2re[n + N], c2i = h_c2im[n + N];
    double* e = &h_table[6 * (n + N)];
    e[0] = h * n;
    e[1] = c1r * hmu;
    e[2] = c1i * hmu;
    e[3] = c2r;
    e[4] = c2i;
    e[5] = 0.0;
    const double hn = h * n, d = q + hn * hn;
    R0r += (e[1] + c2r * hn) / d;
    R0i += (e[2] + c2i * hn) / d;
  }
  cudaError_t e = cudaSuccess;
  if (e == cudaSuccess) e = cudaMemcpyAsync(base + kTwX, h_tw_x, nx * sizeof(double2), cudaMemcpyHostToDevice, s);
  if (e == cudaSuccess) e = cudaMemcpyAsync(base + kTwY, h_tw_y, ny * sizeof(double2), cudaMemcpyHostToDevice, s);
  if (e == cudaSuccess) e = cudaMemcpyAsync(base + kHalfX, h_half_x, nx * sizeof(double2), cudaMemcpyHostToDevice, s);
  if (e == cudaSuccess) e = cudaMemcpyAsync(base + kHalfY, h_half_y, ny * sizeof(double2), cudaMemcpyHostToDevice, s);
  if (e == cudaSuccess)
    e = cudaMemcpyAsync(base + kTable, h_table, (size_t)nterms * 6 * sizeof(double), cudaMemcpyHostToDevice, s);
  if (e != cudaSuccess) return fail(REXI_ECUDA, "rexi_step_noalloc: table copy failed");

  fx.tw = reinterpret_cast<const double2*>(base + kTwX);
  fy.tw = reinterpret_cast<const double2*>(base + kTwY);
  double2* spec = reinterpret_cast<double2*>(base + kSpec);
  SymbolParams sp;
  sp.nx = nx;
  sp.ny = ny;
  sp.inv_dx = 1.0 / dx;
  sp.inv_dy = 1.0 / dy;
  sp.g = g;
  sp.f = f;
  sp.H = H;
  sp.half_x = reinterpret_cast<const double2*>(base + kHalfX);
  sp.half_y = reinterpret_cast<const double2*>(base + kHalfY);
  FusedScalars fs;
  fs.tau = dt;
  fs.q = q;
  fs.R0re = R0r;
  fs.R0im = R0i;
  fs.nterms = nterms;
  fs.adjoint = 0;
  e = fft2d(static_cast<const double2*>(in_dev), spec, 3, fx, fy, -1, 1.0, real_input, 0, s);
  if (e == cudaSuccess) e = pole_fused_fp64(spec, sp, reinterpret_cast<const double*>(base + kTable), fs, s);
  if (e == cudaSuccess)
    e = fft2d(spec, static_cast<double2*>(out_dev), 3, fx, fy, +1, 1.0 / ((double)nx * ny), 0, real_input, s);
  if (e != cudaSuccess) return fail(REXI_ECUDA, "rexi_step_noalloc: kernel launch failed");
  return REXI_OK;
}
