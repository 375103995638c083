// Variable-depth (Krylov) path: pole-batched conjugate gradients on the REXII
// pair operators, matrix-free C-grid stencils, FP64 accumulation over terms.
//
// For variable depth H(x, y) the operator A is no longer Fourier-diagonal.  A
// is skew-adjoint in the energy inner product <a, b>_W = sum w conj(a) b with
// w = (g/H, 1, 1) (the discrete energy is conserved), so for every REXII term n
//   N_n = (alpha_{-n} I - tau A)(alpha_n I + tau A) = B_n^* B_n,  B_n = alpha_n I + tau A
// (alpha_{-n} = conj(alpha_n)) is self-adjoint positive definite in that
// inner product.  The term of eq. REXI_Modified_matrix,
//   Gamma_n C2 (alpha_n + tau A)^{-1} f + Gamma_n (C1 - C2 alpha_{-n}) N_n^{-1} f
//     = Gamma_n (C1 - C2 tau A) N_n^{-1} f,
// is therefore one CG solve with N_n (two stencil applications per
// iteration) followed by one more stencil application.  All terms are
// independent: a launch covers a batch of terms (grid = spatial tiles x terms),
// each term with its own CG scalars, convergence flag and iteration count.
//
// Per CG iteration two kernels (p' = r + beta p is formed on the fly where it
// is needed, so that no kernel writes a vector that a neighbouring tile reads
// in its halo):
//   cg_apply_B : t <- B_n p'  (stencil on p') ;  ||t||_W^2
//   cg_update  : q <- B_n^* t (stencil on t) ; p <- p' ; x += a p ; r -= a q ; ||r||_W^2
// Dot products reduce in registers (warp shuffles), per block in shared
// memory, then deterministically across blocks: each block writes a partial,
// and the last block to finish (atomic ticket, no waiting) sums the partials
// in index order and updates the term's scalars.  The host polls the status
// flags every few iterations.  A final kernel adds
// Gamma_n (C1 x - C2 tau A x) over the batch into the FP64 accumulator.
#include <math.h>
#include <string.h>

#include <algorithm>
#include <vector>

#include "internal.h"
#include "krylov.h"

namespace rexi {

namespace {

constexpr int TX = 32;        // tile width (x, contiguous)
constexpr int TY = 16;        // tile height
constexpr int THREADS = 256;  // 2 rows per thread
constexpr int HX = TX + 2, HY = TY + 2;

struct TermScalars {
  double2 alpha_n, alpha_mn;  // shifts of B_n and B_n^*
  double2 gC1, gC2;           // Gamma_n C1_n, Gamma_n C2_n
  double gamma, gamma0, dot1, a, beta;
  int iters, status;          // status 0 active, 1 converged, 2 iteration cap
  int pad0, pad1;
};

struct Geom {
  int nx, ny, tiles_x, tiles_y;
  double inv_dx, inv_dy, g, f, tau;
  size_t fstride;  // nx * ny
};

__device__ __forceinline__ double2 cadd(double2 a, double2 b) { return make_double2(a.x + b.x, a.y + b.y); }
__device__ __forceinline__ double2 csub(double2 a, double2 b) { return make_double2(a.x - b.x, a.y - b.y); }
__device__ __forceinline__ double2 cscale(double s, double2 a) { return make_double2(s * a.x, s * a.y); }
__device__ __forceinline__ double2 cmul(double2 a, double2 b) {
  return make_double2(fma(a.x, b.x, -a.y * b.y), fma(a.x, b.y, a.y * b.x));
}
__device__ __forceinline__ double cabs2(double2 a) { return fma(a.x, a.x, a.y * a.y); }

// Stencil of A at tile point (li, lj) of the shared arrays (with a halo of 1).
// eta: -H (d_x^b u + d_y^b v);  u: -g d_x^f eta + f avg4(v);  v: -g d_y^f eta - f avg4(u)
__device__ __forceinline__ void apply_A(const double2 (*E)[HX], const double2 (*U)[HX],
                                        const double2 (*V)[HX], int li, int lj, double Hij,
                                        const Geom& G, double2& ae, double2& au, double2& av) {
  const double2 div = cadd(cscale(G.inv_dx, csub(U[lj][li], U[lj][li - 1])),
                           cscale(G.inv_dy, csub(V[lj][li], V[lj - 1][li])));
  ae = cscale(-Hij, div);
  const double2 v4 = cadd(cadd(V[lj][li], V[lj][li + 1]), cadd(V[lj - 1][li], V[lj - 1][li + 1]));
  au = cadd(cscale(-G.g * G.inv_dx, csub(E[lj][li + 1], E[lj][li])), cscale(0.25 * G.f, v4));
  const double2 u4 = cadd(cadd(U[lj][li], U[lj][li - 1]), cadd(U[lj + 1][li], U[lj + 1][li - 1]));
  av = csub(cscale(-G.g * G.inv_dy, csub(E[lj + 1][li], E[lj][li])), cscale(0.25 * G.f, u4));
}

__device__ __forceinline__ double block_sum(double v, double* red) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
  const int w = threadIdx.x >> 5, l = threadIdx.x & 31;
  if (l == 0) red[w] = v;
  __syncthreads();
  double s = 0.0;
  if (threadIdx.x == 0)
    for (int i = 0; i < THREADS / 32; ++i) s += red[i];  // fixed order
  return s;  // valid in thread 0
}

// Last-block reduction over the tiles of one term.  Returns true in thread 0
// of the last block, with *total the sum of all partials in index order.
__device__ __forceinline__ bool last_block_total(double mine, double* partials, unsigned* counter,
                                                 int ntiles, int tile, double* total) {
  __shared__ bool is_last;
  if (threadIdx.x == 0) {
    partials[tile] = mine;
    __threadfence();
    const unsigned ticket = atomicAdd(counter, 1u);
    is_last = (ticket == (unsigned)ntiles - 1);
  }
  __syncthreads();
  if (!is_last) return false;
  if (threadIdx.x == 0) {
    __threadfence();
    double s = 0.0;
    const volatile double* vp = partials;
    for (int i = 0; i < ntiles; ++i) s += vp[i];
    *total = s;
    *counter = 0u;
  }
  return threadIdx.x == 0;
}

__device__ __forceinline__ size_t gidx(const Geom& G, int i, int j) {
  i = (i + G.nx) % G.nx;
  j = (j + G.ny) % G.ny;
  return (size_t)j * G.nx + i;
}

// --- initialisation: x = 0, r = f (real part only for real input), p = 0, gamma0 = ||f||_W^2
__global__ void __launch_bounds__(THREADS) cg_init(Geom G, const double* __restrict__ H,
                                                   const double2* __restrict__ f, int real_input,
                                                   double2* x, double2* r, double2* p, size_t vstride,
                                                   TermScalars* sc, double* partials, unsigned* counters,
                                                   double rtol) {
  __shared__ double red[THREADS / 32];
  const int term = blockIdx.z;
  const int tile = blockIdx.y * G.tiles_x + blockIdx.x;
  const int ntiles = G.tiles_x * G.tiles_y;
  double2* xb = x + (size_t)term * vstride;
  double2* rb = r + (size_t)term * vstride;
  double2* pb = p + (size_t)term * vstride;
  double loc = 0.0;
  for (int k = threadIdx.x; k < TX * TY; k += THREADS) {
    const int i = blockIdx.x * TX + (k % TX), j = blockIdx.y * TY + (k / TX);
    if (i >= G.nx || j >= G.ny) continue;
    const size_t id = (size_t)j * G.nx + i;
    const double w0 = G.g / H[id];
#pragma unroll
    for (int c = 0; c < 3; ++c) {
      double2 v = f[id + c * G.fstride];
      if (real_input) v.y = 0.0;
      rb[id + c * G.fstride] = v;
      xb[id + c * G.fstride] = make_double2(0.0, 0.0);
      pb[id + c * G.fstride] = make_double2(0.0, 0.0);
      loc += (c == 0 ? w0 : 1.0) * cabs2(v);
    }
  }
  const double s = block_sum(loc, red);
  double tot;
  if (last_block_total(s, partials + (size_t)term * ntiles, counters + term, ntiles, tile, &tot)) {
    TermScalars& S = sc[term];
    S.gamma = tot;
    S.gamma0 = tot;
    S.beta = 0.0;
    S.a = 0.0;
    S.iters = 0;
    S.status = (tot == 0.0) ? 1 : 0;  // zero right-hand side: x = 0 is exact
  }
}

// Loads p_new = r + beta p (3 fields) on the tile plus halo into shared memory.
template <bool UPDATE_P>
__device__ __forceinline__ void load_tile(const Geom& G, const double2* a, const double2* b, double beta,
                                          double2 (*E)[HX], double2 (*U)[HX], double2 (*V)[HX]) {
  const int i0 = blockIdx.x * TX - 1, j0 = blockIdx.y * TY - 1;
  for (int k = threadIdx.x; k < HX * HY; k += THREADS) {
    const int li = k % HX, lj = k / HX;
    const size_t id = gidx(G, i0 + li, j0 + lj);
    double2 e = a[id], u = a[id + G.fstride], v = a[id + 2 * G.fstride];
    if (UPDATE_P) {
      const double2 pe = b[id], pu = b[id + G.fstride], pv = b[id + 2 * G.fstride];
      e = make_double2(fma(beta, pe.x, e.x), fma(beta, pe.y, e.y));
      u = make_double2(fma(beta, pu.x, u.x), fma(beta, pu.y, u.y));
      v = make_double2(fma(beta, pv.x, v.x), fma(beta, pv.y, v.y));
    }
    E[lj][li] = e;
    U[lj][li] = u;
    V[lj][li] = v;
  }
  __syncthreads();
}

// t <- alpha_n p' + tau A p' with p' = r + beta p formed on the fly (p itself
// is not written here: neighbouring tiles read p in their halo);
// dot1 = ||t||_W^2 ; a = gamma / dot1
__global__ void __launch_bounds__(THREADS) cg_apply_B(Geom G, const double* __restrict__ H, const double2* p,
                                                      const double2* r, double2* t, size_t vstride,
                                                      TermScalars* sc, double* partials, unsigned* counters) {
  __shared__ double2 E[HY][HX], U[HY][HX], V[HY][HX];
  __shared__ double red[THREADS / 32];
  const int term = blockIdx.z;
  TermScalars& S = sc[term];
  if (S.status != 0) return;
  const int tile = blockIdx.y * G.tiles_x + blockIdx.x;
  const int ntiles = G.tiles_x * G.tiles_y;
  const double2* pb = p + (size_t)term * vstride;
  const double2* rb = r + (size_t)term * vstride;
  double2* tb = t + (size_t)term * vstride;
  load_tile<true>(G, rb, pb, S.beta, E, U, V);
  const double2 al = S.alpha_n;
  double loc = 0.0;
  for (int k = threadIdx.x; k < TX * TY; k += THREADS) {
    const int li = k % TX + 1, lj = k / TX + 1;
    const int i = blockIdx.x * TX + li - 1, j = blockIdx.y * TY + lj - 1;
    if (i >= G.nx || j >= G.ny) continue;
    const size_t id = (size_t)j * G.nx + i;
    const double Hij = H[id];
    double2 ae, au, av;
    apply_A(E, U, V, li, lj, Hij, G, ae, au, av);
    const double2 te = cadd(cmul(al, E[lj][li]), cscale(G.tau, ae));
    const double2 tu = cadd(cmul(al, U[lj][li]), cscale(G.tau, au));
    const double2 tv = cadd(cmul(al, V[lj][li]), cscale(G.tau, av));
    tb[id] = te;
    tb[id + G.fstride] = tu;
    tb[id + 2 * G.fstride] = tv;
    loc += (G.g / Hij) * cabs2(te) + cabs2(tu) + cabs2(tv);
  }
  const double s = block_sum(loc, red);
  double tot;
  if (last_block_total(s, partials + (size_t)term * ntiles, counters + term, ntiles, tile, &tot)) {
    S.dot1 = tot;
    S.a = tot > 0.0 ? S.gamma / tot : 0.0;
  }
}

// q = alpha_{-n} t - tau A t ; p <- r + beta p ; x += a p ; r -= a q ;
// gamma_new = ||r||_W^2 ; convergence.  Only t is read across tile borders.
__global__ void __launch_bounds__(THREADS) cg_update(Geom G, const double* __restrict__ H, const double2* t,
                                                     double2* p, double2* x, double2* r, size_t vstride,
                                                     TermScalars* sc, double* partials, unsigned* counters,
                                                     double rtol, int max_iters) {
  __shared__ double2 E[HY][HX], U[HY][HX], V[HY][HX];
  __shared__ double red[THREADS / 32];
  const int term = blockIdx.z;
  TermScalars& S = sc[term];
  if (S.status != 0) return;
  const int tile = blockIdx.y * G.tiles_x + blockIdx.x;
  const int ntiles = G.tiles_x * G.tiles_y;
  const double2* tb = t + (size_t)term * vstride;
  double2* pb = p + (size_t)term * vstride;
  double2* xb = x + (size_t)term * vstride;
  double2* rb = r + (size_t)term * vstride;
  load_tile<false>(G, tb, nullptr, 0.0, E, U, V);
  const double2 am = S.alpha_mn;
  const double a = S.a;
  const double beta = S.beta;
  double loc = 0.0;
  for (int k = threadIdx.x; k < TX * TY; k += THREADS) {
    const int li = k % TX + 1, lj = k / TX + 1;
    const int i = blockIdx.x * TX + li - 1, j = blockIdx.y * TY + lj - 1;
    if (i >= G.nx || j >= G.ny) continue;
    const size_t id = (size_t)j * G.nx + i;
    const double Hij = H[id];
    double2 ae, au, av;
    apply_A(E, U, V, li, lj, Hij, G, ae, au, av);
    const double2 q[3] = {csub(cmul(am, E[lj][li]), cscale(G.tau, ae)),
                          csub(cmul(am, U[lj][li]), cscale(G.tau, au)),
                          csub(cmul(am, V[lj][li]), cscale(G.tau, av))};
#pragma unroll
    for (int c = 0; c < 3; ++c) {
      const size_t o = id + c * G.fstride;
      double2 xv = xb[o], rv = rb[o];
      double2 pv = pb[o];
      pv = make_double2(fma(beta, pv.x, rv.x), fma(beta, pv.y, rv.y));
      pb[o] = pv;
      xv = make_double2(fma(a, pv.x, xv.x), fma(a, pv.y, xv.y));
      rv = make_double2(fma(-a, q[c].x, rv.x), fma(-a, q[c].y, rv.y));
      xb[o] = xv;
      rb[o] = rv;
      loc += (c == 0 ? G.g / Hij : 1.0) * cabs2(rv);
    }
  }
  const double s = block_sum(loc, red);
  double tot;
  if (last_block_total(s, partials + (size_t)term * ntiles, counters + term, ntiles, tile, &tot)) {
    S.beta = S.gamma > 0.0 ? tot / S.gamma : 0.0;
    S.gamma = tot;
    S.iters += 1;
    if (tot <= rtol * rtol * S.gamma0)
      S.status = 1;
    else if (S.iters >= max_iters)
      S.status = 2;
  }
}

// acc += sum over the batch of Gamma_n (C1 x - C2 tau A x), batch order fixed.
__global__ void __launch_bounds__(THREADS) cg_accumulate(Geom G, const double* __restrict__ H,
                                                         const double2* x, size_t vstride, int nbatch,
                                                         const TermScalars* sc, double2* acc, int first) {
  __shared__ double2 E[HY][HX], U[HY][HX], V[HY][HX];
  double2 s[2][3];
  for (int q = 0; q < 2; ++q)
    for (int c = 0; c < 3; ++c) s[q][c] = make_double2(0.0, 0.0);
  for (int b = 0; b < nbatch; ++b) {
    __syncthreads();
    load_tile<false>(G, x + (size_t)b * vstride, nullptr, 0.0, E, U, V);
    const double2 c1 = sc[b].gC1, c2 = sc[b].gC2;
    int q = 0;
    for (int k = threadIdx.x; k < TX * TY; k += THREADS, ++q) {
      const int li = k % TX + 1, lj = k / TX + 1;
      const int i = blockIdx.x * TX + li - 1, j = blockIdx.y * TY + lj - 1;
      if (i >= G.nx || j >= G.ny) continue;
      const double Hij = H[(size_t)j * G.nx + i];
      double2 ae, au, av;
      apply_A(E, U, V, li, lj, Hij, G, ae, au, av);
      s[q][0] = cadd(s[q][0], csub(cmul(c1, E[lj][li]), cmul(c2, cscale(G.tau, ae))));
      s[q][1] = cadd(s[q][1], csub(cmul(c1, U[lj][li]), cmul(c2, cscale(G.tau, au))));
      s[q][2] = cadd(s[q][2], csub(cmul(c1, V[lj][li]), cmul(c2, cscale(G.tau, av))));
    }
  }
  int q = 0;
  for (int k = threadIdx.x; k < TX * TY; k += THREADS, ++q) {
    const int i = blockIdx.x * TX + k % TX, j = blockIdx.y * TY + k / TX;
    if (i >= G.nx || j >= G.ny) continue;
    const size_t id = (size_t)j * G.nx + i;
    for (int c = 0; c < 3; ++c) {
      const size_t o = id + c * G.fstride;
      acc[o] = first ? s[q][c] : cadd(acc[o], s[q][c]);
    }
  }
}

__global__ void finish_output(const double2* acc, double2* out, size_t n3, int real_out) {
  const size_t i = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n3) return;
  double2 v = acc[i];
  if (real_out) v.y = 0.0;
  out[i] = v;
}

// Diagonal scaling used by the adjoint: out_eta = s * in_eta * (H / g)^e, others copied.
__global__ void scale_eta(const double2* in, double2* out, const double* H, size_t nk, double g, int inverse,
                          int real_in) {
  const size_t i = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= 3 * nk) return;
  double2 v = in[i];
  if (real_in) v.y = 0.0;
  if (i < nk) {
    const double w = g / H[i];  // energy weight of eta
    const double s = inverse ? 1.0 / w : w;
    v.x *= s;
    v.y *= s;
  }
  out[i] = v;
}

struct KLayout {
  size_t acc_off, vec_off, vec_bytes, sc_off, part_off, cnt_off, tmp_off, total;
  int batch, ntiles;
};

KLayout layout(const KrylovSettings* k, int nterms, bool adjoint) {
  KLayout L{};
  const size_t nk = (size_t)k->nx * k->ny;
  const size_t state = 3 * nk * sizeof(double2);
  auto al = [](size_t v) { return (v + 255) / 256 * 256; };
  L.batch = std::max(1, std::min(k->term_batch, nterms));
  L.ntiles = ((k->nx + TX - 1) / TX) * ((k->ny + TY - 1) / TY);
  size_t off = 0;
  L.acc_off = off;
  off += al(state);
  L.tmp_off = off;  // adjoint: scaled input
  if (adjoint) off += al(state);
  L.vec_off = off;
  L.vec_bytes = al(state);
  off += 4 * (size_t)L.batch * L.vec_bytes;  // x, r, p, t per term
  L.sc_off = off;
  off += al((size_t)L.batch * sizeof(TermScalars));
  L.part_off = off;
  off += al((size_t)L.batch * L.ntiles * sizeof(double));
  L.cnt_off = off;
  off += al((size_t)L.batch * sizeof(unsigned));
  L.total = off;
  return L;
}

int n_terms_for(int M, int real_input) {
  const int N = M + kL;
  return real_input ? N + 1 : 2 * N + 1;
}

}  // namespace

rexi_status krylov_init(KrylovSettings* k, int nx, int ny, double Lx, double Ly, double g, double f,
                        const double* depth, double Hmean) {
  k->nx = nx;
  k->ny = ny;
  k->Lx = Lx;
  k->Ly = Ly;
  k->g = g;
  k->f = f;
  k->depth = depth;
  k->Hmean = Hmean;
  return REXI_OK;
}

void krylov_destroy(KrylovSettings*) {}

size_t krylov_workspace_bytes(const KrylovSettings* k, int M, int real_input, int /*form*/) {
  return layout(k, n_terms_for(M, real_input), true).total;
}

rexi_status krylov_step(KrylovSettings* k, int form, double h, int M, const void* in, void* out, double dt,
                        int real_input, int term_begin, int term_end, void* ws, size_t ws_bytes, cudaStream_t s,
                        rexi_step_info* info, bool adjoint, const KrylovHooks& hooks) {
  auto mark = [&](int i) {
    if (hooks.mark) hooks.mark(hooks.ctx, i, s);
  };
  auto count = [&](int64_t n) {
    if (hooks.launches) *hooks.launches += n;
  };
  if (form != REXI_FORM_FP64) {
    set_last_error("variable-depth path: only the FP64 form is available");
    return REXI_EUNSUPPORTED;
  }
  const int N = M + kL;
  if (term_end < 0 || term_end > N + 1) term_end = N + 1;
  if (term_begin < 0 || term_begin > term_end) {
    set_last_error("bad term range");
    return REXI_EINVAL;
  }
  const size_t nk = (size_t)k->nx * k->ny;
  const size_t n3 = 3 * nk;
  if ((const char*)in < (const char*)out + n3 * sizeof(double2) &&
      (const char*)out < (const char*)in + n3 * sizeof(double2)) {
    set_last_error("variable-depth path: input and output must not overlap");
    return REXI_EINVAL;
  }
  // term list: n = 0..N (real input, Gamma) or -N..N, restricted to |n| in [term_begin, term_end)
  TermSet ts;
  rexii_terms(M, h, &ts);
  const double hmu = h * ts.mu;
  std::vector<TermScalars> terms;
  for (int n = real_input ? 0 : -N; n <= N; ++n) {
    const int an = n < 0 ? -n : n;
    if (an < term_begin || an >= term_end) continue;
    const int i = n + N;
    const double gam = (real_input && n > 0) ? 2.0 : 1.0;
    TermScalars t;
    memset(&t, 0, sizeof(t));
    t.alpha_n = make_double2(hmu, h * n);
    t.alpha_mn = make_double2(hmu, -h * n);
    // C1 = c1 h mu + c2 h n,  C2 = i c2
    t.gC1 = make_double2(gam * (ts.c1re[i] * hmu + ts.c2re[i] * h * n), gam * (ts.c1im[i] * hmu + ts.c2im[i] * h * n));
    t.gC2 = make_double2(-gam * ts.c2im[i], gam * ts.c2re[i]);
    terms.push_back(t);
  }
  const KLayout L = layout(k, (int)std::max<size_t>(terms.size(), 1), adjoint);
  if (ws_bytes < L.total) {
    set_last_error("workspace too small for the variable-depth path");
    return REXI_ENOMEM;
  }
  char* base = static_cast<char*>(ws);
  double2* acc = reinterpret_cast<double2*>(base + L.acc_off);
  double2* vecs = reinterpret_cast<double2*>(base + L.vec_off);
  const size_t vstride = L.vec_bytes / sizeof(double2);
  double2* X = vecs;
  double2* R = vecs + (size_t)L.batch * vstride;
  double2* P = vecs + 2 * (size_t)L.batch * vstride;
  double2* T = vecs + 3 * (size_t)L.batch * vstride;
  TermScalars* dsc = reinterpret_cast<TermScalars*>(base + L.sc_off);
  double* partials = reinterpret_cast<double*>(base + L.part_off);
  unsigned* counters = reinterpret_cast<unsigned*>(base + L.cnt_off);

  Geom G;
  G.nx = k->nx;
  G.ny = k->ny;
  G.tiles_x = (k->nx + TX - 1) / TX;
  G.tiles_y = (k->ny + TY - 1) / TY;
  G.inv_dx = k->nx / k->Lx;
  G.inv_dy = k->ny / k->Ly;
  G.g = k->g;
  G.f = k->f;
  // adjoint: r(tau A)^H = r(tau A^T) = W r(-tau A) W^{-1} with W = diag(g/H, 1, 1)
  G.tau = adjoint ? -dt : dt;
  G.fstride = nk;

  const double2* src = static_cast<const double2*>(in);
  cudaError_t e;
  const int eb = 256;
  const unsigned ebl = (unsigned)((n3 + eb - 1) / eb);
  if (adjoint) {
    double2* tmp = reinterpret_cast<double2*>(base + L.tmp_off);
    scale_eta<<<ebl, eb, 0, s>>>(src, tmp, k->depth, nk, k->g, 1, real_input);
    src = tmp;
  }
  if ((e = cudaMemsetAsync(counters, 0, (size_t)L.batch * sizeof(unsigned), s)) != cudaSuccess) {
    set_last_error(cudaGetErrorString(e));
    return REXI_ECUDA;
  }
  if (terms.empty()) {
    if ((e = cudaMemsetAsync(acc, 0, n3 * sizeof(double2), s)) != cudaSuccess) {
      set_last_error(cudaGetErrorString(e));
      return REXI_ECUDA;
    }
  }
  int worst_iters = 0, unconverged = 0;
  int64_t term_iters = 0;
  double worst_res = 0.0;
  const int check_every = 16;
  std::vector<TermScalars> hs(L.batch);
  for (size_t b0 = 0; b0 < terms.size(); b0 += L.batch) {
    const int nb = (int)std::min<size_t>(L.batch, terms.size() - b0);
    mark(0);
    e = cudaMemcpyAsync(dsc, &terms[b0], nb * sizeof(TermScalars), cudaMemcpyHostToDevice, s);
    if (e != cudaSuccess) break;
    mark(1);
    dim3 grid(G.tiles_x, G.tiles_y, nb);
    cg_init<<<grid, THREADS, 0, s>>>(G, k->depth, src, real_input, X, R, P, vstride, dsc, partials, counters,
                                     k->rtol);
    count(1);
    mark(2);
    int it = 0;
    bool done = false;
    while (!done) {
      for (int c = 0; c < check_every; ++c) {
        cg_apply_B<<<grid, THREADS, 0, s>>>(G, k->depth, P, R, T, vstride, dsc, partials, counters);
        cg_update<<<grid, THREADS, 0, s>>>(G, k->depth, T, P, X, R, vstride, dsc, partials, counters, k->rtol,
                                           k->max_iters);
      }
      count(2 * check_every);
      it += check_every;
      if ((e = cudaGetLastError()) != cudaSuccess) break;
      e = cudaMemcpyAsync(hs.data(), dsc, nb * sizeof(TermScalars), cudaMemcpyDeviceToHost, s);
      if (e == cudaSuccess) e = cudaStreamSynchronize(s);
      if (e != cudaSuccess) break;
      done = true;
      for (int b = 0; b < nb; ++b)
        if (hs[b].status == 0) done = false;
      if (it > k->max_iters + check_every) done = true;  // the device caps every term at max_iters
    }
    if (e != cudaSuccess) break;
    mark(3);
    for (int b = 0; b < nb; ++b) {
      term_iters += hs[b].iters;
      worst_iters = std::max(worst_iters, hs[b].iters);
      if (hs[b].status != 1) ++unconverged;
      if (hs[b].gamma0 > 0) worst_res = std::max(worst_res, sqrt(hs[b].gamma / hs[b].gamma0));
    }
    dim3 g2(G.tiles_x, G.tiles_y, 1);
    cg_accumulate<<<g2, THREADS, 0, s>>>(G, k->depth, X, vstride, nb, dsc, acc, b0 == 0 ? 1 : 0);
    count(1);
    if ((e = cudaGetLastError()) != cudaSuccess) break;
    mark(4);
  }
  if (e != cudaSuccess) {
    set_last_error(cudaGetErrorString(e));
    return REXI_ECUDA;
  }
  if (adjoint) {
    scale_eta<<<ebl, eb, 0, s>>>(acc, static_cast<double2*>(out), k->depth, nk, k->g, 0, 0);
    if (real_input) {
      finish_output<<<ebl, eb, 0, s>>>(static_cast<double2*>(out), static_cast<double2*>(out), n3, 1);
    }
  } else {
    finish_output<<<ebl, eb, 0, s>>>(acc, static_cast<double2*>(out), n3, real_input);
  }
  if ((e = cudaGetLastError()) != cudaSuccess) {
    set_last_error(cudaGetErrorString(e));
    return REXI_ECUDA;
  }
  if (info) {
    memset(info, 0, sizeof(*info));
    info->N = N;
    info->n_terms = n_terms_for(M, real_input);
    info->n_poles = real_input ? 2 * (N + 1) : 2 * (2 * N + 1);
    info->krylov_iters = worst_iters;
    info->krylov_unconverged = unconverged;
    info->krylov_max_rel_res = worst_res;
    info->krylov_term_iters = term_iters;
  }
  if (unconverged > 0) {
    set_last_error("variable-depth path: some terms reached the iteration cap");
    return REXI_ENOCONV;
  }
  return REXI_OK;
}

}  // namespace rexi
