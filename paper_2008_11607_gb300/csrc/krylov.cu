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
//
// Forms.  FP64: every vector and stencil in FP64.  On this GPU the FP64 units
// are the bottleneck of that form (one FP64 operation costs about as much
// time as 11 bytes of HBM traffic), so the stencil constants are folded
// (tau, 1/dx, g, f/4, the energy weight g/H) to keep FP64 work low.
// MIXED: per term, iterative refinement in FP64 around an FP32 CG:
//   x = 0, r = f;  repeat { solve N d = r in FP32 (complex64 vectors) to a
//   loose relative residual;  x += d;  r = f - N x in FP64 }  until the FP64
//   residual meets rtol.  The inner kernels move half the bytes of the FP64
//   ones and their arithmetic is cheap, so they are bound by HBM bandwidth.
#include <math.h>
#include <string.h>

#include <algorithm>
#include <type_traits>
#include <vector>

#include "internal.h"
#include "krylov.h"
#include "partials.cuh"

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
  double2 gP, gQ;             // single-shift weights of the term's two poles (depth gradient)
};

// ---- complex arithmetic for float2 / double2 ------------------------------
template <typename R> struct CT;
template <> struct CT<double> { using T = double2; };
template <> struct CT<float> { using T = float2; };
template <typename R> using cplx = typename CT<R>::T;

__device__ __forceinline__ double2 mk(double a, double b) { return make_double2(a, b); }
__device__ __forceinline__ float2 mk(float a, float b) { return make_float2(a, b); }
template <typename R, typename V> __device__ __forceinline__ cplx<R> cvt(V v) { return mk((R)v.x, (R)v.y); }
template <typename V> __device__ __forceinline__ V cadd(V a, V b) { return mk(a.x + b.x, a.y + b.y); }
template <typename V> __device__ __forceinline__ V csub(V a, V b) { return mk(a.x - b.x, a.y - b.y); }
template <typename V> __device__ __forceinline__ V cmul(V a, V b) {
  return mk(fma(a.x, b.x, -a.y * b.y), fma(a.x, b.y, a.y * b.x));
}
template <typename V> __device__ __forceinline__ auto cabs2(V a) -> decltype(a.x) { return fma(a.x, a.x, a.y * a.y); }

// Stencil constants in precision R; tau is folded into every coefficient.
template <typename R>
struct Geom {
  int nx, ny, tiles_x, tiles_y;
  size_t fstride;  // nx * ny
  R tdx, tdy;      // tau / dx, tau / dy (times H per point in the eta row)
  R tgdx, tgdy;    // tau g / dx, tau g / dy
  R tf4;           // tau f / 4
  R idx, idy;      // 1 / dx, 1 / dy
  const R* H;      // depth at eta points
  const R* w;      // energy weight g / H
};

// tau A at tile point (li, lj) of the shared arrays (halo of 1).
// eta: -H (d_x^b u + d_y^b v);  u: -g d_x^f eta + f avg4(v);  v: -g d_y^f eta - f avg4(u)
template <typename R>
__device__ __forceinline__ void apply_tA(const cplx<R> (*E)[HX], const cplx<R> (*U)[HX], const cplx<R> (*V)[HX],
                                         int li, int lj, R Hij, const Geom<R>& G, cplx<R>& ae, cplx<R>& au,
                                         cplx<R>& av) {
  const R hx = -Hij * G.tdx, hy = -Hij * G.tdy;
  const cplx<R> du = csub(U[lj][li], U[lj][li - 1]), dv = csub(V[lj][li], V[lj - 1][li]);
  ae = mk(fma(hx, du.x, hy * dv.x), fma(hx, du.y, hy * dv.y));
  const cplx<R> v4 = cadd(cadd(V[lj][li], V[lj][li + 1]), cadd(V[lj - 1][li], V[lj - 1][li + 1]));
  const cplx<R> de = csub(E[lj][li + 1], E[lj][li]);
  au = mk(fma(G.tf4, v4.x, -G.tgdx * de.x), fma(G.tf4, v4.y, -G.tgdx * de.y));
  const cplx<R> u4 = cadd(cadd(U[lj][li], U[lj][li - 1]), cadd(U[lj + 1][li], U[lj + 1][li - 1]));
  const cplx<R> dn = csub(E[lj + 1][li], E[lj][li]);
  av = mk(fma(-G.tf4, u4.x, -G.tgdy * dn.x), fma(-G.tf4, u4.y, -G.tgdy * dn.y));
}

// Block sum: warp shuffles in the type of v (FP32 for the FP32 kernels, so
// that they issue no FP64 work per point), then FP64 across warps.
template <typename T>
__device__ __forceinline__ double block_sum(T v, double* red) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
  const int w = threadIdx.x >> 5, l = threadIdx.x & 31;
  __syncthreads();  // red may still be read by thread 0 of a previous call
  if (l == 0) red[w] = (double)v;
  __syncthreads();
  double s = 0.0;
  if (threadIdx.x == 0)
    for (int i = 0; i < THREADS / 32; ++i) s += red[i];  // fixed order
  return s;  // valid in thread 0
}

// Last-block reduction over the tiles of one term.  Every block writes its
// partial and takes a ticket; the block that takes the last ticket sums all
// partials (each thread a fixed strided subset, then the fixed-order block
// reduction, so the result does not depend on scheduling) and returns true in
// its thread 0 with *total set.  No block waits for another.
__device__ __forceinline__ bool last_block_total(double mine, double* partials, unsigned* counter, int ntiles,
                                                 int tile, double* total, double* red) {
  __shared__ bool is_last;
  if (threadIdx.x == 0) {
    partials[tile] = mine;
    __threadfence();
    const unsigned ticket = atomicAdd(counter, 1u);
    is_last = (ticket == (unsigned)ntiles - 1);
  }
  __syncthreads();
  if (!is_last) return false;  // uniform across the block
  __threadfence();
  double s = strided_partial_sum(partials, ntiles, threadIdx.x, THREADS, 0.0, [](double a, double b) { return a + b; });
  s = block_sum(s, red);
  if (threadIdx.x == 0) {
    *total = s;
    *counter = 0u;
  }
  return threadIdx.x == 0;
}

// Periodic index; tiles reach at most one halo point beyond the grid when the
// grid is wider than a tile, so two compares replace the division there.
template <typename R>
__device__ __forceinline__ size_t gidx(const Geom<R>& G, int i, int j) {
  if (G.nx > TX) {
    i = i < 0 ? i + G.nx : (i >= G.nx ? i - G.nx : i);
  } else {
    i = (i + G.nx) % G.nx;
  }
  if (G.ny > TY) {
    j = j < 0 ? j + G.ny : (j >= G.ny ? j - G.ny : j);
  } else {
    j = (j + G.ny) % G.ny;
  }
  return (size_t)j * G.nx + i;
}

// Loads a + beta b (3 fields, converted to precision R) on the tile plus halo.
template <typename R, bool COMBINE, typename VA, typename VB>
__device__ __forceinline__ void load_tile(const Geom<R>& G, const VA* a, const VB* b, R beta, cplx<R> (*E)[HX],
                                          cplx<R> (*U)[HX], cplx<R> (*V)[HX]) {
  const int i0 = blockIdx.x * TX - 1, j0 = blockIdx.y * TY - 1;
  for (int k = threadIdx.x; k < HX * HY; k += THREADS) {
    const int li = k % HX, lj = k / HX;
    const size_t id = gidx(G, i0 + li, j0 + lj);
    cplx<R> f3[3];
#pragma unroll
    for (int c = 0; c < 3; ++c) {
      cplx<R> v = cvt<R>(a[id + c * G.fstride]);
      if (COMBINE) {
        const cplx<R> q = cvt<R>(b[id + c * G.fstride]);
        v = mk(fma(beta, q.x, v.x), fma(beta, q.y, v.y));
      }
      f3[c] = v;
    }
    E[lj][li] = f3[0];
    U[lj][li] = f3[1];
    V[lj][li] = f3[2];
  }
  __syncthreads();
}

// ---- kernels -----------------------------------------------------------------

// x = 0, r = f (real part only for real input), p = 0, gamma0 = ||f||_W^2.
// With `outer`, terms whose outer (refinement) status is not active are
// marked done at once.
template <typename R, typename VF>
__global__ void __launch_bounds__(THREADS) cg_init(Geom<R> G, const VF* __restrict__ f, int real_input,
                                                   cplx<R>* x, cplx<R>* r, cplx<R>* p, size_t vstride,
                                                   size_t fterm_stride, TermScalars* sc, const TermScalars* outer,
                                                   double* partials, unsigned* counters) {
  __shared__ double red[THREADS / 32];
  const int term = blockIdx.z;
  if (outer && outer[term].status != 0) {
    if (blockIdx.x == 0 && blockIdx.y == 0 && threadIdx.x == 0) {
      sc[term].status = 1;
      sc[term].iters = 0;
    }
    return;
  }
  const int tile = blockIdx.y * G.tiles_x + blockIdx.x;
  const int ntiles = G.tiles_x * G.tiles_y;
  cplx<R>* xb = x + (size_t)term * vstride;
  cplx<R>* rb = r + (size_t)term * vstride;
  cplx<R>* pb = p + (size_t)term * vstride;
  const VF* fb = f + (size_t)term * fterm_stride;
  const cplx<R> zero = mk((R)0, (R)0);
  R loc = 0;
  for (int k = threadIdx.x; k < TX * TY; k += THREADS) {
    const int i = blockIdx.x * TX + (k % TX), j = blockIdx.y * TY + (k / TX);
    if (i >= G.nx || j >= G.ny) continue;
    const size_t id = (size_t)j * G.nx + i;
    R acc = 0;
#pragma unroll
    for (int c = 0; c < 3; ++c) {
      cplx<R> v = cvt<R>(fb[id + c * G.fstride]);
      if (real_input) v.y = 0;
      rb[id + c * G.fstride] = v;
      xb[id + c * G.fstride] = zero;
      pb[id + c * G.fstride] = zero;
      acc += (c == 0 ? G.w[id] : (R)1) * cabs2(v);
    }
    loc += acc;
  }
  const double s = block_sum(loc, red);
  double tot;
  if (last_block_total(s, partials + (size_t)term * ntiles, counters + term, ntiles, tile, &tot, red)) {
    TermScalars& S = sc[term];
    S.gamma = tot;
    S.gamma0 = tot;
    S.beta = 0.0;
    S.a = 0.0;
    S.iters = 0;
    // zero right-hand side: x = 0 is exact; a non-finite one (NaN or Inf in
    // the input) stops the term at once with status 3 (reported as ENOCONV)
    S.status = !isfinite(tot) ? 3 : (tot == 0.0) ? 1 : 0;
  }
}

// t <- alpha_n p' + tau A p' with p' = a + beta b formed on the fly (nothing
// that a neighbouring tile reads is written here); dot1 = ||t||_W^2 and
// a = gamma / dot1.  beta is the term's CG beta, or 1 when unit_beta is set
// (the refinement step t = B (x + d)).
template <typename R, typename VA, typename VB>
__global__ void __launch_bounds__(THREADS) cg_apply_B(Geom<R> G, const VA* a, const VB* b, cplx<R>* t,
                                                      size_t vstride, size_t bstride, TermScalars* sc,
                                                      double* partials, unsigned* counters, int unit_beta) {
  __shared__ cplx<R> E[HY][HX], U[HY][HX], V[HY][HX];
  __shared__ double red[THREADS / 32];
  const int term = blockIdx.z;
  TermScalars& S = sc[term];
  if (S.status != 0) return;
  const int tile = blockIdx.y * G.tiles_x + blockIdx.x;
  const int ntiles = G.tiles_x * G.tiles_y;
  // per-point coefficients first, so their loads overlap the tile load
  constexpr int PP = TX * TY / THREADS;
  R Hp[PP], wp[PP];
#pragma unroll
  for (int q = 0; q < PP; ++q) {
    const int k = threadIdx.x + q * THREADS;
    const int i = blockIdx.x * TX + k % TX, j = blockIdx.y * TY + k / TX;
    const bool ok = i < G.nx && j < G.ny;
    const size_t id = ok ? (size_t)j * G.nx + i : 0;
    Hp[q] = G.H[id];
    wp[q] = G.w[id];
  }
  load_tile<R, true>(G, a + (size_t)term * vstride, b + (size_t)term * bstride, unit_beta ? (R)1 : (R)S.beta, E,
                     U, V);
  cplx<R>* tb = t + (size_t)term * vstride;
  const cplx<R> al = cvt<R>(S.alpha_n);
  R loc = 0;
#pragma unroll
  for (int q = 0; q < PP; ++q) {
    const int k = threadIdx.x + q * THREADS;
    const int li = k % TX + 1, lj = k / TX + 1;
    const int i = blockIdx.x * TX + li - 1, j = blockIdx.y * TY + lj - 1;
    if (i >= G.nx || j >= G.ny) continue;
    const size_t id = (size_t)j * G.nx + i;
    cplx<R> ae, au, av;
    apply_tA<R>(E, U, V, li, lj, Hp[q], G, ae, au, av);
    const cplx<R> te = cadd(cmul(al, E[lj][li]), ae);
    const cplx<R> tu = cadd(cmul(al, U[lj][li]), au);
    const cplx<R> tv = cadd(cmul(al, V[lj][li]), av);
    tb[id] = te;
    tb[id + G.fstride] = tu;
    tb[id + 2 * G.fstride] = tv;
    loc += wp[q] * cabs2(te) + cabs2(tu) + cabs2(tv);
  }
  const double s = block_sum(loc, red);
  double tot;
  if (last_block_total(s, partials + (size_t)term * ntiles, counters + term, ntiles, tile, &tot, red)) {
    S.dot1 = tot;
    S.a = tot > 0.0 ? S.gamma / tot : 0.0;
  }
}

// q = alpha_{-n} t - tau A t ; p <- r + beta p ; x += a p ; r -= a q ;
// gamma_new = ||r||_W^2 ; convergence.  Only t is read across tile borders.
template <typename R>
__global__ void __launch_bounds__(THREADS) cg_update(Geom<R> G, const cplx<R>* t, cplx<R>* p, cplx<R>* x,
                                                     cplx<R>* r, size_t vstride, TermScalars* sc, double* partials,
                                                     unsigned* counters, double rtol, int max_iters) {
  __shared__ cplx<R> E[HY][HX], U[HY][HX], V[HY][HX];
  __shared__ double red[THREADS / 32];
  const int term = blockIdx.z;
  TermScalars& S = sc[term];
  if (S.status != 0) return;
  const int tile = blockIdx.y * G.tiles_x + blockIdx.x;
  const int ntiles = G.tiles_x * G.tiles_y;
  cplx<R>* pb = p + (size_t)term * vstride;
  cplx<R>* xb = x + (size_t)term * vstride;
  cplx<R>* rb = r + (size_t)term * vstride;
  // pointwise operands first, so their loads overlap the tile load
  constexpr int PP = TX * TY / THREADS;
  cplx<R> xv[PP][3], rv[PP][3], pv[PP][3];
  R Hp[PP], wp[PP];
#pragma unroll
  for (int q = 0; q < PP; ++q) {
    const int k = threadIdx.x + q * THREADS;
    const int i = blockIdx.x * TX + k % TX, j = blockIdx.y * TY + k / TX;
    const bool ok = i < G.nx && j < G.ny;
    const size_t id = ok ? (size_t)j * G.nx + i : 0;
    Hp[q] = G.H[id];
    wp[q] = G.w[id];
#pragma unroll
    for (int c = 0; c < 3; ++c) {
      xv[q][c] = xb[id + c * G.fstride];
      rv[q][c] = rb[id + c * G.fstride];
      pv[q][c] = pb[id + c * G.fstride];
    }
  }
  load_tile<R, false>(G, t + (size_t)term * vstride, (const cplx<R>*)nullptr, (R)0, E, U, V);
  const cplx<R> am = cvt<R>(S.alpha_mn);
  const R a = (R)S.a, beta = (R)S.beta;
  R loc = 0;
#pragma unroll
  for (int q = 0; q < PP; ++q) {
    const int k = threadIdx.x + q * THREADS;
    const int li = k % TX + 1, lj = k / TX + 1;
    const int i = blockIdx.x * TX + li - 1, j = blockIdx.y * TY + lj - 1;
    if (i >= G.nx || j >= G.ny) continue;
    const size_t id = (size_t)j * G.nx + i;
    cplx<R> ae, au, av;
    apply_tA<R>(E, U, V, li, lj, Hp[q], G, ae, au, av);
    const cplx<R> qv[3] = {csub(cmul(am, E[lj][li]), ae), csub(cmul(am, U[lj][li]), au),
                           csub(cmul(am, V[lj][li]), av)};
    R acc = 0;
#pragma unroll
    for (int c = 0; c < 3; ++c) {
      const size_t o = id + c * G.fstride;
      const cplx<R> pn = mk(fma(beta, pv[q][c].x, rv[q][c].x), fma(beta, pv[q][c].y, rv[q][c].y));
      const cplx<R> xn = mk(fma(a, pn.x, xv[q][c].x), fma(a, pn.y, xv[q][c].y));
      const cplx<R> rn = mk(fma(-a, qv[c].x, rv[q][c].x), fma(-a, qv[c].y, rv[q][c].y));
      pb[o] = pn;
      xb[o] = xn;
      rb[o] = rn;
      acc += (c == 0 ? wp[q] : (R)1) * cabs2(rn);
    }
    loc += acc;
  }
  const double s = block_sum(loc, red);
  double tot;
  if (last_block_total(s, partials + (size_t)term * ntiles, counters + term, ntiles, tile, &tot, red)) {
    S.beta = S.gamma > 0.0 ? tot / S.gamma : 0.0;
    S.gamma = tot;
    S.iters += 1;
    if (!isfinite(tot))
      S.status = 3;  // a non-finite residual ends the term (reported as ENOCONV)
    else if (tot <= rtol * rtol * S.gamma0)
      S.status = 1;
    else if (S.iters >= max_iters)
      S.status = 2;
  }
}

// Refinement (FP64): x += d (pointwise) and r = f - B^* t with t = B (x + d);
// gamma = ||r||_W^2 ; outer convergence against gamma0 = ||f||_W^2.
__global__ void __launch_bounds__(THREADS) refine_residual(Geom<double> G, const double2* __restrict__ f,
                                                           int real_input, const double2* t, const float2* d,
                                                           double2* x, double2* r, size_t vstride, size_t dstride,
                                                           TermScalars* sc, double* partials, unsigned* counters,
                                                           double rtol, int max_outer) {
  __shared__ double2 E[HY][HX], U[HY][HX], V[HY][HX];
  __shared__ double red[THREADS / 32];
  const int term = blockIdx.z;
  TermScalars& S = sc[term];
  if (S.status != 0) return;
  const int tile = blockIdx.y * G.tiles_x + blockIdx.x;
  const int ntiles = G.tiles_x * G.tiles_y;
  load_tile<double, false>(G, t + (size_t)term * vstride, (const double2*)nullptr, 0.0, E, U, V);
  double2* xb = x + (size_t)term * vstride;
  double2* rb = r + (size_t)term * vstride;
  const float2* db = d + (size_t)term * dstride;
  const double2 am = S.alpha_mn;
  double loc = 0.0;
  for (int k = threadIdx.x; k < TX * TY; k += THREADS) {
    const int li = k % TX + 1, lj = k / TX + 1;
    const int i = blockIdx.x * TX + li - 1, j = blockIdx.y * TY + lj - 1;
    if (i >= G.nx || j >= G.ny) continue;
    const size_t id = (size_t)j * G.nx + i;
    double2 ae, au, av;
    apply_tA<double>(E, U, V, li, lj, G.H[id], G, ae, au, av);
    const double2 q[3] = {csub(cmul(am, E[lj][li]), ae), csub(cmul(am, U[lj][li]), au),
                          csub(cmul(am, V[lj][li]), av)};
#pragma unroll
    for (int c = 0; c < 3; ++c) {
      const size_t o = id + c * G.fstride;
      const float2 dv = db[o];
      const double2 xv = xb[o];
      xb[o] = mk(xv.x + (double)dv.x, xv.y + (double)dv.y);
      double2 fv = f[o];
      if (real_input) fv.y = 0.0;
      const double2 rv = csub(fv, q[c]);
      rb[o] = rv;
      loc += (c == 0 ? G.w[id] : 1.0) * cabs2(rv);
    }
  }
  const double s = block_sum(loc, red);
  double tot;
  if (last_block_total(s, partials + (size_t)term * ntiles, counters + term, ntiles, tile, &tot, red)) {
    S.gamma = tot;
    S.iters += 1;  // refinement steps
    if (!isfinite(tot))
      S.status = 3;
    else if (tot <= rtol * rtol * S.gamma0)
      S.status = 1;
    else if (S.iters >= max_outer)
      S.status = 2;
  }
}

// acc += sum over the batch of Gamma_n (C1 x - C2 tau A x), batch order fixed.
__global__ void __launch_bounds__(THREADS) cg_accumulate(Geom<double> G, const double2* x, size_t vstride,
                                                         int nbatch, const TermScalars* sc, double2* acc,
                                                         int first) {
  __shared__ double2 E[HY][HX], U[HY][HX], V[HY][HX];
  double2 s[2][3];
  for (int q = 0; q < 2; ++q)
    for (int c = 0; c < 3; ++c) s[q][c] = make_double2(0.0, 0.0);
  for (int b = 0; b < nbatch; ++b) {
    __syncthreads();
    load_tile<double, false>(G, x + (size_t)b * vstride, (const double2*)nullptr, 0.0, E, U, V);
    const double2 c1 = sc[b].gC1, c2 = sc[b].gC2;
    int q = 0;
    for (int k = threadIdx.x; k < TX * TY; k += THREADS, ++q) {
      const int li = k % TX + 1, lj = k / TX + 1;
      const int i = blockIdx.x * TX + li - 1, j = blockIdx.y * TY + lj - 1;
      if (i >= G.nx || j >= G.ny) continue;
      double2 ae, au, av;
      apply_tA<double>(E, U, V, li, lj, G.H[(size_t)j * G.nx + i], G, ae, au, av);
      s[q][0] = cadd(s[q][0], csub(cmul(c1, E[lj][li]), cmul(c2, ae)));
      s[q][1] = cadd(s[q][1], csub(cmul(c1, U[lj][li]), cmul(c2, au)));
      s[q][2] = cadd(s[q][2], csub(cmul(c1, V[lj][li]), cmul(c2, av)));
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

// Energy-weight scaling used by the adjoint: eta *= w (inverse: eta /= w).
__global__ void scale_eta(const double2* in, double2* out, const double* w, size_t nk, int inverse, int real_in) {
  const size_t i = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= 3 * nk) return;
  double2 v = in[i];
  if (real_in) v.y = 0.0;
  if (i < nk) {
    const double s = inverse ? 1.0 / w[i] : w[i];
    v.x *= s;
    v.y *= s;
  }
  out[i] = v;
}

__global__ void depth_tables(const double* H, size_t nk, double g, double* w64, float* H32, float* w32) {
  const size_t i = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= nk) return;
  const double w = g / H[i];
  w64[i] = w;
  H32[i] = (float)H[i];
  w32[i] = (float)w;
}

// ---- depth gradient ------------------------------------------------------------
// For one REXII term with x = N^{-1} f and y = N^{-1} W^{-1} G (both CG solves
// with N = B^* B), the term's two single-shift poles contribute
//   tau Re[ Gamma Q w conj((B y)_eta) div(B^* x) - Gamma P w conj((B^* y)_eta) div(B x) ]
// to dL/dH at each eta point (B = alpha_n + tau A, B^* = alpha_{-n} - tau A,
// w = g/H, P and Q the partial-fraction weights).  Stage 1 forms the u, v
// components of B^* x and B x and the eta components of B y and B^* y; stage 2
// takes the divergences and sums over the batch in a fixed order.

// out1 fields: (B* x)_u, (B* x)_v, (B y)_eta ; out2 fields: (B x)_u, (B x)_v, (B* y)_eta
__global__ void __launch_bounds__(THREADS) grad_stage1(Geom<double> G, const double2* xs, const double2* ys,
                                                       double2* out1, double2* out2, size_t vstride,
                                                       const TermScalars* sc) {
  __shared__ double2 E[HY][HX], U[HY][HX], V[HY][HX];
  const int term = blockIdx.z;
  const TermScalars& S = sc[term];
  const double2 al = S.alpha_n, am = S.alpha_mn;
  double2* o1 = out1 + (size_t)term * vstride;
  double2* o2 = out2 + (size_t)term * vstride;
  load_tile<double, false>(G, xs + (size_t)term * vstride, (const double2*)nullptr, 0.0, E, U, V);
  for (int k = threadIdx.x; k < TX * TY; k += THREADS) {
    const int li = k % TX + 1, lj = k / TX + 1;
    const int i = blockIdx.x * TX + li - 1, j = blockIdx.y * TY + lj - 1;
    if (i >= G.nx || j >= G.ny) continue;
    const size_t id = (size_t)j * G.nx + i;
    double2 ae, au, av;
    apply_tA<double>(E, U, V, li, lj, G.H[id], G, ae, au, av);
    o1[id] = csub(cmul(am, U[lj][li]), au);
    o1[id + G.fstride] = csub(cmul(am, V[lj][li]), av);
    o2[id] = cadd(cmul(al, U[lj][li]), au);
    o2[id + G.fstride] = cadd(cmul(al, V[lj][li]), av);
  }
  __syncthreads();
  load_tile<double, false>(G, ys + (size_t)term * vstride, (const double2*)nullptr, 0.0, E, U, V);
  for (int k = threadIdx.x; k < TX * TY; k += THREADS) {
    const int li = k % TX + 1, lj = k / TX + 1;
    const int i = blockIdx.x * TX + li - 1, j = blockIdx.y * TY + lj - 1;
    if (i >= G.nx || j >= G.ny) continue;
    const size_t id = (size_t)j * G.nx + i;
    double2 ae, au, av;
    apply_tA<double>(E, U, V, li, lj, G.H[id], G, ae, au, av);
    o1[id + 2 * G.fstride] = cadd(cmul(al, E[lj][li]), ae);
    o2[id + 2 * G.fstride] = csub(cmul(am, E[lj][li]), ae);
  }
}

__global__ void grad_stage2(Geom<double> G, const double2* out1, const double2* out2, size_t vstride, int nbatch,
                            const TermScalars* sc, double tau, double* grad) {
  const size_t id = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (id >= G.fstride) return;
  const int i = (int)(id % G.nx), j = (int)(id / G.nx);
  const size_t iw = (size_t)j * G.nx + (i == 0 ? G.nx - 1 : i - 1);
  const size_t js = (size_t)(j == 0 ? G.ny - 1 : j - 1) * G.nx + i;
  const size_t F = G.fstride;
  const double w = G.w[id];
  double acc = 0.0;
  for (int b = 0; b < nbatch; ++b) {
    const double2* a = out1 + (size_t)b * vstride;
    const double2* c = out2 + (size_t)b * vstride;
    const double2 div1 = cadd(mk(G.idx * (a[id].x - a[iw].x), G.idx * (a[id].y - a[iw].y)),
                              mk(G.idy * (a[F + id].x - a[F + js].x), G.idy * (a[F + id].y - a[F + js].y)));
    const double2 div2 = cadd(mk(G.idx * (c[id].x - c[iw].x), G.idx * (c[id].y - c[iw].y)),
                              mk(G.idy * (c[F + id].x - c[F + js].x), G.idy * (c[F + id].y - c[F + js].y)));
    const double2 s1 = a[2 * F + id], s2 = c[2 * F + id];
    const double2 t1 = cmul(sc[b].gQ, cmul(mk(s1.x, -s1.y), div1));
    const double2 t2 = cmul(sc[b].gP, cmul(mk(s2.x, -s2.y), div2));
    acc += w * (t1.x - t2.x);
  }
  grad[id] += tau * acc;
}

// ---- workspace layout ------------------------------------------------------

struct KLayout {
  size_t acc_off, tmp_off, total;
  size_t v64_off, v64_bytes;  // FP64 vectors per term: x, r, p, t
  size_t v32_off, v32_bytes;  // FP32 vectors per term (mixed): d, r, p, t
  size_t sc_off, sc32_off, part_off, cnt_off;
  int batch, ntiles;
};

size_t al256(size_t v) { return (v + 255) / 256 * 256; }

KLayout layout(const KrylovSettings* k, int nterms, int form) {
  KLayout L{};
  const size_t nk = (size_t)k->nx * k->ny;
  L.batch = std::max(1, std::min(k->term_batch, nterms));
  L.ntiles = ((k->nx + TX - 1) / TX) * ((k->ny + TY - 1) / TY);
  size_t off = 0;
  L.acc_off = off;
  off += al256(3 * nk * sizeof(double2));
  L.tmp_off = off;  // adjoint: scaled input
  off += al256(3 * nk * sizeof(double2));
  L.v64_off = off;
  L.v64_bytes = al256(3 * nk * sizeof(double2));
  off += 5 * (size_t)L.batch * L.v64_bytes;  // x, r, p, t and a saved solution (depth gradient)
  L.v32_off = off;
  L.v32_bytes = al256(3 * nk * sizeof(float2));
  if (form == REXI_FORM_MIXED) off += 4 * (size_t)L.batch * L.v32_bytes;
  L.sc_off = off;
  off += al256((size_t)L.batch * sizeof(TermScalars));
  L.sc32_off = off;
  off += al256((size_t)L.batch * sizeof(TermScalars));
  L.part_off = off;
  off += al256((size_t)L.batch * L.ntiles * sizeof(double));
  L.cnt_off = off;
  off += al256((size_t)L.batch * sizeof(unsigned));
  L.total = off;
  return L;
}

int n_terms_for(int M, int real_input) {
  const int N = M + kL;
  return real_input ? N + 1 : 2 * N + 1;
}

template <typename R>
Geom<R> make_geom(const KrylovSettings* k, double tau, const R* H, const R* w) {
  Geom<R> G;
  G.nx = k->nx;
  G.ny = k->ny;
  G.tiles_x = (k->nx + TX - 1) / TX;
  G.tiles_y = (k->ny + TY - 1) / TY;
  G.fstride = (size_t)k->nx * k->ny;
  const double idx = k->nx / k->Lx, idy = k->ny / k->Ly;
  G.tdx = (R)(tau * idx);
  G.tdy = (R)(tau * idy);
  G.tgdx = (R)(tau * k->g * idx);
  G.tgdy = (R)(tau * k->g * idy);
  G.tf4 = (R)(0.25 * tau * k->f);
  G.idx = (R)idx;
  G.idy = (R)idy;
  G.H = H;
  G.w = w;
  return G;
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
  const size_t nk = (size_t)nx * ny;
  char* mem = nullptr;
  const size_t bytes = al256(nk * sizeof(double)) + 2 * al256(nk * sizeof(float)) + 2 * al256(nk * sizeof(float2));
  if (cudaMalloc(&mem, bytes) != cudaSuccess) {
    set_last_error("cudaMalloc of the depth tables failed");
    return REXI_ENOMEM;
  }
  k->dev_state = mem;
  k->w64 = reinterpret_cast<double*>(mem);
  k->H32 = reinterpret_cast<float*>(mem + al256(nk * sizeof(double)));
  k->w32 = reinterpret_cast<float*>(mem + al256(nk * sizeof(double)) + al256(nk * sizeof(float)));
  k->Hdf = reinterpret_cast<float2*>(mem + al256(nk * sizeof(double)) + 2 * al256(nk * sizeof(float)));
  k->wdf = reinterpret_cast<float2*>(mem + al256(nk * sizeof(double)) + 2 * al256(nk * sizeof(float)) +
                                     al256(nk * sizeof(float2)));
  if (cudaMallocHost(reinterpret_cast<void**>(&k->pinned), 8 * sizeof(double)) != cudaSuccess ||
      cudaEventCreateWithFlags(&k->ev[0], cudaEventDisableTiming) != cudaSuccess ||
      cudaEventCreateWithFlags(&k->ev[1], cudaEventDisableTiming) != cudaSuccess) {
    set_last_error("pinned buffer or event creation failed");
    return REXI_ECUDA;
  }
  depth_tables<<<(unsigned)((nk + 255) / 256), 256>>>(depth, nk, g, k->w64, k->H32, k->w32);
  if (lanczos_tables(k) != REXI_OK) return REXI_ECUDA;
  if (cudaDeviceSynchronize() != cudaSuccess) {
    set_last_error("depth table kernel failed");
    return REXI_ECUDA;
  }
  return REXI_OK;
}

void krylov_destroy(KrylovSettings* k) {
  if (k->dev_state) cudaFree(k->dev_state);
  k->dev_state = nullptr;
  if (k->pinned) cudaFreeHost(k->pinned);
  k->pinned = nullptr;
  for (auto& e : k->ev) {
    if (e) cudaEventDestroy(e);
    e = nullptr;
  }
}

size_t krylov_workspace_bytes(const KrylovSettings* k, int M, int real_input, int form) {
  if (k->method == 1) return lanczos_workspace_bytes(k, M, real_input);
  return layout(k, n_terms_for(M, real_input), form).total;
}

size_t krylov_grad_workspace_bytes(const KrylovSettings* k, int M, int real_input, int form, double h) {
  if (k->method == 1 && real_input) return lanczos_grad_workspace_bytes(k, M, h);
  return layout(k, n_terms_for(M, real_input), form).total;
}

namespace {

// One call of the Krylov path: the term list, the carve-up of the workspace
// and the CG driver for one batch of terms (FP64, or FP32 with FP64
// refinement).  The solution of the batch's pair systems is left in X.
struct KrylovRun {
  KrylovSettings* k = nullptr;
  bool mixed = false;
  cudaStream_t s = nullptr;
  const KrylovHooks* hooks = nullptr;
  KLayout L{};
  char* base = nullptr;
  double2 *acc = nullptr, *tmp = nullptr, *X = nullptr, *R = nullptr, *P = nullptr, *T = nullptr, *XS = nullptr;
  float2 *D32 = nullptr, *R32 = nullptr, *P32 = nullptr, *T32 = nullptr;
  size_t vs64 = 0, vs32 = 0;
  TermScalars *dsc = nullptr, *dsc32 = nullptr;
  double* partials = nullptr;
  unsigned* counters = nullptr;
  Geom<double> G{};
  Geom<float> G32{};
  std::vector<TermScalars> terms, hs, hs32;
  int worst_iters = 0, unconverged = 0, nonfinite = 0;
  int64_t term_iters = 0;
  double worst_res = 0.0;
  static constexpr int check_every = 16;

  void mark(int i) {
    if (hooks && hooks->mark) hooks->mark(hooks->ctx, i, s);
  }
  void count(int64_t n) {
    if (hooks && hooks->launches) *hooks->launches += n;
  }

  rexi_status setup(KrylovSettings* kk, int form, double h, int M, double tau, int real_input, int tb, int te,
                    void* ws, size_t ws_bytes, cudaStream_t st, const KrylovHooks* hk) {
    k = kk;
    s = st;
    hooks = hk;
    if (form != REXI_FORM_FP64 && form != REXI_FORM_MIXED) {
      set_last_error("variable-depth path: the plain form is Fourier-path only");
      return REXI_EUNSUPPORTED;
    }
    mixed = form == REXI_FORM_MIXED;
    const int N = M + kL;
    if (te < 0 || te > N + 1) te = N + 1;
    if (tb < 0 || tb > te) {
      set_last_error("bad term range");
      return REXI_EINVAL;
    }
    // n = 0..N (real input, Gamma) or -N..N, restricted to |n| in [tb, te)
    TermSet ts;
    rexii_terms(M, h, &ts);
    const double hmu = h * ts.mu;
    for (int n = real_input ? 0 : -N; n <= N; ++n) {
      const int an = n < 0 ? -n : n;
      if (an < tb || an >= te) continue;
      const int i = n + N;
      const double gam = (real_input && n > 0) ? 2.0 : 1.0;
      TermScalars t;
      memset(&t, 0, sizeof(t));
      t.alpha_n = make_double2(hmu, h * n);
      t.alpha_mn = make_double2(hmu, -h * n);
      // C1 = c1 h mu + c2 h n,  C2 = i c2
      const double C1r = ts.c1re[i] * hmu + ts.c2re[i] * h * n, C1i = ts.c1im[i] * hmu + ts.c2im[i] * h * n;
      const double C2r = -ts.c2im[i], C2i = ts.c2re[i];
      t.gC1 = make_double2(gam * C1r, gam * C1i);
      t.gC2 = make_double2(gam * C2r, gam * C2i);
      // P = (C1 - C2 alpha_{-n}) / (2 h mu),  Q = (C1 + C2 alpha_n) / (2 h mu)
      const double inv2 = 1.0 / (2.0 * hmu), hn = h * n;
      t.gP = make_double2(gam * (C1r - (C2r * hmu + C2i * hn)) * inv2, gam * (C1i - (-C2r * hn + C2i * hmu)) * inv2);
      t.gQ = make_double2(gam * (C1r + (C2r * hmu - C2i * hn)) * inv2, gam * (C1i + (C2r * hn + C2i * hmu)) * inv2);
      terms.push_back(t);
    }
    L = layout(k, (int)std::max<size_t>(terms.size(), 1), form);
    if (ws_bytes < L.total) {
      set_last_error("workspace too small for the variable-depth path");
      return REXI_ENOMEM;
    }
    base = static_cast<char*>(ws);
    acc = reinterpret_cast<double2*>(base + L.acc_off);
    tmp = reinterpret_cast<double2*>(base + L.tmp_off);
    vs64 = L.v64_bytes / sizeof(double2);
    X = reinterpret_cast<double2*>(base + L.v64_off);
    R = X + (size_t)L.batch * vs64;
    P = X + 2 * (size_t)L.batch * vs64;
    T = X + 3 * (size_t)L.batch * vs64;
    XS = X + 4 * (size_t)L.batch * vs64;
    vs32 = L.v32_bytes / sizeof(float2);
    D32 = reinterpret_cast<float2*>(base + L.v32_off);
    R32 = D32 + (size_t)L.batch * vs32;
    P32 = D32 + 2 * (size_t)L.batch * vs32;
    T32 = D32 + 3 * (size_t)L.batch * vs32;
    dsc = reinterpret_cast<TermScalars*>(base + L.sc_off);
    dsc32 = reinterpret_cast<TermScalars*>(base + L.sc32_off);
    partials = reinterpret_cast<double*>(base + L.part_off);
    counters = reinterpret_cast<unsigned*>(base + L.cnt_off);
    G = make_geom<double>(k, tau, k->depth, k->w64);
    G32 = make_geom<float>(k, tau, k->H32, k->w32);
    hs.resize(L.batch);
    hs32.resize(L.batch);
    cudaError_t e = cudaMemsetAsync(counters, 0, (size_t)L.batch * sizeof(unsigned), s);
    if (e != cudaSuccess) {
      set_last_error(cudaGetErrorString(e));
      return REXI_ECUDA;
    }
    return REXI_OK;
  }

  // CG iterations on (sc, vectors) until every term of the batch has stopped.
  template <typename Rt>
  cudaError_t run_cg(const Geom<Rt>& geom, cplx<Rt>* Xv, cplx<Rt>* Rv, cplx<Rt>* Pv, cplx<Rt>* Tv, size_t vs,
                     TermScalars* sc, int nb, double rtol, std::vector<TermScalars>& host) {
    dim3 grid(geom.tiles_x, geom.tiles_y, nb);
    int it = 0;
    for (;;) {
      for (int c = 0; c < check_every; ++c) {
        cg_apply_B<Rt><<<grid, THREADS, 0, s>>>(geom, Rv, Pv, Tv, vs, vs, sc, partials, counters, 0);
        cg_update<Rt><<<grid, THREADS, 0, s>>>(geom, Tv, Pv, Xv, Rv, vs, sc, partials, counters, rtol, k->max_iters);
      }
      count(2 * check_every);
      it += check_every;
      cudaError_t err = cudaGetLastError();
      if (err == cudaSuccess)
        err = cudaMemcpyAsync(host.data(), sc, nb * sizeof(TermScalars), cudaMemcpyDeviceToHost, s);
      if (err == cudaSuccess) err = cudaStreamSynchronize(s);
      if (err != cudaSuccess) return err;
      bool done = true;
      for (int b = 0; b < nb; ++b)
        if (host[b].status == 0) done = false;
      if (done || it > k->max_iters + check_every) break;
    }
    for (int b = 0; b < nb; ++b) term_iters += host[b].iters;
    return cudaSuccess;
  }

  // Solves the pair systems of terms [b0, b0 + nb) for the right-hand side rhs.
  cudaError_t solve_batch(size_t b0, int nb, const double2* rhs, int real_rhs) {
    cudaError_t e = cudaMemcpyAsync(dsc, &terms[b0], nb * sizeof(TermScalars), cudaMemcpyHostToDevice, s);
    if (e == cudaSuccess) e = cudaMemcpyAsync(dsc32, &terms[b0], nb * sizeof(TermScalars), cudaMemcpyHostToDevice, s);
    if (e != cudaSuccess) return e;
    mark(1);
    dim3 grid(G.tiles_x, G.tiles_y, nb);
    cg_init<double, double2><<<grid, THREADS, 0, s>>>(G, rhs, real_rhs, X, R, P, vs64, 0, dsc, nullptr, partials,
                                                      counters);
    count(1);
    mark(2);
    if (!mixed) {
      e = run_cg<double>(G, X, R, P, T, vs64, dsc, nb, k->rtol, hs);
      if (e != cudaSuccess) return e;
    } else {
      // iterative refinement: FP32 CG on N d = r, then x += d, r = f - N x in FP64
      for (int outer = 0;; ++outer) {
        cg_init<float, double2><<<grid, THREADS, 0, s>>>(G32, R, 0, D32, R32, P32, vs32, vs64, dsc32, dsc, partials,
                                                         counters);
        count(1);
        e = run_cg<float>(G32, D32, R32, P32, T32, vs32, dsc32, nb, k->inner_rtol, hs32);
        if (e != cudaSuccess) return e;
        cg_apply_B<double><<<grid, THREADS, 0, s>>>(G, X, D32, T, vs64, vs32, dsc, partials, counters, 1);
        refine_residual<<<grid, THREADS, 0, s>>>(G, rhs, real_rhs, T, D32, X, R, vs64, vs32, dsc, partials, counters,
                                                 k->rtol, k->max_outer);
        count(2);
        e = cudaGetLastError();
        if (e == cudaSuccess) e = cudaMemcpyAsync(hs.data(), dsc, nb * sizeof(TermScalars), cudaMemcpyDeviceToHost, s);
        if (e == cudaSuccess) e = cudaStreamSynchronize(s);
        if (e != cudaSuccess) return e;
        bool done = true;
        for (int b = 0; b < nb; ++b)
          if (hs[b].status == 0) done = false;
        if (done || outer > k->max_outer) break;
      }
    }
    mark(3);
    for (int b = 0; b < nb; ++b) {
      worst_iters = std::max(worst_iters, mixed ? hs32[b].iters : hs[b].iters);
      if (hs[b].status != 1) ++unconverged;
      if (hs[b].status == 3 || (mixed && hs32[b].status == 3)) ++nonfinite;
      if (hs[b].gamma0 > 0) worst_res = std::max(worst_res, sqrt(hs[b].gamma / hs[b].gamma0));
    }
    return cudaSuccess;
  }

  void fill_info(rexi_step_info* info, int M, int real_input) const {
    if (!info) return;
    const int N = M + kL;
    memset(info, 0, sizeof(*info));
    info->N = N;
    info->n_terms = n_terms_for(M, real_input);
    info->n_poles = real_input ? 2 * (N + 1) : 2 * (2 * N + 1);
    info->krylov_iters = worst_iters;
    info->krylov_unconverged = unconverged;
    info->krylov_max_rel_res = worst_res;
    info->krylov_term_iters = term_iters;
  }
};

rexi_status cuda_status(cudaError_t e) {
  set_last_error(cudaGetErrorString(e));
  return REXI_ECUDA;
}

bool overlaps(const void* a, const void* b, size_t bytes) {
  return (const char*)a < (const char*)b + bytes && (const char*)b < (const char*)a + bytes;
}

}  // namespace

rexi_status krylov_step(KrylovSettings* k, int form, double h, int M, const void* in, void* out, double dt,
                        int real_input, int term_begin, int term_end, void* ws, size_t ws_bytes, cudaStream_t s,
                        rexi_step_info* info, bool adjoint, const KrylovHooks& hooks) {
  if (k->method == 1)
    return krylov_step_lanczos(k, form, h, M, in, out, dt, real_input, term_begin, term_end, ws, ws_bytes, s, info,
                               adjoint, hooks);
  const size_t nk = (size_t)k->nx * k->ny, n3 = 3 * nk;
  if (overlaps(in, out, n3 * sizeof(double2))) {
    set_last_error("variable-depth path: input and output must not overlap");
    return REXI_EINVAL;
  }
  KrylovRun run;
  // adjoint: r(tau A)^H = r(tau A^T) = W r(-tau A) W^{-1} with W = diag(g/H, 1, 1)
  rexi_status st = run.setup(k, form, h, M, adjoint ? -dt : dt, real_input, term_begin, term_end, ws, ws_bytes, s,
                             &hooks);
  if (st != REXI_OK) return st;
  const double2* src = static_cast<const double2*>(in);
  const unsigned ebl = (unsigned)((n3 + 255) / 256);
  cudaError_t e = cudaSuccess;
  if (adjoint) {
    scale_eta<<<ebl, 256, 0, s>>>(src, run.tmp, k->w64, nk, 1, real_input);
    run.count(1);
    src = run.tmp;
  }
  if (run.terms.empty()) e = cudaMemsetAsync(run.acc, 0, n3 * sizeof(double2), s);
  for (size_t b0 = 0; b0 < run.terms.size() && e == cudaSuccess; b0 += run.L.batch) {
    const int nb = (int)std::min<size_t>(run.L.batch, run.terms.size() - b0);
    run.mark(0);
    e = run.solve_batch(b0, nb, src, real_input);
    if (e != cudaSuccess) break;
    cg_accumulate<<<dim3(run.G.tiles_x, run.G.tiles_y, 1), THREADS, 0, s>>>(run.G, run.X, run.vs64, nb, run.dsc,
                                                                            run.acc, b0 == 0 ? 1 : 0);
    run.count(1);
    e = cudaGetLastError();
    run.mark(4);
  }
  if (e != cudaSuccess) return cuda_status(e);
  double2* o = static_cast<double2*>(out);
  if (adjoint) {
    scale_eta<<<ebl, 256, 0, s>>>(run.acc, o, k->w64, nk, 0, 0);
    run.count(1);
    if (real_input) {
      finish_output<<<ebl, 256, 0, s>>>(o, o, n3, 1);
      run.count(1);
    }
  } else {
    finish_output<<<ebl, 256, 0, s>>>(run.acc, o, n3, real_input);
    run.count(1);
  }
  if ((e = cudaGetLastError()) != cudaSuccess) return cuda_status(e);
  if (info) run.fill_info(info, M, real_input);
  if (run.unconverged > 0) {
    set_last_error(run.nonfinite > 0 ? "variable-depth path: non-finite residual (NaN or Inf in the input?)"
                                     : "variable-depth path: some terms reached the iteration cap");
    return REXI_ENOCONV;
  }
  return REXI_OK;
}

rexi_status krylov_grad_depth(KrylovSettings* k, int form, double h, int M, const void* f_in, const void* g_out,
                              double* grad_depth, double dt, int real_input, void* ws, size_t ws_bytes,
                              cudaStream_t s, rexi_step_info* info, const KrylovHooks& hooks) {
  if (k->method == 1 && real_input)
    return krylov_grad_depth_lanczos(k, form, h, M, f_in, g_out, grad_depth, dt, ws, ws_bytes, s, info, hooks);
  const size_t nk = (size_t)k->nx * k->ny, n3 = 3 * nk;
  KrylovRun run;
  rexi_status st = run.setup(k, form, h, M, dt, real_input, 0, -1, ws, ws_bytes, s, &hooks);
  if (st != REXI_OK) return st;
  const unsigned ebl = (unsigned)((n3 + 255) / 256);
  // adjoint right-hand side W^{-1} G
  scale_eta<<<ebl, 256, 0, s>>>(static_cast<const double2*>(g_out), run.tmp, k->w64, nk, 1, real_input);
  run.count(1);
  cudaError_t e = cudaGetLastError();
  for (size_t b0 = 0; b0 < run.terms.size() && e == cudaSuccess; b0 += run.L.batch) {
    const int nb = (int)std::min<size_t>(run.L.batch, run.terms.size() - b0);
    run.mark(0);
    e = run.solve_batch(b0, nb, static_cast<const double2*>(f_in), real_input);  // x = N^{-1} f
    if (e == cudaSuccess)
      e = cudaMemcpyAsync(run.XS, run.X, (size_t)nb * run.vs64 * sizeof(double2), cudaMemcpyDeviceToDevice, s);
    if (e == cudaSuccess) e = run.solve_batch(b0, nb, run.tmp, 0);  // y = N^{-1} W^{-1} G
    if (e != cudaSuccess) break;
    grad_stage1<<<dim3(run.G.tiles_x, run.G.tiles_y, nb), THREADS, 0, s>>>(run.G, run.XS, run.X, run.R, run.P,
                                                                           run.vs64, run.dsc);
    grad_stage2<<<(unsigned)((nk + 255) / 256), 256, 0, s>>>(run.G, run.R, run.P, run.vs64, nb, run.dsc, dt,
                                                             grad_depth);
    run.count(2);
    e = cudaGetLastError();
    run.mark(4);
  }
  if (e != cudaSuccess) return cuda_status(e);
  if (info) run.fill_info(info, M, real_input);
  if (run.unconverged > 0) {
    set_last_error("depth gradient: some terms reached the iteration cap");
    return REXI_ENOCONV;
  }
  return REXI_OK;
}

}  // namespace rexi
