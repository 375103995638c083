// Variable-depth path, shared-Krylov method: every single-shift pole of the
// rational approximation uses one Lanczos basis.
//
// With K = -i tau A, which is self-adjoint in the energy inner product
// <a, b>_W = sum (g/H, 1, 1) conj(a) b (A is skew there), each pole term is
//   (tau A - z_j)^{-1} f = -i (K + i z_j)^{-1} f,
// a shifted system of one self-adjoint operator.  The Krylov space
// span{f, K f, K^2 f, ...} does not depend on the shift, so k Lanczos steps
// (K V_k = V_k T_k + b_k v_k e_{k-1}^T, T_k real symmetric tridiagonal) give
// every pole its Galerkin solution x_j = ||f|| V_k (T_k + s_j)^{-1} e_0,
// s_j = i z_j, at once.  The weighted sum over poles is
//   sum_j beta_j (tau A - z_j)^{-1} f ~ V_k c,
//   c = -i ||f|| sum_j beta_j (T_k + s_j)^{-1} e_0.
// Error: every pole's residual is a multiple of v_k, so the error of the sum
// is -i ||f|| b_k phi(K) v_k with the rational function
//   phi(l) = sum_j beta_j y_j / (l + s_j),  y_j = e_{k-1}^T (T_k + s_j)^{-1} e_0,
// and ||error|| <= ||f|| b_k max |phi| over the spectrum of K, which lies in
// [-tau rho, tau rho] (rho >= ||A||_W).  For real input the step keeps only the
// real part, which is the same sum over the conjugate-closed pole set
// {z_j, conj z_j} with weights {beta_j / 2, conj beta_j / 2}; the bound uses
// that set (its phi has no cancelling imaginary remainder).  With a_j = 0 its
// phi is (phi(l) + (-1)^(k-1) conj(phi(-l))) / 2 in terms of the original
// set's, so the device evaluates the original set on a symmetric grid.  The
// bound is evaluated every kChunk steps by sampling l at spacing d / 4 or
// finer, d = h |mu| the distance of every pole from the real axis, first on
// every 8th sample and, once that passes, on all of them.
//
// One fused kernel per Lanczos step (v_j formed on the fly from w'_{j-1} and
// v_{j-1}; both inner products of the step in one deterministic reduction,
// b_{j+1}^2 = ||w'_j||^2 - a_j^2).  For real input the vectors alternate
// between purely real and purely imaginary (a_j = 0), and the step runs in
// real arithmetic on the unnormalised vectors alone.  Vectors that fit in the caller's extra
// workspace are kept; the rest of the basis is regenerated in a second pass
// with the stored scalars (same operations in the same order, so the same
// vectors).  FP64 throughout.
#include <math.h>
#include <string.h>

#include <algorithm>
#include <complex>
#include <type_traits>
#include <vector>

#include "dfloat.cuh"
#include "internal.h"
#include "krylov.h"
#include "partials.cuh"

namespace rexi {
namespace {

constexpr int TX = 32, TY = 16, THREADS = 256, HX = TX + 2, HY = TY + 2;
constexpr int kChunk = 16;         // Lanczos steps between convergence checks
constexpr int kCoarse = 8;         // coarse check: every 8th sample of the fine grid
constexpr int kMinScratchPoles = 32;
// Threads per block of the per-pole recurrences (one thread per pole, a
// chain of dependent FP64 operations each): one warp per block spreads the
// poles over as many SMs, and so FP64 pipes, as there are warps.
constexpr int kPoleThreads = 32;

struct LGeom {
  int nx, ny, tiles_x, tiles_y;
  size_t fstride;
  double tdx, tdy, tgdx, tgdy, tf4;  // tau folded in
  const double* H;
  const double* w;
};

__device__ __forceinline__ double2 ladd(double2 a, double2 b) { return make_double2(a.x + b.x, a.y + b.y); }
__device__ __forceinline__ double2 lsub(double2 a, double2 b) { return make_double2(a.x - b.x, a.y - b.y); }

__device__ __forceinline__ size_t lidx(const LGeom& G, int i, int j) {
  i = G.nx > TX ? (i < 0 ? i + G.nx : (i >= G.nx ? i - G.nx : i)) : (i + G.nx) % G.nx;
  j = G.ny > TY ? (j < 0 ? j + G.ny : (j >= G.ny ? j - G.ny : j)) : (j + G.ny) % G.ny;
  return (size_t)j * G.nx + i;
}

// Two block sums at once (result valid in thread 0).
__device__ __forceinline__ double2 lblock_sum2(double2 v, double2* red) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) {
    v.x += __shfl_down_sync(0xffffffffu, v.x, o);
    v.y += __shfl_down_sync(0xffffffffu, v.y, o);
  }
  const int w = threadIdx.x >> 5, l = threadIdx.x & 31;
  __syncthreads();
  if (l == 0) red[w] = v;
  __syncthreads();
  double2 s = make_double2(0.0, 0.0);
  if (threadIdx.x == 0)
    for (int i = 0; i < THREADS / 32; ++i) s = ladd(s, red[i]);
  return s;
}

// Deterministic cross-block sum of two values (fixed order), finished by the
// last block to arrive; returns true in that block's thread 0.
__device__ __forceinline__ bool llast_block2(double2 mine, double2* partials, unsigned* counter, int ntiles, int tile,
                                            double2* total, double2* red) {
  __shared__ bool is_last;
  if (threadIdx.x == 0) {
    partials[tile] = mine;
    __threadfence();
    is_last = atomicAdd(counter, 1u) == (unsigned)ntiles - 1;
  }
  __syncthreads();
  if (!is_last) return false;
  __threadfence();
  double2 s = strided_partial_sum(partials, ntiles, threadIdx.x, THREADS, make_double2(0.0, 0.0),
                                  [](double2 a, double2 b) { return ladd(a, b); });
  s = lblock_sum2(s, red);
  if (threadIdx.x == 0) {
    *total = s;
    *counter = 0u;
  }
  return threadIdx.x == 0;
}

__device__ __forceinline__ double safe_inv(double b) { return b > 0.0 ? 1.0 / b : 0.0; }

// Vector arithmetic for the two representations of a Lanczos vector: complex
// (double2) in general, and real (double) for real input, where the vectors
// alternate between purely real and purely imaginary (v_j = i^j u_j with u_j
// real, a_j = 0) and the recurrence becomes u_{j+1} b_{j+1} = -tau A u_j + b_j u_{j-1}.
__device__ __forceinline__ double vadd(double a, double b) { return a + b; }
__device__ __forceinline__ double2 vadd(double2 a, double2 b) { return ladd(a, b); }
__device__ __forceinline__ double vsub(double a, double b) { return a - b; }
__device__ __forceinline__ double2 vsub(double2 a, double2 b) { return lsub(a, b); }
__device__ __forceinline__ double vscal(double s, double a) { return s * a; }
__device__ __forceinline__ double2 vscal(double s, double2 a) { return make_double2(s * a.x, s * a.y); }
__device__ __forceinline__ double vfma(double s, double a, double b) { return fma(s, a, b); }
__device__ __forceinline__ double2 vfma(double s, double2 a, double2 b) {
  return make_double2(fma(s, a.x, b.x), fma(s, a.y, b.y));
}
__device__ __forceinline__ double vnrm2(double a) { return a * a; }
__device__ __forceinline__ double vnrm2(double2 a) { return fma(a.x, a.x, a.y * a.y); }
__device__ __forceinline__ double vredot(double2 a, double2 b) { return fma(a.x, b.x, a.y * b.y); }
template <typename T>
__device__ __forceinline__ T vzero() {
  return T{};
}
// acc += c v; the real form takes c' = Re(i^j c), the real part of
// c_j v_j = c_j i^j u_j
__device__ __forceinline__ double2 vcfma(double2 c, double2 v, double2 a) {
  return make_double2(fma(c.x, v.x, fma(-c.y, v.y, a.x)), fma(c.x, v.y, fma(c.y, v.x, a.y)));
}
__device__ __forceinline__ double real_coeff(double2 c, int j) {
  switch (j & 3) {
    case 0: return c.x;
    case 1: return -c.y;
    case 2: return -c.x;
    default: return c.y;
  }
}
template <typename T>
__device__ __forceinline__ T cvec_at(const double2* cvec, int j);
template <>
__device__ __forceinline__ double2 cvec_at<double2>(const double2* cvec, int j) {
  return cvec[j];
}
template <typename T>
__device__ __forceinline__ T from_in(double2 v);
template <>
__device__ __forceinline__ double from_in<double>(double2 v) {
  return v.x;
}
template <>
__device__ __forceinline__ double2 from_in<double2>(double2 v) {
  return v;
}
__device__ __forceinline__ double2 to_out(double v) { return make_double2(v, 0.0); }
__device__ __forceinline__ double2 to_out(double2 v) { return v; }

// s tau A t at a tile point (C-grid stencil: eta row -H div, momentum rows
// -g grad eta and the four-point Coriolis average); s is folded into the
// coefficients (c = s tau / dx etc.).
struct StencilCoef {
  double cdx, cdy, cgdx, cgdy, cf4;
};
template <typename T>
__device__ __forceinline__ void apply_sA(const T (*E)[HX], const T (*U)[HX], const T (*V)[HX], int li, int lj,
                                         double Hij, const StencilCoef& c, T out[3]) {
  const double hx = -Hij * c.cdx, hy = -Hij * c.cdy;
  out[0] = vfma(hx, vsub(U[lj][li], U[lj][li - 1]), vscal(hy, vsub(V[lj][li], V[lj - 1][li])));
  const T v4 = vadd(vadd(V[lj][li], V[lj][li + 1]), vadd(V[lj - 1][li], V[lj - 1][li + 1]));
  out[1] = vfma(c.cf4, v4, vscal(-c.cgdx, vsub(E[lj][li + 1], E[lj][li])));
  const T u4 = vadd(vadd(U[lj][li], U[lj][li - 1]), vadd(U[lj + 1][li], U[lj + 1][li - 1]));
  out[2] = vfma(-c.cf4, u4, vscal(-c.cgdy, vsub(E[lj + 1][li], E[lj][li])));
}
// K = -i (tau A) applied to the scaled-stencil output
__device__ __forceinline__ double2 op_out(double2 a) { return make_double2(a.y, -a.x); }

// f0 = in (eta / w for the adjoint), imaginary parts dropped for real input;
// beta[0] = ||f0||_W.
template <typename T>
__global__ void __launch_bounds__(THREADS) lz_init(LGeom G, const double2* in, int adjoint, T* f0, double* beta,
                                                   double* invb, double2* partials, unsigned* counter) {
  __shared__ double2 red[THREADS / 32];
  const int tile = blockIdx.y * G.tiles_x + blockIdx.x;
  double loc = 0.0;
  for (int k = threadIdx.x; k < TX * TY; k += THREADS) {
    const int i = blockIdx.x * TX + k % TX, j = blockIdx.y * TY + k / TX;
    if (i >= G.nx || j >= G.ny) continue;
    const size_t id = (size_t)j * G.nx + i;
    for (int c = 0; c < 3; ++c) {
      T v = from_in<T>(in[id + c * G.fstride]);
      if (adjoint && c == 0) v = vscal(1.0 / G.w[id], v);
      f0[id + c * G.fstride] = v;
      loc += (c == 0 ? G.w[id] : 1.0) * vnrm2(v);
    }
  }
  const double2 s = lblock_sum2(make_double2(loc, 0.0), red);
  double2 tot;
  if (llast_block2(s, partials, counter, G.tiles_x * G.tiles_y, tile, &tot, red)) {
    beta[0] = sqrt(tot.x);
    invb[0] = safe_inv(beta[0]);
  }
}

// One Lanczos step j of the complex form (K = -i tau A, w'_j = K v_j - b_j v_{j-1}).
//   MODE 0 (first pass): v_j = (w'_{j-1} - a_{j-1} v_{j-1}) / b_j  (v_0 = f0 / b_0);
//     the stencil runs on the unscaled tile with 1 / b_j folded into its
//     coefficients; writes v_j, w'_j; a_j = Re <v_j, w'_j>_W (complex) and
//     b_{j+1} = sqrt(||w'_j||_W^2 - a_j^2), one deterministic reduction.
//   MODE 1 (second pass): as MODE 0 with the stored scalars, no reduction,
//     and acc += c_j v_j.
template <int MODE, typename T>
__global__ void __launch_bounds__(THREADS) lz_step(LGeom G, int j, const T* __restrict__ wprev,
                                                   const T* __restrict__ vprev, T* __restrict__ vout,
                                                   T* __restrict__ wout, double* alpha,
                                                   double* beta, double* invb, double2* partials, unsigned* counter,
                                                   T* acc, const double2* cvec, const unsigned* stop) {
  constexpr bool CPLX = sizeof(T) == sizeof(double2);
  __shared__ T E[HY][HX], U[HY][HX], V[HY][HX];
  __shared__ double2 red[THREADS / 32];
  if (MODE == 0 && stop && *stop) return;  // the recurrence already met its bound
  const double bj = beta[j];
  const double sc = invb[j];
  const double am = (CPLX && j > 0) ? alpha[j - 1] : 0.0;
  const double sg = CPLX ? sc : -sc;  // real form: -(tau A)
  StencilCoef cf;
  cf.cdx = sg * G.tdx;
  cf.cdy = sg * G.tdy;
  cf.cgdx = sg * G.tgdx;
  cf.cgdy = sg * G.tgdy;
  cf.cf4 = sg * G.tf4;
  const double bsign = CPLX ? -bj : bj;
  const int i0 = blockIdx.x * TX - 1, j0 = blockIdx.y * TY - 1;
  for (int k = threadIdx.x; k < HX * HY; k += THREADS) {
    const int li = k % HX, lj = k / HX;
    const size_t id = lidx(G, i0 + li, j0 + lj);
    T t[3];
#pragma unroll
    for (int c = 0; c < 3; ++c) {
      t[c] = wprev[id + c * G.fstride];
      if (CPLX && vprev) t[c] = vfma(-am, vprev[id + c * G.fstride], t[c]);
    }
    E[lj][li] = t[0];
    U[lj][li] = t[1];
    V[lj][li] = t[2];
  }
  __syncthreads();
  T cj = vzero<T>();
  if (MODE == 1) cj = cvec_at<T>(cvec, j);
  double dot = 0.0, nrm = 0.0;
  for (int k = threadIdx.x; k < TX * TY; k += THREADS) {
    const int li = k % TX + 1, lj = k / TX + 1;
    const int i = blockIdx.x * TX + li - 1, jj = blockIdx.y * TY + lj - 1;
    if (i >= G.nx || jj >= G.ny) continue;
    const size_t id = (size_t)jj * G.nx + i;
    T ka[3];
    apply_sA<T>(E, U, V, li, lj, G.H[id], cf, ka);
    const T tc[3] = {E[lj][li], U[lj][li], V[lj][li]};
    const double wt = G.w[id];
#pragma unroll
    for (int c = 0; c < 3; ++c) {
      const size_t o = id + c * G.fstride;
      const T vc = vscal(sc, tc[c]);
      const T vp = vprev ? vprev[o] : vzero<T>();
      const T w = vfma(bsign, vp, op_out(ka[c]));
      wout[o] = w;
      vout[o] = vc;
      if (MODE == 1) acc[o] = vcfma(cj, vc, acc[o]);
      if (MODE == 0) {
        const double wc = c == 0 ? wt : 1.0;
        if (CPLX) dot += wc * vredot(vc, w);  // Re conj(v) w
        nrm += wc * vnrm2(w);
      }
    }
  }
  if (MODE != 0) return;
  const double2 s = lblock_sum2(make_double2(dot, nrm), red);
  double2 tot;
  if (llast_block2(s, partials, counter, G.tiles_x * G.tiles_y, blockIdx.y * G.tiles_x + blockIdx.x, &tot, red)) {
    alpha[j] = tot.x;
    beta[j + 1] = sqrt(fmax(tot.y - tot.x * tot.x, 0.0));
    invb[j + 1] = safe_inv(beta[j + 1]);
  }
}

// Real form (real input) on the unnormalised vectors W_j = b_{j+1} u_{j+1}
// alone (u_j = W_{j-1} / b_j is never written):
//   W_j = -(tau / b_j) A W_{j-1} + (b_j / b_{j-1}) W_{j-2},  W_{-1} = f0,
//   b_{j+1} = ||W_j||_W,  a_j = 0.
//   MODE 0 (first pass): writes W_j and b_{j+1} (one deterministic reduction).
//   MODE 1 (second pass): stored scalars, acc += (c'_j / b_j) W_{j-1}.
template <int MODE>
__global__ void __launch_bounds__(THREADS) lz_wstep(LGeom G, int j, const double* __restrict__ wm1,
                                                    const double* __restrict__ wm2, double* __restrict__ wout,
                                                    double* alpha, double* beta, double* invb, double2* partials,
                                                    unsigned* counter, double* acc, const double* coef,
                                                    const unsigned* stop) {
  __shared__ double E[HY][HX], U[HY][HX], V[HY][HX];
  __shared__ double2 red[THREADS / 32];
  __shared__ StencilCoef cfs;
  __shared__ double r2s;
  if (MODE == 0 && stop && *stop) return;  // the recurrence already met its bound
  if (threadIdx.x == 0) {  // step scalars, once per block
    const double sc = invb[j];
    cfs.cdx = -sc * G.tdx;
    cfs.cdy = -sc * G.tdy;
    cfs.cgdx = -sc * G.tgdx;
    cfs.cgdy = -sc * G.tgdy;
    cfs.cf4 = -sc * G.tf4;
    r2s = wm2 ? beta[j] * invb[j - 1] : 0.0;
  }
  const int i0 = blockIdx.x * TX - 1, j0 = blockIdx.y * TY - 1;
  for (int k = threadIdx.x; k < HX * HY; k += THREADS) {
    const int li = k % HX, lj = k / HX;
    const size_t id = lidx(G, i0 + li, j0 + lj);
    E[lj][li] = wm1[id];
    U[lj][li] = wm1[id + G.fstride];
    V[lj][li] = wm1[id + 2 * G.fstride];
  }
  __syncthreads();
  const StencilCoef cf = cfs;
  const double r2 = r2s;
  const double cu = MODE == 1 ? coef[j] : 0.0;
  double nrm = 0.0;
  for (int k = threadIdx.x; k < TX * TY; k += THREADS) {
    const int li = k % TX + 1, lj = k / TX + 1;
    const int i = blockIdx.x * TX + li - 1, jj = blockIdx.y * TY + lj - 1;
    if (i >= G.nx || jj >= G.ny) continue;
    const size_t id = (size_t)jj * G.nx + i;
    double ka[3];
    apply_sA<double>(E, U, V, li, lj, G.H[id], cf, ka);
    const double tc[3] = {E[lj][li], U[lj][li], V[lj][li]};
    double w[3];
#pragma unroll
    for (int c = 0; c < 3; ++c) {
      const size_t o = id + c * G.fstride;
      w[c] = wm2 ? fma(r2, wm2[o], ka[c]) : ka[c];
      wout[o] = w[c];
      if (MODE == 1) acc[o] = fma(cu, tc[c], acc[o]);
    }
    if (MODE == 0) nrm = fma(G.w[id] * w[0], w[0], fma(w[1], w[1], fma(w[2], w[2], nrm)));
  }
  if (MODE != 0) return;
  const double2 s = lblock_sum2(make_double2(nrm, 0.0), red);
  double2 tot;
  if (llast_block2(s, partials, counter, G.tiles_x * G.tiles_y, blockIdx.y * G.tiles_x + blockIdx.x, &tot, red)) {
    alpha[j] = 0.0;
    beta[j + 1] = sqrt(tot.x);
    invb[j + 1] = safe_inv(beta[j + 1]);
  }
}

// ---------------------------------------------------------------------------
// Double-float real form (mixed form, real input): every vector value is a
// pair of floats (hi, lo), value = hi + lo (about 48 significant bits), and
// the step runs on the FP32 pipes with error-free transformations: Knuth's
// TwoSum, Dekker's FastTwoSum and the FMA TwoProduct.  Additions use the
// short form (TwoSum of the high parts, low parts added in FP32), whose error
// is a few units of 2^-48 of the operands: the absolute accuracy the
// Lanczos relation needs.  Scalars and inner products stay FP64.
__device__ __forceinline__ float2 df_fast(float s, float e) {
  const float h = s + e;
  return make_float2(h, e - (h - s));
}
__device__ __forceinline__ float2 df_add(float2 x, float2 y) {
  const float s = x.x + y.x, bb = s - x.x;
  const float e = ((x.x - (s - bb)) + (y.x - bb)) + (x.y + y.y);
  return df_fast(s, e);
}
__device__ __forceinline__ float2 df_neg(float2 x) { return make_float2(-x.x, -x.y); }
__device__ __forceinline__ float2 df_sub(float2 x, float2 y) { return df_add(x, df_neg(y)); }
__device__ __forceinline__ float2 df_mul(float2 x, float2 c) {
  const float p = x.x * c.x;
  const float e = fmaf(x.x, c.y, fmaf(x.y, c.x, fmaf(x.x, c.x, -p)));
  return df_fast(p, e);
}
__device__ __forceinline__ float2 df_from(double v) {
  const float h = (float)v;
  return make_float2(h, (float)(v - (double)h));
}
__device__ __forceinline__ double df_to(float2 v) { return (double)v.x + (double)v.y; }
__device__ __forceinline__ double2 to_out(float2 v) { return make_double2(df_to(v), 0.0); }

// Block sum of double-float values in double-float (FP32 pipes; result valid
// in thread 0).  On this GPU an FP64 warp instruction holds its pipe for many
// cycles even with one active lane, so the reductions of the double-float step
// stay off the FP64 pipe up to one final conversion.
__device__ __forceinline__ float2 df_block_reduce(float2 v, float2* red) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1)
    v = df_add(v, make_float2(__shfl_down_sync(0xffffffffu, v.x, o), __shfl_down_sync(0xffffffffu, v.y, o)));
  const int w = threadIdx.x >> 5, l = threadIdx.x & 31;
  __syncthreads();
  if (l == 0) red[w] = v;
  __syncthreads();
  float2 t = red[0];
  if (threadIdx.x == 0)
    for (int i = 1; i < THREADS / 32; ++i) t = df_add(t, red[i]);
  return t;
}

// Deterministic cross-block double-float sum (fixed order) finished by the
// last block; returns true in that block's thread 0 with *total.
__device__ __forceinline__ bool llast_block_df(float2 mine, float2* partials, unsigned* counter, int ntiles, int tile,
                                               float2* total, float2* red) {
  __shared__ bool is_last;
  if (threadIdx.x == 0) {
    partials[tile] = mine;
    __threadfence();
    is_last = atomicAdd(counter, 1u) == (unsigned)ntiles - 1;
  }
  __syncthreads();
  if (!is_last) return false;
  __threadfence();
  float2 s = strided_partial_sum(partials, ntiles, threadIdx.x, THREADS, make_float2(0.f, 0.f),
                                 [](float2 a, float2 b) { return df_add(a, b); });
  s = df_block_reduce(s, red);
  if (threadIdx.x == 0) {
    *total = s;
    *counter = 0u;
  }
  return threadIdx.x == 0;
}

// Double-float coefficients of step j (computed once, by the reduction that
// produces b_j): the stencil coefficients times -1 / b_j, r2 = b_j / b_{j-1}
// and 1 / b_j itself.
struct DfCoef {
  float2 cdx, cdy, cgdx, cgdy, cf4, r2, ib;
};
__device__ __forceinline__ void df_coef_store(const LGeom& G, double ib, double r2, DfCoef* dst) {
  DfCoef c;
  c.ib = df_from(ib);
  c.cdx = df_from(-ib * G.tdx);
  c.cdy = df_from(-ib * G.tdy);
  c.cgdx = df_from(-ib * G.tgdx);
  c.cgdy = df_from(-ib * G.tgdy);
  c.cf4 = df_from(-ib * G.tf4);
  c.r2 = df_from(r2);
  *dst = c;
}

// sqrt(s) and 1 / b for non-negative double-float values on the FP32 pipes:
// a correctly rounded FP32 root (reciprocal) and one correction from the
// exact FMA residual (Markstein), within about 2^-48 of the result.  Zero
// gives zero (1 / 0 too: b = 0 ends the recurrence); a NaN or an infinity in
// s comes out non-finite.  On this GPU a dependent FP64 operation waits about
// a hundred cycles, so the scalars at the end of each step stay off the FP64
// pipe.
__device__ __forceinline__ float2 df_sqrt(float2 s) {
  if (s.x == 0.f) return make_float2(0.f, 0.f);
  const float h = __fsqrt_rn(s.x);
  const float e = __fadd_rn(__fmaf_rn(-h, h, s.x), s.y);  // s - h^2
  return df_fast(h, __fdiv_rn(e, 2.f * h));
}
__device__ __forceinline__ float2 df_recip(float2 b) {
  if (b.x == 0.f) return make_float2(0.f, 0.f);
  const float r = __frcp_rn(b.x);
  const float e = __fmaf_rn(-b.y, r, __fmaf_rn(-b.x, r, 1.f));  // 1 - b r
  return df_fast(r, __fmul_rn(e, r));
}

__global__ void lz_df_tables(const double* H, const double* w, size_t nk, float2* Hdf, float2* wdf) {
  const size_t i = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= nk) return;
  Hdf[i] = df_from(H[i]);
  wdf[i] = df_from(w[i]);
}

// f0 = Re in (eta / w for the adjoint) as double-float; beta[0] = ||f0||_W (FP64).
__global__ void __launch_bounds__(THREADS) lz_init_df(LGeom G, const double2* in, int adjoint, float2* f0,
                                                      double* beta, double* invb, DfCoef* dfc, double2* partials,
                                                      unsigned* counter) {
  __shared__ double2 red[THREADS / 32];
  const int tile = blockIdx.y * G.tiles_x + blockIdx.x;
  double loc = 0.0;
  for (int k = threadIdx.x; k < TX * TY; k += THREADS) {
    const int i = blockIdx.x * TX + k % TX, j = blockIdx.y * TY + k / TX;
    if (i >= G.nx || j >= G.ny) continue;
    const size_t id = (size_t)j * G.nx + i;
    for (int c = 0; c < 3; ++c) {
      double v = in[id + c * G.fstride].x;
      if (adjoint && c == 0) v /= G.w[id];
      const float2 d = df_from(v);
      f0[id + c * G.fstride] = d;
      const double vv = df_to(d);
      loc += (c == 0 ? G.w[id] : 1.0) * vv * vv;
    }
  }
  const double2 s = lblock_sum2(make_double2(loc, 0.0), red);
  double2 tot;
  if (llast_block2(s, partials, counter, G.tiles_x * G.tiles_y, tile, &tot, red)) {
    beta[0] = sqrt(tot.x);
    invb[0] = safe_inv(beta[0]);
    df_coef_store(G, invb[0], 0.0, dfc);
  }
}

// Programmatic dependent launch of consecutive Lanczos steps: a step's CTAs
// may start while the previous step drains.  griddepcontrol.wait blocks until
// the previous grid has completed and its writes are visible; a step lets the
// next one start only after its own wait, so every grid that can run early
// finds the step before its predecessor complete (W_{j-2} may be read early).
// Resident CTAs per SM the double-float step is compiled for (48 registers at
// 5: the step is bound by load latency, so occupancy pays).
#ifndef REXI_LZ_DFSTEP_BLOCKS
#define REXI_LZ_DFSTEP_BLOCKS 5
#endif
constexpr int kDfStepBlocks = REXI_LZ_DFSTEP_BLOCKS;

// 8-byte global-to-shared copy (cp.async, cached at all levels) and the wait
// for all of the thread's copies.
__device__ __forceinline__ void cp_async8(void* smem, const void* gmem) {
  const unsigned sa = (unsigned)__cvta_generic_to_shared(smem);
  asm volatile("cp.async.ca.shared.global [%0], [%1], 8;" ::"r"(sa), "l"(gmem) : "memory");
}
__device__ __forceinline__ void cp_async_wait_all() { asm volatile("cp.async.wait_all;" ::: "memory"); }

__device__ __forceinline__ void pdl_wait() { asm volatile("griddepcontrol.wait;" ::: "memory"); }
__device__ __forceinline__ void pdl_release() { asm volatile("griddepcontrol.launch_dependents;" ::: "memory"); }

// The real-form step (lz_wstep) in double-float.  The point-wise operands of
// the thread's points (W_{j-2}, H, g/H: complete before this grid may start)
// are loaded before waiting for the previous step, so that their latency
// overlaps its tail and the halo loads.
template <int MODE>
__global__ void __launch_bounds__(THREADS, kDfStepBlocks) lz_dfstep(LGeom G, const float2* __restrict__ Hdf,
                                                     const float2* __restrict__ wdf, int j,
                                                     const float2* __restrict__ wm1, const float2* __restrict__ wm2,
                                                     float2* __restrict__ wout, double* alpha, double* beta,
                                                     double* invb, DfCoef* dfc, double2* partials,
                                                     unsigned* counter, float2* acc, const float2* coef_df,
                                                     const unsigned* stop) {
  constexpr int PPT = TX * TY / THREADS;  // interior points per thread
  __shared__ float2 E[HY][HX], U[HY][HX], V[HY][HX];
  __shared__ float2 red[THREADS / 32];
  const float2 z2 = make_float2(0.f, 0.f);
  size_t pid[PPT];
  bool live[PPT];
  float2 pw2[PPT][3], pH[PPT], pw[PPT];
#pragma unroll
  for (int q = 0; q < PPT; ++q) {
    const int k = threadIdx.x + q * THREADS;
    const int i = blockIdx.x * TX + k % TX, jj = blockIdx.y * TY + k / TX;
    live[q] = i < G.nx && jj < G.ny;
    pid[q] = live[q] ? (size_t)jj * G.nx + i : 0;
#pragma unroll
    for (int c = 0; c < 3; ++c) pw2[q][c] = (live[q] && wm2) ? wm2[pid[q] + c * G.fstride] : z2;
    pH[q] = live[q] ? Hdf[pid[q]] : z2;
    pw[q] = (live[q] && MODE == 0) ? wdf[pid[q]] : z2;
  }
  pdl_wait();
  pdl_release();
  const int i0 = blockIdx.x * TX - 1, j0 = blockIdx.y * TY - 1;
  // halo tile by asynchronous 8-byte copies straight into shared memory: every
  // copy of the thread is in flight before the first wait (2048^2: 89 us per
  // step against 95 us with loads through registers)
#pragma unroll
  for (int r = 0; r < (HX * HY + THREADS - 1) / THREADS; ++r) {
    const int k = threadIdx.x + r * THREADS;
    if (k < HX * HY) {
      const int li = k % HX, lj = k / HX;
      const size_t id = lidx(G, i0 + li, j0 + lj);
      cp_async8(&E[lj][li], wm1 + id);
      cp_async8(&U[lj][li], wm1 + id + G.fstride);
      cp_async8(&V[lj][li], wm1 + id + 2 * G.fstride);
    }
  }
  // read while the halo copies are in flight; a block leaves only after its
  // copies have landed
  const unsigned stopped = (MODE == 0 && stop) ? *stop : 0u;
  cp_async_wait_all();
  __syncthreads();
  if (stopped) return;  // the recurrence already met its bound
  const DfCoef cf = dfc[j];
  const float2 cu = MODE == 1 ? coef_df[j] : z2;
  float2 nrm = z2;
#pragma unroll
  for (int q = 0; q < PPT; ++q) {
    if (!live[q]) continue;
    const int k = threadIdx.x + q * THREADS;
    const int li = k % TX + 1, lj = k / TX + 1;
    const size_t id = pid[q];
    float2 ka[3];
    // eta: -H (cdx du + cdy dv)
    const float2 du = df_sub(U[lj][li], U[lj][li - 1]), dv = df_sub(V[lj][li], V[lj - 1][li]);
    ka[0] = df_neg(df_mul(df_add(df_mul(du, cf.cdx), df_mul(dv, cf.cdy)), pH[q]));
    // u: cf4 v4 - cgdx de
    const float2 v4 = df_add(df_add(V[lj][li], V[lj][li + 1]), df_add(V[lj - 1][li], V[lj - 1][li + 1]));
    const float2 de = df_sub(E[lj][li + 1], E[lj][li]);
    ka[1] = df_sub(df_mul(v4, cf.cf4), df_mul(de, cf.cgdx));
    // v: -cf4 u4 - cgdy dn
    const float2 u4 = df_add(df_add(U[lj][li], U[lj][li - 1]), df_add(U[lj + 1][li], U[lj + 1][li - 1]));
    const float2 dn = df_sub(E[lj + 1][li], E[lj][li]);
    ka[2] = df_neg(df_add(df_mul(u4, cf.cf4), df_mul(dn, cf.cgdy)));
    const float2 tc[3] = {E[lj][li], U[lj][li], V[lj][li]};
    float2 w[3];
#pragma unroll
    for (int c = 0; c < 3; ++c) {
      const size_t o = id + c * G.fstride;
      w[c] = wm2 ? df_add(df_mul(pw2[q][c], cf.r2), ka[c]) : ka[c];
      wout[o] = w[c];
      if (MODE == 1) acc[o] = df_add(acc[o], df_mul(tc[c], cu));
    }
    if (MODE == 0) {
      nrm = df_add(nrm, df_mul(df_mul(w[0], w[0]), pw[q]));
      nrm = df_add(nrm, df_mul(w[1], w[1]));
      nrm = df_add(nrm, df_mul(w[2], w[2]));
    }
  }
  if (MODE != 0) return;
  const float2 bs = df_block_reduce(nrm, red);
  float2 tot;
  if (llast_block_df(bs, reinterpret_cast<float2*>(partials), counter, G.tiles_x * G.tiles_y,
                     blockIdx.y * G.tiles_x + blockIdx.x, &tot, red)) {
    // b_{j+1} = ||W_j||_W and the next step's coefficients in double-float
    // (the FP64 copies of b and 1 / b for the tridiagonal solves after them)
    const float2 b = df_sqrt(tot), ib = df_recip(b), nib = df_neg(ib);
    DfCoef c;
    c.cdx = df_mul(nib, df_from_double(G.tdx));
    c.cdy = df_mul(nib, df_from_double(G.tdy));
    c.cgdx = df_mul(nib, df_from_double(G.tgdx));
    c.cgdy = df_mul(nib, df_from_double(G.tgdy));
    c.cf4 = df_mul(nib, df_from_double(G.tf4));
    c.r2 = df_mul(b, cf.ib);
    c.ib = ib;
    dfc[j + 1] = c;
    alpha[j] = 0.0;
    beta[j + 1] = df_to_double(b);
    invb[j + 1] = df_to_double(ib);
  }
}

// Launch of a Lanczos step that may overlap the previous step's tail (see
// pdl_wait); a launch error is left for the caller's cudaGetLastError.
template <typename... KArgs, typename... Args>
void launch_step_pdl(void (*kern)(KArgs...), dim3 grid, cudaStream_t s, Args... args) {
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = grid;
  cfg.blockDim = dim3(THREADS);
  cfg.dynamicSmemBytes = 0;
  cfg.stream = s;
  cudaLaunchAttribute at[1];
  at[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
  at[0].val.programmaticStreamSerializationAllowed = 1;
  cfg.attrs = at;
  cfg.numAttrs = 1;
  cudaLaunchKernelEx(&cfg, kern, static_cast<KArgs>(args)...);
}

// Double-float: acc = sum_{b < nb} coef_b S_b (S_0 = f0, S_b = W_{b-1}).
__global__ void lz_dfbasis_sum(const float2* __restrict__ f0, const float2* __restrict__ basis, size_t vstride,
                               int nb, const float2* coef_df, float2* acc, size_t n) {
  const size_t i = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  float2 a = make_float2(0.f, 0.f);
  if (nb > 0) a = df_add(a, df_mul(f0[i], coef_df[0]));
  int b = 1;
  for (; b + 4 <= nb; b += 4) {
    const float2 v0 = basis[(size_t)(b - 1) * vstride + i], v1 = basis[(size_t)b * vstride + i];
    const float2 v2 = basis[(size_t)(b + 1) * vstride + i], v3 = basis[(size_t)(b + 2) * vstride + i];
    a = df_add(a, df_mul(v0, coef_df[b]));
    a = df_add(a, df_mul(v1, coef_df[b + 1]));
    a = df_add(a, df_mul(v2, coef_df[b + 2]));
    a = df_add(a, df_mul(v3, coef_df[b + 3]));
  }
  for (; b < nb; ++b) a = df_add(a, df_mul(basis[(size_t)(b - 1) * vstride + i], coef_df[b]));
  acc[i] = a;
}

// Real form: coef[b] = c'_b / b_b for b < kk.
__global__ void lz_wcoef(const double2* cvec, const double* invb, int kk, double* coef, float2* coef_df) {
  const int b = blockIdx.x * blockDim.x + threadIdx.x;
  if (b >= kk) return;
  coef[b] = real_coeff(cvec[b], b) * invb[b];
  coef_df[b] = df_from(coef[b]);
}

// Real form: acc = sum_{b < nb} coef_b S_b, S_0 = f0, S_b = W_{b-1} (kept
// vector b - 1); the same coefficients and order as the second-pass steps.
__global__ void lz_wbasis_sum(const double* __restrict__ f0, const double* __restrict__ basis, size_t vstride, int nb,
                              const double* coef, double* acc, size_t n) {
  const size_t i = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  double a = 0.0;
  if (nb > 0) a = fma(coef[0], f0[i], a);
  int b = 1;
  for (; b + 4 <= nb; b += 4) {
    const double v0 = basis[(size_t)(b - 1) * vstride + i], v1 = basis[(size_t)b * vstride + i];
    const double v2 = basis[(size_t)(b + 1) * vstride + i], v3 = basis[(size_t)(b + 2) * vstride + i];
    a = fma(coef[b], v0, a);
    a = fma(coef[b + 1], v1, a);
    a = fma(coef[b + 2], v2, a);
    a = fma(coef[b + 3], v3, a);
  }
  for (; b < nb; ++b) a = fma(coef[b], basis[(size_t)(b - 1) * vstride + i], a);
  acc[i] = a;
}

// acc = sum_{b < nb} c_b basis_b (acc = 0 for nb = 0); fixed summation order,
// four vectors per pass for loads in flight.
template <typename T>
__global__ void lz_basis_sum(const T* __restrict__ basis, size_t vstride, int nb, const double2* cvec, T* acc,
                             size_t n) {
  const size_t i = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  T a = vzero<T>();
  int b = 0;
  for (; b + 4 <= nb; b += 4) {
    const T v0 = basis[(size_t)b * vstride + i], v1 = basis[(size_t)(b + 1) * vstride + i];
    const T v2 = basis[(size_t)(b + 2) * vstride + i], v3 = basis[(size_t)(b + 3) * vstride + i];
    a = vcfma(cvec_at<T>(cvec, b), v0, a);
    a = vcfma(cvec_at<T>(cvec, b + 1), v1, a);
    a = vcfma(cvec_at<T>(cvec, b + 2), v2, a);
    a = vcfma(cvec_at<T>(cvec, b + 3), v3, a);
  }
  for (; b < nb; ++b) a = vcfma(cvec_at<T>(cvec, b), basis[(size_t)b * vstride + i], a);
  acc[i] = a;
}

// out = acc (eta times w for the adjoint), real part only for real input.
template <typename T>
__global__ void lz_finish(const T* acc, double2* out, const double* w, size_t nk, int real_out, int adjoint) {
  const size_t i = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= 3 * nk) return;
  double2 v = to_out(acc[i]);
  if (adjoint && i < nk) {
    v.x *= w[i];
    v.y *= w[i];
  }
  if (real_out) v.y = 0.0;
  out[i] = v;
}

// 1 / x for normal FP64 x: the hardware's approximate FP64 reciprocal r0 as
// the seed, then r0 (1 + e + e^2) with e = 1 - x r0 (1 / x = r0 / (1 - e)),
// which leaves a relative error of order e^3, below FP64 rounding: four
// dependent operations, where a dependent FP64 operation on this GPU waits
// about a hundred cycles.
__device__ __forceinline__ double lrcp(double x) {
  double r0;
  asm("rcp.approx.ftz.f64 %0, %1;" : "=d"(r0) : "d"(x));
  const double e = fma(-x, r0, 1.0);
  return fma(r0, fma(e, e, e), r0);
}
// 1 / z for the pivots of the shifted tridiagonal systems (T_k + s_p): every
// shift lies h |mu| from the line that holds the spectrum of T_k, and each
// pivot d_j = a_j + s_p - b_j^2 / d_{j-1} keeps at least that distance (the
// term -b_j^2 / d_{j-1} moves it away from the line, never towards it), so
// |z|^2 is a normal number for lrcp.  The hardware seed and three FMAs
// instead of an FP64 division, the longest step of the per-pole recurrences.
__device__ __forceinline__ double2 crcp(double2 z) {
  const double r = lrcp(fma(z.x, z.x, z.y * z.y));
  return make_double2(z.x * r, -z.y * r);
}
__device__ __forceinline__ double2 cmuld(double2 a, double2 b) {
  return make_double2(fma(a.x, b.x, -a.y * b.y), fma(a.x, b.y, a.y * b.x));
}


// Per pole p: forward elimination of (T + s_p) over the new steps [j0, j1);
// wy_p = weight_p * e_{j1-1}^T (T_{j1} + s_p)^{-1} e_0 = weight_p g / d.
// `clear` (nullable): the two maxima of the check that follows, zeroed here.
__global__ void lz_poles_advance(int np, const double2* s, const double2* wgt, const double* alpha,
                                 const double* beta, int j0, int j1, double2* dg, double2* wy, const unsigned* stop,
                                 unsigned long long* clear) {
  const int p = blockIdx.x * blockDim.x + threadIdx.x;
  if (clear && p == 0) clear[0] = clear[1] = 0ull;
  if (p >= np || *stop) return;
  double2 d = dg[2 * p], g = dg[2 * p + 1];
  const double2 sp = s[p];
  for (int j = j0; j < j1; ++j) {
    if (j == 0) {
      d = make_double2(alpha[0] + sp.x, sp.y);
      g = make_double2(1.0, 0.0);
    } else {
      // m = b / d; d <- a + s - m b, g <- -m g
      const double b = beta[j];
      const double2 id = crcp(d);
      const double2 mg = cmuld(id, g);
      d = make_double2(fma(-b * b, id.x, alpha[j] + sp.x), fma(-b * b, id.y, sp.y));
      g = make_double2(-b * mg.x, -b * mg.y);
    }
  }
  dg[2 * p] = d;
  dg[2 * p + 1] = g;
  const double2 y = cmuld(g, crcp(d)), wp = wgt[p];
  wy[p] = make_double2(wp.x * y.x - wp.y * y.y, wp.x * y.y + wp.y * y.x);
}


constexpr int BT = 64;  // threads per block of the error-bound kernels

// Partial sums of phi(l_m) = sum_p wy_p / (l_m + s_p) over the poles of group
// blockIdx.y (G poles each) at samples l_m = -L + m dl, m = slot * stride:
// part[group * nslot + slot].  With `gate`, runs only if
// beta[jk] * (max of the gate pass) <= rtol.
__global__ void __launch_bounds__(BT) lz_bound_part(int np, int G, const double2* s, const double2* wy, double L,
                                                    double dl, int nslot, int stride, const double* beta, int jk,
                                                    double rtol, const unsigned long long* gate, double2* part,
                                                    const unsigned* stop) {
  if (*stop || (gate && beta[jk] * __longlong_as_double((long long)*gate) > rtol)) return;
  __shared__ double2 ss[BT], sw[BT];
  const int slot = blockIdx.x * BT + threadIdx.x;
  const double lam = -L + (double)slot * stride * dl;
  const int pb = blockIdx.y * G, pe = min(np, pb + G);
  double re = 0.0, im = 0.0;
  for (int p0 = pb; p0 < pe; p0 += BT) {
    __syncthreads();
    if (p0 + threadIdx.x < pe) {
      ss[threadIdx.x] = s[p0 + threadIdx.x];
      sw[threadIdx.x] = wy[p0 + threadIdx.x];
    }
    __syncthreads();
    const int cnt = min(BT, pe - p0);
    for (int q = 0; q < cnt; ++q) {
      const double a = lam + ss[q].x, b = ss[q].y;
      const double r = lrcp(fma(a, a, b * b));
      re = fma(r, fma(sw[q].x, a, sw[q].y * b), re);   // Re w / (a + ib)
      im = fma(r, fma(sw[q].y, a, -sw[q].x * b), im);  // Im w / (a + ib)
    }
  }
  if (slot < nslot) part[(size_t)blockIdx.y * nslot + slot] = make_double2(re, im);
}

// max over slots of |phi| (sum over groups in fixed order), as the bits of a
// non-negative double (atomicMax on those bits is order-independent).  Real
// form (sym != 0): the bound function of the conjugate-closed pole set,
// (phi(l) + sym conj(phi(-l))) / 2 with sym = (-1)^(k-1); the sample grid is
// symmetric (slot nslot - 1 - m sits at -l_m).
__global__ void __launch_bounds__(BT) lz_bound_max(int groups, int nslot, const double2* part, int sym,
                                                   const double* beta, int jk, double rtol,
                                                   const unsigned long long* gate, unsigned long long* out,
                                                   const unsigned* stop) {
  if (*stop || (gate && beta[jk] * __longlong_as_double((long long)*gate) > rtol)) return;
  __shared__ double red[BT / 32];
  const int slot = blockIdx.x * BT + threadIdx.x;
  double v = 0.0;
  if (slot < nslot) {
    double re = 0.0, im = 0.0;
    for (int g = 0; g < groups; ++g) {
      const double2 t = part[(size_t)g * nslot + slot];
      re += t.x;
      im += t.y;
    }
    if (sym) {
      double re2 = 0.0, im2 = 0.0;
      for (int g = 0; g < groups; ++g) {
        const double2 t = part[(size_t)g * nslot + (nslot - 1 - slot)];
        re2 += t.x;
        im2 += t.y;
      }
      re = 0.5 * fma((double)sym, re2, re);
      im = 0.5 * fma(-(double)sym, im2, im);
    }
    v = sqrt(fma(re, re, im * im));
  }
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v = fmax(v, __shfl_down_sync(0xffffffffu, v, o));
  if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = v;
  __syncthreads();
  if (threadIdx.x == 0) {
    double b = 0.0;
    for (int i = 0; i < BT / 32; ++i) b = fmax(b, red[i]);
    atomicMax(out, (unsigned long long)__double_as_longlong(b));
  }
}

// The host's convergence test of a checked chunk, repeated on the device so
// that the chunk enqueued behind it (the host tests one chunk while the next
// runs) stops at once: *stop = 1 once beta[jk] times the sampled maximum of
// |phi| meets rtol (the fine maximum when the coarse one passed), or when
// either is not finite (the host then reports the non-finite scalars).
// Every later kernel of the first pass returns on *stop.  `report` receives
// (b, coarse, fine) for the host's copy.
__global__ void lz_gate(const double* beta, int jk, const unsigned long long* maxslots, double rtol,
                        unsigned* stop, double* report) {
  const double b = beta[jk];
  const double coarse = __longlong_as_double((long long)maxslots[0]);
  const double fine = __longlong_as_double((long long)maxslots[1]);
  // what the host tests, in one block for one copy: b, coarse, fine
  report[0] = b;
  report[1] = coarse;
  report[2] = fine;
  if (!isfinite(b) || !isfinite(coarse) || !isfinite(fine)) {
    *stop = 1u;
    return;
  }
  const double bound = b * coarse > rtol ? b * coarse : b * fine;
  if (bound <= rtol) *stop = 1u;
}

// Coefficients of V c for the poles [p0, p0 + P): per pole the UL sweep of
// (T_k + s_p) (psi_{k-1} = a_{k-1} + s_p, psi_i = a_i + s_p - b_{i+1}^2 / psi_{i+1})
// gives y = (T_k + s_p)^{-1} e_0 forward (y_0 = 1 / psi_0,
// y_{i+1} = -b_{i+1} y_i / psi_{i+1}); scratch[i P + q] = -i ||f|| weight_p y_i.
__global__ void lz_coeff_solve(int p0, int P, const double2* s, const double2* wgt, const double* alpha,
                               const double* beta, int kk, double2* scratch) {
  const int q = blockIdx.x * blockDim.x + threadIdx.x;
  if (q >= P) return;
  const double2 sp = s[p0 + q], wp = wgt[p0 + q];
  // the sweep keeps 1 / psi_i, so that the forward recurrence multiplies
  double2 ip = crcp(make_double2(alpha[kk - 1] + sp.x, sp.y));
  scratch[(size_t)(kk - 1) * P + q] = ip;
#pragma unroll 4
  for (int i = kk - 2; i >= 0; --i) {
    const double b2 = beta[i + 1] * beta[i + 1];
    ip = crcp(make_double2(fma(-b2, ip.x, alpha[i] + sp.x), fma(-b2, ip.y, sp.y)));
    scratch[(size_t)i * P + q] = ip;
  }
  // scale = -i ||f|| weight; y_0 = 1 / psi_0, y_i = -b_i y_{i-1} / psi_i
  const double fn = beta[0];
  const double2 sc = make_double2(fn * wp.y, -fn * wp.x);
  double2 y = ip;
  scratch[q] = cmuld(sc, y);
#pragma unroll 4
  for (int i = 1; i < kk; ++i) {
    const double2 t = cmuld(y, scratch[(size_t)i * P + q]);
    y = make_double2(-beta[i] * t.x, -beta[i] * t.y);
    scratch[(size_t)i * P + q] = cmuld(sc, y);
  }
}

// cvec[i] (+)= sum_q scratch[i P + q], one block per i, fixed order.
__global__ void __launch_bounds__(THREADS) lz_coeff_sum(int P, const double2* scratch, double2* cvec, int first) {
  __shared__ double2 red[THREADS / 32];
  const int i = blockIdx.x;
  double2 a = make_double2(0.0, 0.0);
  for (int q = threadIdx.x; q < P; q += THREADS) a = ladd(a, scratch[(size_t)i * P + q]);
  a = lblock_sum2(a, red);
  if (threadIdx.x == 0) cvec[i] = first ? a : ladd(cvec[i], a);
}

size_t al(size_t v) { return (v + 255) / 256 * 256; }

struct LLayout {
  size_t vb, scratch_bytes, alpha, beta, invb, coef, coef_df, dfc, cvec, partials, counter, maxslots, wy, dg, sc, wc, part, min_total;
};

// Error-bound sampling: spacing at most d / 4 over [-tau rho, tau rho],
// d = h |mu|, sample count 1 mod kCoarse (symmetric coarse subgrid); with
// tau rho <= M h (pole-count rule) at most 8 M / |mu| + 2 + kCoarse samples.
int nsamp_cap(int M) { return (int)std::ceil(8.0 * M / std::fabs(table_mu())) + 2 + kCoarse; }
// poles per group of the partial sums (at most 128 groups).  The grouping
// sets the rounding of phi, whose floor the bound reaches at tight
// tolerances: groups of 16 instead of 64 raised that floor enough for a
// 1e-13 bound to take four times the Lanczos steps.
int bound_group(int np) { return std::max(64, (np + 127) / 128); }

LLayout lz_layout(const KrylovSettings* k, int np_c, int M, size_t esize) {
  LLayout L{};
  const size_t nk = (size_t)k->nx * k->ny;
  const size_t ntiles = (size_t)((k->nx + TX - 1) / TX) * ((k->ny + TY - 1) / TY);
  const size_t nmax = (size_t)k->max_iters + 2;
  L.vb = al(3 * nk * esize);
  // f0 | acc vA vB wA wB (+ extra): the five vectors double as the coefficient
  // scratch once the first pass is over
  const size_t smin = (size_t)kMinScratchPoles * nmax * sizeof(double2);
  L.scratch_bytes = std::max(5 * L.vb, al(smin));
  size_t o = L.vb + L.scratch_bytes;
  L.alpha = o;
  o += al(nmax * sizeof(double));
  L.beta = o;
  o += al(nmax * sizeof(double));
  L.invb = o;
  o += al(nmax * sizeof(double));
  L.coef = o;
  o += al(nmax * sizeof(double));
  L.coef_df = o;
  o += al(nmax * sizeof(float2));
  L.dfc = o;
  o += al(nmax * sizeof(DfCoef));
  L.cvec = o;
  o += al(nmax * sizeof(double2));
  L.partials = o;
  o += al(ntiles * sizeof(double2));
  L.counter = o;
  o += 256;
  L.maxslots = o;
  o += 256;
  L.wy = o;
  o += al((size_t)np_c * sizeof(double2));
  L.dg = o;
  o += al((size_t)np_c * 2 * sizeof(double2));
  L.sc = o;
  o += al((size_t)np_c * sizeof(double2));
  L.wc = o;
  o += al((size_t)np_c * sizeof(double2));
  L.part = o;  // bound_group keeps the group count at or below 128
  o += al((size_t)128 * nsamp_cap(M) * sizeof(double2));
  L.min_total = o;
  return L;
}

int poles_c(int M, int real_input) {
  const int N = M + kL;
  return real_input ? 2 * (N + 1) : 2 * (2 * N + 1);
}

template <typename T>
rexi_status lanczos_impl(KrylovSettings* k, double h, int M, const void* in, void* out, double dt, int real_input,
                         int term_begin, int term_end, void* ws, size_t ws_bytes, cudaStream_t s,
                         rexi_step_info* info, bool adjoint, const KrylovHooks& hooks) {
  using cd = std::complex<double>;
  auto mark = [&](int i) {
    if (hooks.mark) hooks.mark(hooks.ctx, i, s);
  };
  int64_t launches = 0;
  const int N = M + kL;
  if (term_end < 0 || term_end > N + 1) term_end = N + 1;
  if (term_begin < 0 || term_begin > term_end) {
    set_last_error("bad term range");
    return REXI_EINVAL;
  }
  const size_t nk = (size_t)k->nx * k->ny, n3 = 3 * nk;
  if ((const char*)in < (const char*)out + n3 * sizeof(double2) &&
      (const char*)out < (const char*)in + n3 * sizeof(double2)) {
    set_last_error("variable-depth path: input and output must not overlap");
    return REXI_EINVAL;
  }
  if (!(k->rho_bound > 0.0) || !k->pinned) {
    set_last_error("shared-Krylov method: plan has no spectral bound");
    return REXI_EINVAL;
  }
  const int npc_max = poles_c(M, real_input);
  const LLayout L = lz_layout(k, npc_max, M, sizeof(T));
  if (ws_bytes < L.min_total) {
    set_last_error("workspace too small for the shared-Krylov method");
    return REXI_ENOMEM;
  }

  // poles z_j and weights beta_j of the selected REXII terms (partial fractions
  // of each term: z = alpha_{-n} with -Gamma P_n, z = -alpha_n with Gamma Q_n)
  TermSet ts;
  rexii_terms(M, h, &ts);
  const double hmu = h * ts.mu;
  std::vector<double2> sc, wc;
  const cd I(0.0, 1.0);
  auto push = [&](cd z, cd w) {
    const cd sz = I * z;  // shift of K: (tau A - z)^{-1} = -i (K + i z)^{-1}
    sc.push_back(make_double2(sz.real(), sz.imag()));
    wc.push_back(make_double2(w.real(), w.imag()));
  };
  for (int n = real_input ? 0 : -N; n <= N; ++n) {
    const int an = n < 0 ? -n : n;
    if (an < term_begin || an >= term_end) continue;
    const int i = n + N;
    const double gam = (real_input && n > 0) ? 2.0 : 1.0;
    const cd C1(ts.c1re[i] * hmu + ts.c2re[i] * h * n, ts.c1im[i] * hmu + ts.c2im[i] * h * n);
    const cd C2 = I * cd(ts.c2re[i], ts.c2im[i]);
    const cd a_n(hmu, h * n), a_mn(hmu, -h * n);
    const cd P = (C1 - C2 * a_mn) / (2.0 * hmu), Q = (C1 + C2 * a_n) / (2.0 * hmu);
    push(a_mn, -gam * P);
    push(-a_n, gam * Q);
  }
  const int npc = (int)sc.size();

  char* base = static_cast<char*>(ws);
  T* f0 = reinterpret_cast<T*>(base);
  T* acc = reinterpret_cast<T*>(base + L.vb);
  T* vA = reinterpret_cast<T*>(base + 2 * L.vb);
  T* vB = reinterpret_cast<T*>(base + 3 * L.vb);
  T* wA = reinterpret_cast<T*>(base + 4 * L.vb);
  T* wB = reinterpret_cast<T*>(base + 5 * L.vb);
  double2* scratch = reinterpret_cast<double2*>(base + L.vb);
  double* alpha = reinterpret_cast<double*>(base + L.alpha);
  double* beta = reinterpret_cast<double*>(base + L.beta);
  double* invb = reinterpret_cast<double*>(base + L.invb);  // 1 / b_j (0 for b_j = 0)
  double* coef = reinterpret_cast<double*>(base + L.coef);  // real form: c'_j / b_j
  float2* coef_df = reinterpret_cast<float2*>(base + L.coef_df);
  DfCoef* dfc = reinterpret_cast<DfCoef*>(base + L.dfc);  // double-float step coefficients
  double2* cvec = reinterpret_cast<double2*>(base + L.cvec);
  double2* partials = reinterpret_cast<double2*>(base + L.partials);
  unsigned* counter = reinterpret_cast<unsigned*>(base + L.counter);
  unsigned long long* maxslots = reinterpret_cast<unsigned long long*>(base + L.maxslots);
  double2* d_wy = reinterpret_cast<double2*>(base + L.wy);
  double2* d_dg = reinterpret_cast<double2*>(base + L.dg);
  double2* d_sc = reinterpret_cast<double2*>(base + L.sc);
  double2* d_wc = reinterpret_cast<double2*>(base + L.wc);
  double2* d_part = reinterpret_cast<double2*>(base + L.part);
  // Lanczos vectors kept in the caller's extra workspace
  T* basis = reinterpret_cast<T*>(base + L.min_total);
  const size_t vstride = L.vb / sizeof(T);
  constexpr bool DF = std::is_same<T, float2>::value;  // double-float real form
  constexpr bool REAL = DF || std::is_same<T, double>::value;
  // complex form: kept v_j (at least two, or none); w'_{nbasis-1} goes to f0's
  // buffer (f0 is read only by step 0) so that the second pass can resume the
  // recurrence at step nbasis with exactly the first pass's operands.
  // real form: kept W_j; the second pass resumes from W_{nbasis-1}, W_{nbasis-2}.
  int nbasis = (int)std::min<size_t>((ws_bytes - L.min_total) / L.vb, (size_t)k->max_iters + 1);
  if (!REAL && nbasis < 2) nbasis = 0;
  auto vptr = [&](int j) -> T* {
    if (j < 0) return nullptr;
    if (j < nbasis) return basis + (size_t)j * vstride;
    return (j & 1) ? vB : vA;
  };
  auto wptr = [&](int j) -> T* { return (j < 0 || j == nbasis - 1) ? f0 : ((j & 1) ? wB : wA); };
  T* const rot[3] = {vA, vB, wA};
  auto Wptr = [&](int j) -> T* {  // real form
    if (j < 0) return j == -1 ? f0 : nullptr;
    if (j < nbasis) return basis + (size_t)j * vstride;
    return rot[j % 3];
  };

  const double tau = adjoint ? -dt : dt;
  LGeom G_;
  G_.nx = k->nx;
  G_.ny = k->ny;
  G_.tiles_x = (k->nx + TX - 1) / TX;
  G_.tiles_y = (k->ny + TY - 1) / TY;
  G_.fstride = nk;
  const double idx = k->nx / k->Lx, idy = k->ny / k->Ly;
  G_.tdx = tau * idx;
  G_.tdy = tau * idy;
  G_.tgdx = tau * k->g * idx;
  G_.tgdy = tau * k->g * idy;
  G_.tf4 = 0.25 * tau * k->f;
  G_.H = k->depth;
  G_.w = k->w64;
  const dim3 grid(G_.tiles_x, G_.tiles_y, 1);
  const unsigned ebl = (unsigned)((n3 + 255) / 256);

  cudaError_t e = cudaSuccess;
  mark(0);
  if (npc == 0) {  // empty term slice
    e = cudaMemsetAsync(out, 0, n3 * sizeof(double2), s);
    mark(1);
    mark(2);
    mark(3);
    mark(4);
    if (e != cudaSuccess) {
      set_last_error(cudaGetErrorString(e));
      return REXI_ECUDA;
    }
    if (info) {
      memset(info, 0, sizeof(*info));
      info->N = N;
      info->n_terms = real_input ? N + 1 : 2 * N + 1;
      info->n_poles = npc_max;
    }
    return REXI_OK;
  }
  e = cudaMemcpyAsync(d_sc, sc.data(), npc * sizeof(double2), cudaMemcpyHostToDevice, s);
  if (e == cudaSuccess) e = cudaMemcpyAsync(d_wc, wc.data(), npc * sizeof(double2), cudaMemcpyHostToDevice, s);
  // the reduction counter and the stop flag of the first pass (lz_gate)
  if (e == cudaSuccess) e = cudaMemsetAsync(counter, 0, 2 * sizeof(unsigned), s);
  mark(1);
  if (e == cudaSuccess) {
    if constexpr (DF)
      lz_init_df<<<grid, THREADS, 0, s>>>(G_, static_cast<const double2*>(in), adjoint ? 1 : 0, f0, beta, invb,
                                          dfc, partials, counter);
    else
      lz_init<T><<<grid, THREADS, 0, s>>>(G_, static_cast<const double2*>(in), adjoint ? 1 : 0, f0, beta, invb,
                                          partials, counter);
    ++launches;
    e = cudaGetLastError();
  }

  // ---- first pass: Lanczos steps, convergence checked on the device ----
  const double dist = std::fabs(hmu);  // every pole's distance from the real axis
  const double Lh = std::fabs(tau) * k->rho_bound;
  int nsamp = (int)std::ceil(2.0 * Lh / (dist / 4.0)) + 1;
  nsamp = std::max(nsamp, kCoarse + 1);
  nsamp = (nsamp - 1 + kCoarse - 1) / kCoarse * kCoarse + 1;  // 1 mod kCoarse: symmetric coarse subgrid
  while (nsamp > nsamp_cap(M)) nsamp -= kCoarse;              // rho above the one behind M: coarser grid
  const double dl = 2.0 * Lh / (nsamp - 1);
  const int chunk = std::min(512, std::max(kChunk, npc / 128));
  const int G = bound_group(npc), groups = (npc + G - 1) / G;
  const int nslot_c = (nsamp - 1) / kCoarse + 1, nslot_f = nsamp;
  double* pin = k->pinned;
  // A Krylov polynomial of degree k resolves e^{ix} on [-Lh, Lh] only for k
  // of the order of Lh, so no chunk ending below Lh / 2 can meet the bound:
  // the bound is checked from there on (and at the step cap).
  const int first_check = (int)std::floor(0.5 * Lh);
  // the device's copy of the convergence test (lz_gate), zeroed with the counter
  unsigned* stop_w = counter + 1;
  const unsigned* stop = stop_w;
  // (b, coarse, fine) of a check for the host, beside the two maxima
  double* report = reinterpret_cast<double*>(maxslots + 2);
  // par: pinned slot and event of a checked chunk (alternating over checked chunks)
  auto launch_chunk = [&](int par, int j0, int j1, bool check) -> cudaError_t {
    for (int j = j0; j < j1; ++j) {
      if constexpr (DF)
        launch_step_pdl(lz_dfstep<0>, grid, s, G_, k->Hdf, k->wdf, j, Wptr(j - 1), Wptr(j - 2), Wptr(j), alpha, beta,
                        invb, dfc, partials, counter, static_cast<float2*>(nullptr),
                        static_cast<const float2*>(nullptr), stop);
      else if constexpr (REAL)
        lz_wstep<0><<<grid, THREADS, 0, s>>>(G_, j, Wptr(j - 1), Wptr(j - 2), Wptr(j), alpha, beta, invb, partials,
                                             counter, nullptr, nullptr, stop);
      else
        lz_step<0, T><<<grid, THREADS, 0, s>>>(G_, j, wptr(j - 1), vptr(j - 1), vptr(j), wptr(j), alpha, beta,
                                               invb, partials, counter, nullptr, nullptr, stop);
    }
    lz_poles_advance<<<(npc + kPoleThreads - 1) / kPoleThreads, kPoleThreads, 0, s>>>(
        npc, d_sc, d_wc, alpha, beta, j0, j1, d_dg, d_wy, stop, check ? maxslots : nullptr);
    if (!check) {
      launches += (j1 - j0) + 1;
      return cudaGetLastError();
    }
    cudaError_t err;
    const int sym = REAL ? (((j1 - 1) & 1) ? -1 : 1) : 0;  // (-1)^(k-1), k = j1 steps
    const dim3 gc((nslot_c + BT - 1) / BT, groups), gf((nslot_f + BT - 1) / BT, groups);
    lz_bound_part<<<gc, BT, 0, s>>>(npc, G, d_sc, d_wy, Lh, dl, nslot_c, kCoarse, beta, j1, k->rtol, nullptr,
                                    d_part, stop);
    lz_bound_max<<<gc.x, BT, 0, s>>>(groups, nslot_c, d_part, sym, beta, j1, k->rtol, nullptr, maxslots, stop);
    lz_bound_part<<<gf, BT, 0, s>>>(npc, G, d_sc, d_wy, Lh, dl, nslot_f, 1, beta, j1, k->rtol, maxslots, d_part,
                                    stop);
    lz_bound_max<<<gf.x, BT, 0, s>>>(groups, nslot_f, d_part, sym, beta, j1, k->rtol, maxslots, maxslots + 1,
                                     stop);
    lz_gate<<<1, 1, 0, s>>>(beta, j1, maxslots, k->rtol, stop_w, report);
    launches += (j1 - j0) + 6;
    err = cudaMemcpyAsync(pin + 3 * par, report, 3 * sizeof(double), cudaMemcpyDeviceToHost, s);
    if (err == cudaSuccess) err = cudaEventRecord(k->ev[par], s);
    if (err == cudaSuccess) err = cudaGetLastError();
    return err;
  };
  int kk = 0;
  bool converged = false, nonfinite = false;
  double bound = INFINITY;
  auto evaluate = [&](int par, int j1) -> cudaError_t {
    cudaError_t err = cudaEventSynchronize(k->ev[par]);
    if (err != cudaSuccess) return err;
    const double b = pin[3 * par], coarse = pin[3 * par + 1], fine = pin[3 * par + 2];
    if (!std::isfinite(b) || !std::isfinite(coarse) || !std::isfinite(fine)) {
      nonfinite = true;
      return cudaSuccess;
    }
    bound = b * coarse > k->rtol ? b * coarse : b * fine;
    if (bound <= k->rtol) {
      converged = true;
      kk = j1;
    }
    return cudaSuccess;
  };
  // the host evaluates a checked chunk while the next one runs
  int pending = -1, pending_j1 = 0, steps_run = 0, nchecked = 0;
  for (int c = 0; e == cudaSuccess; ++c) {
    const int j0 = c * chunk;
    if (j0 >= k->max_iters) break;
    const int j1 = std::min(j0 + chunk, k->max_iters);
    const bool check = j1 >= first_check || j1 >= k->max_iters;
    const int par = nchecked & 1;
    e = launch_chunk(par, j0, j1, check);
    steps_run = j1;
    if (e != cudaSuccess) break;
    if (!check) continue;
    ++nchecked;
    if (pending >= 0) {
      e = evaluate(pending, pending_j1);
      if (e != cudaSuccess || converged || nonfinite) break;
    }
    pending = par;
    pending_j1 = j1;
  }
  if (e == cudaSuccess && !converged && !nonfinite && pending >= 0) e = evaluate(pending, pending_j1);
  // the chunk enqueued behind the converged one finds the device's stop flag
  // set by the same test and returns at once: the steps run are kk
  if (converged) steps_run = kk;
  if (e != cudaSuccess) {
    set_last_error(cudaGetErrorString(e));
    return REXI_ECUDA;
  }
  if (nonfinite) {
    set_last_error("shared-Krylov method: non-finite Lanczos scalars");
    if (hooks.launches) *hooks.launches += launches;
    return REXI_ENOCONV;
  }
  if (!converged) {
    if (hooks.launches) *hooks.launches += launches;
    if (info) {
      memset(info, 0, sizeof(*info));
      info->N = N;
      info->krylov_iters = k->max_iters;
      info->krylov_unconverged = npc;
      info->krylov_max_rel_res = bound;
    }
    set_last_error("shared-Krylov method: step cap reached before the error bound");
    return REXI_ENOCONV;
  }
  mark(2);

  // ---- c = -i ||f|| sum_j beta_j (T_kk + s_j)^{-1} e_0, poles in chunks ----
  const int P = (int)std::min<size_t>((size_t)npc, L.scratch_bytes / ((size_t)kk * sizeof(double2)));
  for (int p0 = 0; p0 < npc && e == cudaSuccess; p0 += P) {
    const int Pc = std::min(P, npc - p0);
    lz_coeff_solve<<<(Pc + kPoleThreads - 1) / kPoleThreads, kPoleThreads, 0, s>>>(p0, Pc, d_sc, d_wc, alpha, beta, kk, scratch);
    lz_coeff_sum<<<kk, THREADS, 0, s>>>(Pc, scratch, cvec, p0 == 0 ? 1 : 0);
    launches += 2;
    e = cudaGetLastError();
  }
  mark(3);

  // ---- second pass: acc = V c from the kept vectors, the rest regenerated ----
  const int nb = std::min(nbasis, kk);
  if (e == cudaSuccess) {
    if constexpr (REAL) {
      lz_wcoef<<<(kk + 255) / 256, 256, 0, s>>>(cvec, invb, kk, coef, coef_df);
      ++launches;
      if constexpr (DF)
        lz_dfbasis_sum<<<ebl, 256, 0, s>>>(f0, basis, vstride, nb, coef_df, acc, n3);
      else
        lz_wbasis_sum<<<ebl, 256, 0, s>>>(f0, basis, vstride, nb, coef, acc, n3);
    } else {
      lz_basis_sum<T><<<ebl, 256, 0, s>>>(basis, vstride, nb, cvec, acc, n3);
    }
    ++launches;
  }
  if (e == cudaSuccess && nb < kk) {
    for (int j = nb; j < kk; ++j) {
      if constexpr (DF)
        launch_step_pdl(lz_dfstep<1>, grid, s, G_, k->Hdf, k->wdf, j, Wptr(j - 1), Wptr(j - 2), Wptr(j), alpha, beta,
                        invb, dfc, partials, counter, acc, coef_df, static_cast<const unsigned*>(nullptr));
      else if constexpr (REAL)
        lz_wstep<1><<<grid, THREADS, 0, s>>>(G_, j, Wptr(j - 1), Wptr(j - 2), Wptr(j), alpha, beta, invb, partials,
                                             counter, acc, coef, nullptr);
      else
        lz_step<1, T><<<grid, THREADS, 0, s>>>(G_, j, wptr(j - 1), vptr(j - 1), vptr(j), wptr(j), alpha, beta,
                                               invb, partials, counter, acc, cvec, nullptr);
    }
    launches += kk - nb;
  }
  if (e == cudaSuccess) {
    lz_finish<T><<<ebl, 256, 0, s>>>(acc, static_cast<double2*>(out), k->w64, nk, real_input, adjoint ? 1 : 0);
    ++launches;
    e = cudaGetLastError();
  }
  mark(4);
  if (hooks.launches) *hooks.launches += launches;
  if (e != cudaSuccess) {
    set_last_error(cudaGetErrorString(e));
    return REXI_ECUDA;
  }
  if (info) {
    memset(info, 0, sizeof(*info));
    info->N = N;
    info->n_terms = real_input ? N + 1 : 2 * N + 1;
    info->n_poles = npc_max;
    info->krylov_iters = kk;
    info->krylov_unconverged = 0;
    info->krylov_max_rel_res = bound;
    info->krylov_term_iters = steps_run;  // first-pass steps run
  }
  return REXI_OK;
}

// ---------------------------------------------------------------------------
// Depth gradient from two kept Lanczos bases (real input, FP64 real form).
//
// dL/dH_k = tau Re sum_j beta_j conj(y_j,eta,k) (div x_j)_k with
// x_j = (tau A - z_j)^{-1} f and y_j = (tau A - z_j)^{-H} G.  A is W-skew, so
// y_j = W (-tau A - conj z_j)^{-1} W^{-1} G: a Lanczos run on f (operator
// K = -i tau A, shifts i z_j) and one on W^{-1} G (operator i tau A, shifts
// i conj z_j) give x_j = -i ||f|| V c_j and y_j = -i ||W^{-1}G|| W V~ d_j with
// c_j, d_j the resolvent columns of the two tridiagonal matrices.  With the
// real-form vectors (v_b = i^b u_b) the gradient is
//   grad_k = w_k sum_{a,b} u~_{eta,a,k} R_ab (div u_b)_k,
//   R_ab = tau ||f|| ||W^{-1}G|| Re(i^{b-a} sum_j beta_j conj(d_ja) c_jb),
// a two-sided Galerkin form whose middle matrix holds the divided differences
// of r at pairs of Ritz values; it converges like the step itself (both runs
// stop on the step's error bound), not like the single poles.

// (T_k + s_p)^{-1} e_0 for every pole, out[i np + p] (UL sweep as lz_coeff_solve).
__global__ void lz_resolvent(int np, const double2* s, const double* alpha, const double* beta, int kk,
                             double2* out) {
  const int p = blockIdx.x * blockDim.x + threadIdx.x;
  if (p >= np) return;
  const double2 sp = s[p];
  double2 ip = crcp(make_double2(alpha[kk - 1] + sp.x, sp.y));
  out[(size_t)(kk - 1) * np + p] = ip;
#pragma unroll 4
  for (int i = kk - 2; i >= 0; --i) {
    const double b2 = beta[i + 1] * beta[i + 1];
    ip = crcp(make_double2(fma(-b2, ip.x, alpha[i] + sp.x), fma(-b2, ip.y, sp.y)));
    out[(size_t)i * np + p] = ip;
  }
  double2 y = ip;
  out[p] = y;
#pragma unroll 4
  for (int i = 1; i < kk; ++i) {
    const double2 t = cmuld(y, out[(size_t)i * np + p]);
    y = make_double2(-beta[i] * t.x, -beta[i] * t.y);
    out[(size_t)i * np + p] = y;
  }
}

// R[a kA + b] = tau b0A b0B invbB[a] invbA[b] Re(i^{b-a} sum_j w_j conj(DB[a][j]) CA[b][j]),
// 16 x 16 tiles, poles in chunks of 16 through shared memory.
__global__ void __launch_bounds__(256) lz_bilinear(int np, int kA, int kB, const double2* CA, const double2* DB,
                                                   const double2* w, const double* betaA, const double* invbA,
                                                   const double* betaB, const double* invbB, double tau, double* R) {
  __shared__ double2 Ds[16][17], Cs[16][17];
  const int ta = threadIdx.x / 16, tb = threadIdx.x % 16;
  const int a = blockIdx.y * 16 + ta, b = blockIdx.x * 16 + tb;
  double re = 0.0, im = 0.0;
  for (int j0 = 0; j0 < np; j0 += 16) {
    __syncthreads();
    {
      const int ra = blockIdx.y * 16 + ta, rb = blockIdx.x * 16 + ta, jj = j0 + tb;
      Ds[ta][tb] = (ra < kB && jj < np) ? DB[(size_t)ra * np + jj] : make_double2(0.0, 0.0);
      double2 c = (rb < kA && jj < np) ? CA[(size_t)rb * np + jj] : make_double2(0.0, 0.0);
      if (jj < np) {
        const double2 wj = w[jj];
        c = make_double2(wj.x * c.x - wj.y * c.y, wj.x * c.y + wj.y * c.x);
      }
      Cs[ta][tb] = c;
    }
    __syncthreads();
#pragma unroll
    for (int q = 0; q < 16; ++q) {
      const double2 d = Ds[ta][q], c = Cs[tb][q];
      re = fma(d.x, c.x, fma(d.y, c.y, re));  // conj(d) c
      im = fma(d.x, c.y, fma(-d.y, c.x, im));
    }
  }
  if (a < kB && b < kA)
    R[(size_t)a * kA + b] =
        tau * betaA[0] * betaB[0] * invbB[a] * invbA[b] * real_coeff(make_double2(re, im), (b - a) & 3);
}

// grad[p] += w[p] sum_b div(S_b)[p] sum_a R[a][b] S~_a,eta[p]; S_0 = f0, S_b = kept
// W_{b-1} (run on f), the same for S~ (run on W^{-1} G).
constexpr int kGB = 32, kGA = 64;
__global__ void __launch_bounds__(256) lz_grad_contract(int nx, int ny, double idx, double idy, const double* f0,
                                                        const double* basA, const double* g0, const double* basB,
                                                        size_t vstride, int kA, int kB, const double* R,
                                                        const double* w, double* grad) {
  __shared__ double Rs[kGA][kGB];
  const size_t nk = (size_t)nx * ny;
  const size_t p = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
  const bool live = p < nk;
  const int i = live ? (int)(p % nx) : 0, jrow = live ? (int)(p / nx) : 0;
  const size_t pxm = (size_t)jrow * nx + (i == 0 ? nx - 1 : i - 1);
  const size_t pym = (size_t)(jrow == 0 ? ny - 1 : jrow - 1) * nx + i;
  double acc = 0.0;
  for (int b0 = 0; b0 < kA; b0 += kGB) {
    double z[kGB];
#pragma unroll
    for (int q = 0; q < kGB; ++q) z[q] = 0.0;
    for (int a0 = 0; a0 < kB; a0 += kGA) {
      __syncthreads();
      for (int t = threadIdx.x; t < kGA * kGB; t += blockDim.x) {
        const int a = a0 + t / kGB, b = b0 + t % kGB;
        Rs[t / kGB][t % kGB] = (a < kB && b < kA) ? R[(size_t)a * kA + b] : 0.0;
      }
      __syncthreads();
      const int na = min(kGA, kB - a0);
      for (int q = 0; q < na; ++q) {
        const int a = a0 + q;
        const double sv = live ? (a == 0 ? g0[p] : basB[(size_t)(a - 1) * vstride + p]) : 0.0;
#pragma unroll
        for (int bb = 0; bb < kGB; ++bb) z[bb] = fma(Rs[q][bb], sv, z[bb]);
      }
    }
    if (!live) continue;
    const int nbb = min(kGB, kA - b0);
#pragma unroll
    for (int bb = 0; bb < kGB; ++bb) {
      if (bb >= nbb) break;
      const int b = b0 + bb;
      const double* S = b == 0 ? f0 : basA + (size_t)(b - 1) * vstride;
      const double dv = (S[nk + p] - S[nk + pxm]) * idx + (S[2 * nk + p] - S[2 * nk + pym]) * idy;
      acc = fma(z[bb], dv, acc);
    }
  }
  if (live) grad[p] += w[p] * acc;
}

// The same contraction in double-float arithmetic (mixed form) on bases kept
// as double-float pairs; R is split into (hi, lo) FP32 pairs on load (integer
// operations), products and sums run on the FP32 pipes; the result is added
// in FP64.
__global__ void __launch_bounds__(256) lz_grad_contract_df(int nx, int ny, double idx, double idy, const float2* f0,
                                                           const float2* basA, const float2* g0, const float2* basB,
                                                           size_t vstride, int kA, int kB, const double* R,
                                                           const double* w, double* grad) {
  __shared__ float2 Rs[kGA][kGB];
  const size_t nk = (size_t)nx * ny;
  const size_t p = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
  const bool live = p < nk;
  const int i = live ? (int)(p % nx) : 0, jrow = live ? (int)(p / nx) : 0;
  const size_t pxm = (size_t)jrow * nx + (i == 0 ? nx - 1 : i - 1);
  const size_t pym = (size_t)(jrow == 0 ? ny - 1 : jrow - 1) * nx + i;
  const float2 idx_df = df_from_double(idx), idy_df = df_from_double(idy);
  float2 acc = make_float2(0.f, 0.f);
  for (int b0 = 0; b0 < kA; b0 += kGB) {
    float2 z[kGB];
#pragma unroll
    for (int q = 0; q < kGB; ++q) z[q] = make_float2(0.f, 0.f);
    for (int a0 = 0; a0 < kB; a0 += kGA) {
      __syncthreads();
      for (int t = threadIdx.x; t < kGA * kGB; t += blockDim.x) {
        const int a = a0 + t / kGB, b = b0 + t % kGB;
        Rs[t / kGB][t % kGB] = (a < kB && b < kA) ? df_from_double(R[(size_t)a * kA + b]) : make_float2(0.f, 0.f);
      }
      __syncthreads();
      const int na = min(kGA, kB - a0);
      for (int q = 0; q < na; ++q) {
        const int a = a0 + q;
        const float2 sv = live ? (a == 0 ? g0[p] : basB[(size_t)(a - 1) * vstride + p]) : make_float2(0.f, 0.f);
#pragma unroll
        for (int bb = 0; bb < kGB; ++bb) {
          const float2 t = f_mul(Rs[q][bb].x, Rs[q][bb].y, sv.x, sv.y);
          z[bb] = f_add(z[bb].x, z[bb].y, t.x, t.y);
        }
      }
    }
    if (!live) continue;
    const int nbb = min(kGB, kA - b0);
#pragma unroll
    for (int bb = 0; bb < kGB; ++bb) {
      if (bb >= nbb) break;
      const int b = b0 + bb;
      const float2* S = b == 0 ? f0 : basA + (size_t)(b - 1) * vstride;
      const float2 ddx = f_subf(S[nk + p], S[nk + pxm]);
      const float2 ddy = f_subf(S[2 * nk + p], S[2 * nk + pym]);
      const float2 dv = f_addf(f_mulf(ddx, idx_df), f_mulf(ddy, idy_df));
      acc = f_addf(acc, f_mulf(z[bb], dv));
    }
  }
  if (live) grad[p] += w[p] * df_to_double(acc);
}

// Bytes of the gradient workspace; cap = kept Lanczos vectors per run.
int grad_cap(const KrylovSettings* k, int M, double h) {
  return (int)std::min<double>(k->max_iters, std::ceil(3.0 * M * h) + 100.0);
}
struct GLayout {
  size_t vb, f0, g0, basA, basB, alA, beA, ibA, alB, beB, ibB, sA, wA, sB, wB, dg, wy, part, maxslots, partials,
      counter, CA, DB, R, dfc, total;
  int cap;
};
GLayout grad_layout(const KrylovSettings* k, int M, double h) {
  GLayout L{};
  const size_t nk = (size_t)k->nx * k->ny;
  const size_t ntiles = (size_t)((k->nx + TX - 1) / TX) * ((k->ny + TY - 1) / TY);
  const size_t nmax = (size_t)k->max_iters + 2;
  const int np = poles_c(M, 1);
  L.cap = grad_cap(k, M, h);
  L.vb = al(3 * nk * sizeof(double));
  size_t o = 0;
  auto take = [&](size_t bytes) {
    const size_t at = o;
    o += al(bytes);
    return at;
  };
  L.f0 = take(L.vb);
  L.g0 = take(L.vb);
  L.basA = take((size_t)L.cap * L.vb);
  L.basB = take((size_t)L.cap * L.vb);
  L.alA = take(nmax * sizeof(double));
  L.beA = take(nmax * sizeof(double));
  L.ibA = take(nmax * sizeof(double));
  L.alB = take(nmax * sizeof(double));
  L.beB = take(nmax * sizeof(double));
  L.ibB = take(nmax * sizeof(double));
  L.sA = take((size_t)np * sizeof(double2));
  L.wA = take((size_t)np * sizeof(double2));
  L.sB = take((size_t)np * sizeof(double2));
  L.wB = take((size_t)np * sizeof(double2));
  L.dg = take((size_t)np * 2 * sizeof(double2));
  L.wy = take((size_t)np * sizeof(double2));
  L.part = take((size_t)128 * nsamp_cap(M) * sizeof(double2));
  L.maxslots = take(256);
  L.partials = take(ntiles * sizeof(double2));
  L.counter = take(256);
  L.CA = take((size_t)L.cap * np * sizeof(double2));
  L.DB = take((size_t)L.cap * np * sizeof(double2));
  L.R = take((size_t)L.cap * L.cap * sizeof(double));
  L.dfc = take(nmax * sizeof(DfCoef));
  L.total = o;
  return L;
}

}  // namespace

size_t lanczos_grad_workspace_bytes(const KrylovSettings* k, int M, double h) { return grad_layout(k, M, h).total; }

rexi_status krylov_grad_depth_lanczos(KrylovSettings* k, int form, double h, int M, const void* f_in,
                                      const void* g_out,
                                      double* grad_depth, double dt, void* ws, size_t ws_bytes, cudaStream_t s,
                                      rexi_step_info* info, const KrylovHooks& hooks) {
  using cd = std::complex<double>;
  auto mark = [&](int i) {
    if (hooks.mark) hooks.mark(hooks.ctx, i, s);
  };
  int64_t launches = 0;
  if (!(k->rho_bound > 0.0) || !k->pinned) {
    set_last_error("shared-Krylov method: plan has no spectral bound");
    return REXI_EINVAL;
  }
  const GLayout L = grad_layout(k, M, h);
  if (ws_bytes < L.total) {
    set_last_error("workspace too small for the shared-Krylov depth gradient");
    return REXI_ENOMEM;
  }
  const int N = M + kL;
  const size_t nk = (size_t)k->nx * k->ny;
  // reduced (real-input) pole set: run on f uses shifts i z_j with beta_j, the run
  // on W^{-1} G uses shifts i conj(z_j) with conj(beta_j)
  TermSet ts;
  rexii_terms(M, h, &ts);
  const double hmu = h * ts.mu;
  const cd I(0.0, 1.0);
  std::vector<double2> sA, wA, sB, wB;
  auto push = [&](cd z, cd w) {
    const cd a = I * z, b = I * std::conj(z), wc = std::conj(w);
    sA.push_back(make_double2(a.real(), a.imag()));
    wA.push_back(make_double2(w.real(), w.imag()));
    sB.push_back(make_double2(b.real(), b.imag()));
    wB.push_back(make_double2(wc.real(), wc.imag()));
  };
  for (int n = 0; n <= N; ++n) {
    const int i = n + N;
    const double gam = n > 0 ? 2.0 : 1.0;
    const cd C1(ts.c1re[i] * hmu + ts.c2re[i] * h * n, ts.c1im[i] * hmu + ts.c2im[i] * h * n);
    const cd C2 = I * cd(ts.c2re[i], ts.c2im[i]);
    const cd a_n(hmu, h * n), a_mn(hmu, -h * n);
    const cd P = (C1 - C2 * a_mn) / (2.0 * hmu), Q = (C1 + C2 * a_n) / (2.0 * hmu);
    push(a_mn, -gam * P);
    push(-a_n, gam * Q);
  }
  const int np = (int)sA.size();
  char* base = static_cast<char*>(ws);
  auto D = [&](size_t off) { return reinterpret_cast<double*>(base + off); };
  auto D2 = [&](size_t off) { return reinterpret_cast<double2*>(base + off); };
  double2* partials = D2(L.partials);
  unsigned* counter = reinterpret_cast<unsigned*>(base + L.counter);
  unsigned long long* maxslots = reinterpret_cast<unsigned long long*>(base + L.maxslots);
  const size_t vstride = L.vb / sizeof(double);
  // mixed form: Lanczos runs and the contraction in double-float
  const bool df = form == REXI_FORM_MIXED;

  mark(0);
  cudaError_t e = cudaMemcpyAsync(D2(L.sA), sA.data(), np * sizeof(double2), cudaMemcpyHostToDevice, s);
  if (e == cudaSuccess) e = cudaMemcpyAsync(D2(L.wA), wA.data(), np * sizeof(double2), cudaMemcpyHostToDevice, s);
  if (e == cudaSuccess) e = cudaMemcpyAsync(D2(L.sB), sB.data(), np * sizeof(double2), cudaMemcpyHostToDevice, s);
  if (e == cudaSuccess) e = cudaMemcpyAsync(D2(L.wB), wB.data(), np * sizeof(double2), cudaMemcpyHostToDevice, s);
  if (e == cudaSuccess) e = cudaMemsetAsync(counter, 0, sizeof(unsigned), s);
  mark(1);

  const double dist = std::fabs(hmu);
  const double Lh = std::fabs(dt) * k->rho_bound;
  int nsamp = (int)std::ceil(2.0 * Lh / (dist / 4.0)) + 1;
  nsamp = std::max(nsamp, kCoarse + 1);
  nsamp = (nsamp - 1 + kCoarse - 1) / kCoarse * kCoarse + 1;
  while (nsamp > nsamp_cap(M)) nsamp -= kCoarse;
  const double dl = 2.0 * Lh / (nsamp - 1);
  const int chunk = std::min(512, std::max(kChunk, np / 128));
  const int Gp = bound_group(np), groups = (np + Gp - 1) / Gp;
  const int nslot_c = (nsamp - 1) / kCoarse + 1, nslot_f = nsamp;
  double* pin = k->pinned;

  // One first pass with every vector kept (slot j = W_j); returns its step count.
  auto keep_run = [&](double tau, const double2* src, int adjoint, double* f0, double* bas, double* alpha,
                      double* beta, double* invb, const double2* d_s, const double2* d_w, int* kk_out,
                      double* bound_out) -> rexi_status {
    LGeom G;
    G.nx = k->nx;
    G.ny = k->ny;
    G.tiles_x = (k->nx + TX - 1) / TX;
    G.tiles_y = (k->ny + TY - 1) / TY;
    G.fstride = nk;
    const double idx = k->nx / k->Lx, idy = k->ny / k->Ly;
    G.tdx = tau * idx;
    G.tdy = tau * idy;
    G.tgdx = tau * k->g * idx;
    G.tgdy = tau * k->g * idy;
    G.tf4 = 0.25 * tau * k->f;
    G.H = k->depth;
    G.w = k->w64;
    const dim3 grid(G.tiles_x, G.tiles_y, 1);
    // mixed form: the kept vectors are double-float pairs (8 bytes per value, as FP64)
    auto W = [&](int j) -> double* { return j < -1 ? nullptr : (j == -1 ? f0 : bas + (size_t)j * vstride); };
    auto Wf = [&](int j) -> float2* { return reinterpret_cast<float2*>(W(j)); };
    DfCoef* dfc = reinterpret_cast<DfCoef*>(base + L.dfc);
    // this run's stop flag (lz_gate), cleared after the previous run's steps
    unsigned* stop = counter + 1;
    if (cudaMemsetAsync(stop, 0, sizeof(unsigned), s) != cudaSuccess) {
      set_last_error("shared-Krylov depth gradient: clearing the stop flag failed");
      return REXI_ECUDA;
    }
    if (df)
      lz_init_df<<<grid, THREADS, 0, s>>>(G, src, adjoint, Wf(-1), beta, invb, dfc, partials, counter);
    else
      lz_init<double><<<grid, THREADS, 0, s>>>(G, src, adjoint, f0, beta, invb, partials, counter);
    ++launches;
    cudaError_t err = cudaGetLastError();
    bool converged = false, nonfinite = false;
    int kk = 0, pending = -1, pending_j1 = 0;
    double bound = INFINITY;
    auto evaluate = [&](int par, int j1) -> cudaError_t {
      cudaError_t er = cudaEventSynchronize(k->ev[par]);
      if (er != cudaSuccess) return er;
      const double b = pin[3 * par], coarse = pin[3 * par + 1], fine = pin[3 * par + 2];
      if (!std::isfinite(b) || !std::isfinite(coarse) || !std::isfinite(fine)) {
        nonfinite = true;
        return cudaSuccess;
      }
      bound = b * coarse > k->rtol ? b * coarse : b * fine;
      if (bound <= k->rtol) {
        converged = true;
        kk = j1;
      }
      return cudaSuccess;
    };
    // checks from Lh / 2 on, as in the step's first pass
    const int first_check = (int)std::floor(0.5 * Lh);
    int nchecked = 0;
    for (int c = 0; err == cudaSuccess; ++c) {
      const int j0 = c * chunk;
      if (j0 >= L.cap) break;
      const int j1 = std::min(j0 + chunk, L.cap);
      for (int j = j0; j < j1; ++j) {
        if (df)
          launch_step_pdl(lz_dfstep<0>, grid, s, G, k->Hdf, k->wdf, j, Wf(j - 1), Wf(j - 2), Wf(j), alpha, beta,
                          invb, dfc, partials, counter, static_cast<float2*>(nullptr),
                          static_cast<const float2*>(nullptr), static_cast<const unsigned*>(stop));
        else
          lz_wstep<0><<<grid, THREADS, 0, s>>>(G, j, W(j - 1), W(j - 2), W(j), alpha, beta, invb, partials, counter,
                                               nullptr, nullptr, stop);
      }
      const bool check = !(j1 < first_check && j1 < L.cap);
      lz_poles_advance<<<(np + kPoleThreads - 1) / kPoleThreads, kPoleThreads, 0, s>>>(
          np, d_s, d_w, alpha, beta, j0, j1, D2(L.dg), D2(L.wy), stop, check ? maxslots : nullptr);
      if (!check) {
        launches += (j1 - j0) + 1;
        err = cudaGetLastError();
        continue;
      }
      const int par = nchecked++ & 1;
      const int sym = ((j1 - 1) & 1) ? -1 : 1;
      const dim3 gc((nslot_c + BT - 1) / BT, groups), gf((nslot_f + BT - 1) / BT, groups);
      lz_bound_part<<<gc, BT, 0, s>>>(np, Gp, d_s, D2(L.wy), Lh, dl, nslot_c, kCoarse, beta, j1, k->rtol, nullptr,
                                      D2(L.part), stop);
      lz_bound_max<<<gc.x, BT, 0, s>>>(groups, nslot_c, D2(L.part), sym, beta, j1, k->rtol, nullptr, maxslots, stop);
      lz_bound_part<<<gf, BT, 0, s>>>(np, Gp, d_s, D2(L.wy), Lh, dl, nslot_f, 1, beta, j1, k->rtol, maxslots,
                                      D2(L.part), stop);
      lz_bound_max<<<gf.x, BT, 0, s>>>(groups, nslot_f, D2(L.part), sym, beta, j1, k->rtol, maxslots,
                                       maxslots + 1, stop);
      double* report = reinterpret_cast<double*>(maxslots + 2);  // (b, coarse, fine) for the host
      lz_gate<<<1, 1, 0, s>>>(beta, j1, maxslots, k->rtol, stop, report);
      launches += (j1 - j0) + 6;
      err = cudaMemcpyAsync(pin + 3 * par, report, 3 * sizeof(double), cudaMemcpyDeviceToHost, s);
      if (err == cudaSuccess) err = cudaEventRecord(k->ev[par], s);
      if (err == cudaSuccess) err = cudaGetLastError();
      if (err != cudaSuccess) break;
      if (pending >= 0) {
        err = evaluate(pending, pending_j1);
        if (err != cudaSuccess || converged || nonfinite) break;
      }
      pending = par;
      pending_j1 = j1;
    }
    if (err == cudaSuccess && !converged && !nonfinite && pending >= 0) err = evaluate(pending, pending_j1);
    if (err != cudaSuccess) {
      set_last_error(cudaGetErrorString(err));
      return REXI_ECUDA;
    }
    *bound_out = bound;
    if (!converged) {
      set_last_error(nonfinite ? "shared-Krylov depth gradient: non-finite Lanczos scalars"
                               : "shared-Krylov depth gradient: step cap reached before the error bound");
      return REXI_ENOCONV;
    }
    *kk_out = kk;
    return REXI_OK;
  };

  int kA = 0, kB = 0;
  double bA = 0.0, bB = 0.0;
  rexi_status st = e == cudaSuccess ? REXI_OK : REXI_ECUDA;
  if (e != cudaSuccess) set_last_error(cudaGetErrorString(e));
  if (st == REXI_OK)
    st = keep_run(dt, static_cast<const double2*>(f_in), 0, D(L.f0), D(L.basA), D(L.alA), D(L.beA), D(L.ibA),
                  D2(L.sA), D2(L.wA), &kA, &bA);
  if (st == REXI_OK)  // W^{-1} G under -tau A
    st = keep_run(-dt, static_cast<const double2*>(g_out), 1, D(L.g0), D(L.basB), D(L.alB), D(L.beB), D(L.ibB),
                  D2(L.sB), D2(L.wB), &kB, &bB);
  mark(2);
  if (st == REXI_OK) {
    lz_resolvent<<<(np + kPoleThreads - 1) / kPoleThreads, kPoleThreads, 0, s>>>(np, D2(L.sA), D(L.alA), D(L.beA), kA, D2(L.CA));
    lz_resolvent<<<(np + kPoleThreads - 1) / kPoleThreads, kPoleThreads, 0, s>>>(np, D2(L.sB), D(L.alB), D(L.beB), kB, D2(L.DB));
    lz_bilinear<<<dim3((kA + 15) / 16, (kB + 15) / 16), 256, 0, s>>>(np, kA, kB, D2(L.CA), D2(L.DB), D2(L.wA),
                                                                     D(L.beA), D(L.ibA), D(L.beB), D(L.ibB), dt,
                                                                     D(L.R));
    launches += 3;
    mark(3);
    auto F = [&](size_t off) { return reinterpret_cast<const float2*>(base + off); };
    if (df)
      lz_grad_contract_df<<<(unsigned)((nk + 255) / 256), 256, 0, s>>>(
          k->nx, k->ny, k->nx / k->Lx, k->ny / k->Ly, F(L.f0), F(L.basA), F(L.g0), F(L.basB), vstride, kA, kB,
          D(L.R), k->w64, grad_depth);
    else
      lz_grad_contract<<<(unsigned)((nk + 255) / 256), 256, 0, s>>>(
          k->nx, k->ny, k->nx / k->Lx, k->ny / k->Ly, D(L.f0), D(L.basA), D(L.g0), D(L.basB), vstride, kA, kB,
          D(L.R), k->w64, grad_depth);
    ++launches;
    e = cudaGetLastError();
    if (e != cudaSuccess) {
      set_last_error(cudaGetErrorString(e));
      st = REXI_ECUDA;
    }
  }
  mark(4);
  if (hooks.launches) *hooks.launches += launches;
  if (info) {
    memset(info, 0, sizeof(*info));
    info->N = N;
    info->n_terms = N + 1;
    info->n_poles = np;
    info->krylov_iters = std::max(kA, kB);
    info->krylov_unconverged = st == REXI_ENOCONV ? np : 0;
    info->krylov_max_rel_res = std::max(bA, bB);
    info->krylov_term_iters = (int64_t)kA + kB;
  }
  return st;
}

size_t lanczos_workspace_bytes(const KrylovSettings* k, int M, int real_input) {
  const int npc = poles_c(M, real_input);
  // real forms: 8-byte values (FP64 or double-float); complex form: 16 bytes
  return lz_layout(k, npc, M, real_input ? sizeof(double) : sizeof(double2)).min_total;
}

rexi_status lanczos_tables(KrylovSettings* k) {
  const size_t nk = (size_t)k->nx * k->ny;
  lz_df_tables<<<(unsigned)((nk + 255) / 256), 256>>>(k->depth, k->w64, nk, k->Hdf, k->wdf);
  const cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) {
    set_last_error(cudaGetErrorString(e));
    return REXI_ECUDA;
  }
  return REXI_OK;
}

rexi_status krylov_step_lanczos(KrylovSettings* k, int form, double h, int M, const void* in, void* out, double dt,
                                int real_input, int term_begin, int term_end, void* ws, size_t ws_bytes,
                                cudaStream_t s, rexi_step_info* info, bool adjoint, const KrylovHooks& hooks) {
  if (form == REXI_FORM_PLAIN) {
    set_last_error("variable-depth path: the plain form is Fourier-path only");
    return REXI_EUNSUPPORTED;
  }
  if (real_input && form == REXI_FORM_MIXED)
    return lanczos_impl<float2>(k, h, M, in, out, dt, 1, term_begin, term_end, ws, ws_bytes, s, info, adjoint,
                                hooks);
  if (real_input)
    return lanczos_impl<double>(k, h, M, in, out, dt, 1, term_begin, term_end, ws, ws_bytes, s, info, adjoint,
                                hooks);
  return lanczos_impl<double2>(k, h, M, in, out, dt, 0, term_begin, term_end, ws, ws_bytes, s, info, adjoint, hooks);
}

}  // namespace rexi
