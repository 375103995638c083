// Device helpers shared by the Fourier-path pole kernels (single instance and
// batched): the C-grid symbol, the combine step, the wavenumber pairing and
// the per-term arithmetic of the FP64 and double-float pole loops.
#pragma once

#include "dfloat.cuh"
#include "internal.h"

namespace rexi {

// ---------------------------------------------------------------------------
// Symbol of the C-grid operator at wavenumber k (half-angle form, no
// cancellation for small k).  With c = cos(theta/2), s = sin(theta/2):
//   forward difference  (e^{i theta} - 1)/dx  = (2 s / dx)(-s + i c)
//   backward difference (1 - e^{-i theta})/dx = (2 s / dx)( s + i c)
//   P = (1 + e^{i theta_x})(1 + e^{-i theta_y}) / 4 = cx cy (cx + i sx)(cy - i sy)
//   omega^2 = g H (4 sx^2/dx^2 + 4 sy^2/dy^2) + f^2 cx^2 cy^2
struct Symbol {
  double2 dxf, dyf, dxb, dyb, P;
  double omega;
};

__device__ __forceinline__ Symbol symbol_at(const SymbolParams& sp, int kx, int ky) {
  if (sp.spectral == 2) {
    // scalar operator i (d_xx + d_yy) (second-order centred differences):
    // eigenvalue i lambda(k), lambda = -(4/dx^2) sin^2(pi kx/nx) - (4/dy^2) sin^2(pi ky/ny);
    // omega carries the signed lambda - sigma of the shifted operator A - i sigma I
    const double sx = sp.half_x[kx].y, sy = sp.half_y[ky].y;
    const double ax = 2.0 * sx * sp.inv_dx, ay = 2.0 * sy * sp.inv_dy;
    Symbol S;
    S.dxf = S.dxb = S.dyf = S.dyb = S.P = make_double2(0.0, 0.0);
    S.omega = -(ax * ax + ay * ay) - sp.shift;
    return S;
  }
  if (sp.spectral) {
    // spectral derivative i k' with the signed wavenumber (Nyquist taken as +n/2),
    // k' = 2 pi k_signed / L = 2 pi k_signed (1/dx) / n; no averaging (P = 1)
    const int sx = 2 * kx <= sp.nx ? kx : kx - sp.nx;
    const int sy = 2 * ky <= sp.ny ? ky : ky - sp.ny;
    const double kxp = 6.283185307179586 * sx * sp.inv_dx / sp.nx;
    const double kyp = 6.283185307179586 * sy * sp.inv_dy / sp.ny;
    Symbol S;
    S.dxf = S.dxb = make_double2(0.0, kxp);
    S.dyf = S.dyb = make_double2(0.0, kyp);
    S.P = make_double2(1.0, 0.0);
    S.omega = sqrt(sp.g * sp.H * (kxp * kxp + kyp * kyp) + sp.f * sp.f);
    return S;
  }
  const double2 hx = sp.half_x[kx];
  const double2 hy = sp.half_y[ky];
  const double cx = hx.x, sx = hx.y, cy = hy.x, sy = hy.y;
  Symbol S;
  const double ax = 2.0 * sx * sp.inv_dx, ay = 2.0 * sy * sp.inv_dy;
  S.dxf = make_double2(-ax * sx, ax * cx);
  S.dxb = make_double2(ax * sx, ax * cx);
  S.dyf = make_double2(-ay * sy, ay * cy);
  S.dyb = make_double2(ay * sy, ay * cy);
  const double cc = cx * cy;
  S.P = make_double2(cc * (cx * cy + sx * sy), cc * (sx * cy - cx * sy));
  const double w2 = sp.g * sp.H * (ax * ax + ay * ay) + sp.f * sp.f * cc * cc;
  S.omega = sqrt(w2);
  return S;
}

__device__ __forceinline__ double2 cm(double2 a, double2 b) {
  return make_double2(fma(a.x, b.x, -a.y * b.y), fma(a.x, b.y, a.y * b.x));
}
__device__ __forceinline__ double2 cj(double2 a) { return make_double2(a.x, -a.y); }
__device__ __forceinline__ double2 ca(double2 a, double2 b) { return make_double2(a.x + b.x, a.y + b.y); }
__device__ __forceinline__ double2 cs(double2 a, double2 b) { return make_double2(a.x - b.x, a.y - b.y); }
__device__ __forceinline__ double2 cr(double a, double2 b) { return make_double2(a * b.x, a * b.y); }

// y = B f (conj_sym: use conj(B), the symbol at -k; adjoint: use B^H).
__device__ __forceinline__ void apply_B(const Symbol& S, const SymbolParams& sp, bool conj_sym,
                                        bool adjoint, const double2 f[3], double2 y[3]) {
  double2 dxf = S.dxf, dyf = S.dyf, dxb = S.dxb, dyb = S.dyb, P = S.P;
  if (conj_sym) {
    dxf = cj(dxf); dyf = cj(dyf); dxb = cj(dxb); dyb = cj(dyb); P = cj(P);
  }
  if (!adjoint) {
    // [[0, -H dxb, -H dyb], [-g dxf, 0, f P], [-g dyf, -f conj(P), 0]]
    y[0] = cr(-sp.H, ca(cm(dxb, f[1]), cm(dyb, f[2])));
    y[1] = cs(cr(sp.f, cm(P, f[2])), cr(sp.g, cm(dxf, f[0])));
    y[2] = cs(cr(-sp.g, cm(dyf, f[0])), cr(sp.f, cm(cj(P), f[1])));
  } else {
    // B^H = [[0, -g conj(dxf), -g conj(dyf)], [-H conj(dxb), 0, -f P], [-H conj(dyb), f conj(P), 0]]
    y[0] = cr(-sp.g, ca(cm(cj(dxf), f[1]), cm(cj(dyf), f[2])));
    y[1] = cs(cr(-sp.H, cm(cj(dxb), f[0])), cr(sp.f, cm(P, f[2])));
    y[2] = ca(cr(-sp.H, cm(cj(dyb), f[0])), cr(sp.f, cm(cj(P), f[1])));
  }
}

// out = R0 f + Im(R+) Bt f + (R0 - Re R+) Bt^2 f, Bt = B / omega, in place on
// the three fields of wavenumber index `idx` (field stride fs).
__device__ __forceinline__ void combine(double2* spec, size_t idx, size_t fs, const Symbol& S,
                                        const SymbolParams& sp, bool conj_sym, bool adjoint,
                                        double2 R0, double2 Rp) {
  double2 f[3], y1[3], y2[3];
#pragma unroll
  for (int c = 0; c < 3; ++c) f[c] = spec[idx + c * fs];
  double2 c0 = adjoint ? cj(R0) : R0;
  double2 out[3];
  if (S.omega > 0.0) {
    const double inv = 1.0 / S.omega;
    apply_B(S, sp, conj_sym, adjoint, f, y1);
#pragma unroll
    for (int c = 0; c < 3; ++c) y1[c] = cr(inv, y1[c]);
    apply_B(S, sp, conj_sym, adjoint, y1, y2);
#pragma unroll
    for (int c = 0; c < 3; ++c) y2[c] = cr(inv, y2[c]);
    const double a1 = Rp.y;
    double2 a2 = make_double2(R0.x - Rp.x, R0.y);
    if (adjoint) a2 = cj(a2);
#pragma unroll
    for (int c = 0; c < 3; ++c) out[c] = ca(ca(cm(c0, f[c]), cr(a1, y1[c])), cm(a2, y2[c]));
  } else {
#pragma unroll
    for (int c = 0; c < 3; ++c) out[c] = cm(c0, f[c]);
  }
#pragma unroll
  for (int c = 0; c < 3; ++c) spec[idx + c * fs] = out[c];
}

// Per-orbit scalars of the combine step: with y1 = B f and y2 = B^2 f
// (unscaled), r(tau B) f = c0 f + s1 y1 + s2 y2, s1 = Im(R+)/omega,
// s2 = (R0 - Re R+)/omega^2 (0 and 0 at omega = 0, where B = 0).
struct OrbitScalars {
  double s1, s2re, s2im, pad;
};

__device__ __forceinline__ OrbitScalars orbit_scalars(double omega, double2 R0, double2 Rp) {
  OrbitScalars o;
  o.pad = 0.0;
  if (omega > 0.0) {
    const double iw = 1.0 / omega, iw2 = iw * iw;
    o.s1 = Rp.y * iw;
    o.s2re = (R0.x - Rp.x) * iw2;
    o.s2im = R0.y * iw2;
  } else {
    o.s1 = o.s2re = o.s2im = 0.0;
  }
  return o;
}

// The six nonzero entries of B(k) with g, H and f folded in (or of B^H for
// the adjoint: (B^H)_ij = conj(B_ji)):
//   y0 = e01 f1 + e02 f2,  y1 = e10 f0 + e12 f2,  y2 = e20 f0 + e21 f1.
struct SymbolEntries {
  double2 e01, e02, e10, e12, e20, e21;
};

__device__ __forceinline__ SymbolEntries symbol_entries(const SymbolParams& sp, int kx, int ky, bool adjoint) {
  const Symbol S = symbol_at(sp, kx, ky);
  SymbolEntries E;
  E.e01 = cr(-sp.H, S.dxb);
  E.e02 = cr(-sp.H, S.dyb);
  E.e10 = cr(-sp.g, S.dxf);
  E.e12 = cr(sp.f, S.P);
  E.e20 = cr(-sp.g, S.dyf);
  E.e21 = cr(-sp.f, cj(S.P));
  if (adjoint) {
    const SymbolEntries F = E;
    E.e01 = cj(F.e10);
    E.e02 = cj(F.e20);
    E.e10 = cj(F.e01);
    E.e12 = cj(F.e21);
    E.e20 = cj(F.e02);
    E.e21 = cj(F.e12);
  }
  return E;
}

// a b + c
__device__ __forceinline__ double2 cma(double2 a, double2 b, double2 c) {
  return make_double2(fma(a.x, b.x, fma(-a.y, b.y, c.x)), fma(a.x, b.y, fma(a.y, b.x, c.y)));
}

__device__ __forceinline__ void apply_entries(const SymbolEntries& E, const double2 f[3], double2 y[3]) {
  y[0] = cma(E.e01, f[1], cm(E.e02, f[2]));
  y[1] = cma(E.e10, f[0], cm(E.e12, f[2]));
  y[2] = cma(E.e20, f[0], cm(E.e21, f[1]));
}

// out = c0 f + s1 B f + s2 B^2 f in place at wavenumber index idx (field
// stride fs); for the adjoint c0 and s2 are conjugated and B is B^H.
__device__ __forceinline__ void combine_scaled(double2* spec, size_t idx, size_t fs, const SymbolEntries& E,
                                               double2 c0, OrbitScalars o, bool adjoint) {
  double2 f[3], y1[3], y2[3];
#pragma unroll
  for (int c = 0; c < 3; ++c) f[c] = spec[idx + c * fs];
  double2 s2 = make_double2(o.s2re, o.s2im);
  if (adjoint) {
    c0 = cj(c0);
    s2 = cj(s2);
  }
  apply_entries(E, f, y1);
  apply_entries(E, y1, y2);
#pragma unroll
  for (int c = 0; c < 3; ++c) {
    const double2 t = cm(c0, f[c]);
    const double2 u = make_double2(fma(o.s1, y1[c].x, t.x), fma(o.s1, y1[c].y, t.y));
    spec[idx + c * fs] = cma(s2, y2[c], u);
  }
}

// Double-float combine on a double-float half spectrum (real input, C-grid):
// out = c0 f + s1 B f + s2 B^2 f with real c0 = Re R0, s1, s2; the symbol from
// double-float half-angle tables (cos, sin of pi k / n as float4 hi/lo pairs).
struct SymbolDF {
  float2 g, H, f, inv_dx, inv_dy;
  const float4* half_x;
  const float4* half_y;
};

__device__ __forceinline__ float4 c_of(float2 re, float2 im) { return make_float4(re.x, re.y, im.x, im.y); }
__device__ __forceinline__ float2 f_neg(float2 a) { return make_float2(-a.x, -a.y); }

// The six non-zero entries of the C-grid symbol at (kx, ky) in double-float
// (B^H for the adjoint): e[0..5] = B01, B02, B10, B12, B20, B21.
__device__ __forceinline__ void symbol_df(const SymbolDF& sd, int kx, int ky, bool adjoint, float4 e[6]) {
  const float4 hx = sd.half_x[kx], hy = sd.half_y[ky];
  const float2 cx = make_float2(hx.x, hx.y), sx = make_float2(hx.z, hx.w);
  const float2 cy = make_float2(hy.x, hy.y), sy = make_float2(hy.z, hy.w);
  const float2 ax = f_mulf(make_float2(2.f * sx.x, 2.f * sx.y), sd.inv_dx);
  const float2 ay = f_mulf(make_float2(2.f * sy.x, 2.f * sy.y), sd.inv_dy);
  const float2 Hax = f_neg(f_mulf(sd.H, ax)), Hay = f_neg(f_mulf(sd.H, ay));
  const float2 gax = f_mulf(sd.g, ax), gay = f_mulf(sd.g, ay);
  e[0] = c_of(f_mulf(Hax, sx), f_mulf(Hax, cx));        // -H dxb
  e[1] = c_of(f_mulf(Hay, sy), f_mulf(Hay, cy));        // -H dyb
  e[2] = c_of(f_mulf(gax, sx), f_neg(f_mulf(gax, cx)));  // -g dxf
  e[4] = c_of(f_mulf(gay, sy), f_neg(f_mulf(gay, cy)));  // -g dyf
  const float2 cxcy = f_mulf(cx, cy);
  const float2 fcc = f_mulf(sd.f, cxcy);
  const float2 pr = f_mulf(fcc, f_addf(cxcy, f_mulf(sx, sy)));
  const float2 pim = f_mulf(fcc, f_subf(f_mulf(sx, cy), f_mulf(cx, sy)));
  e[3] = c_of(pr, pim);          // f P
  e[5] = c_of(f_neg(pr), pim);   // -f conj(P)
  if (adjoint) {  // (B^H)_ij = conj(B_ji)
    const float4 t01 = e[0], t02 = e[1], t10 = e[2], t12 = e[3], t20 = e[4], t21 = e[5];
    e[0] = cconj(t10);
    e[1] = cconj(t20);
    e[2] = cconj(t01);
    e[3] = cconj(t21);
    e[4] = cconj(t02);
    e[5] = cconj(t12);
  }
}

// Complex input on an FP64 spectrum: values become double-float pairs on load
// and FP64 again on store; out = c0 f + s1 B f + s2 B^2 f with c0 and s2
// complex (r(0) enters whole), s1 real.
__device__ __forceinline__ void combine_dfc_at(double2* spec, size_t k, size_t nk, int kx, int ky, const SymbolDF& sd,
                                               float4 c0, float2 s1, float4 s2, bool adjoint) {
  float4 e[6];
  symbol_df(sd, kx, ky, adjoint, e);
  float4 f[3], y1[3], y2[3];
#pragma unroll
  for (int c = 0; c < 3; ++c) {
    const double2 v = spec[k + c * nk];
    f[c] = c_of(df_from_double(v.x), df_from_double(v.y));
  }
  y1[0] = cadd(cmul(e[0], f[1]), cmul(e[1], f[2]));
  y1[1] = cadd(cmul(e[2], f[0]), cmul(e[3], f[2]));
  y1[2] = cadd(cmul(e[4], f[0]), cmul(e[5], f[1]));
  y2[0] = cadd(cmul(e[0], y1[1]), cmul(e[1], y1[2]));
  y2[1] = cadd(cmul(e[2], y1[0]), cmul(e[3], y1[2]));
  y2[2] = cadd(cmul(e[4], y1[0]), cmul(e[5], y1[1]));
#pragma unroll
  for (int c = 0; c < 3; ++c) {
    const float4 o = cadd(cadd(cmul(c0, f[c]), crmul(s1, y1[c])), cmul(s2, y2[c]));
    spec[k + c * nk] = make_double2(df_to_double(make_float2(o.x, o.y)), df_to_double(make_float2(o.z, o.w)));
  }
}

// In place at index k of the three fields (field stride nk), wavenumber (kx, ky).
__device__ __forceinline__ void combine_df_at(float4* spec, size_t k, size_t nk, int kx, int ky, const SymbolDF& sd,
                                              float2 c0, float2 s1, float2 s2, bool adjoint) {
  const float4 hx = sd.half_x[kx], hy = sd.half_y[ky];
  const float2 cx = make_float2(hx.x, hx.y), sx = make_float2(hx.z, hx.w);
  const float2 cy = make_float2(hy.x, hy.y), sy = make_float2(hy.z, hy.w);
  // a = 2 sin(theta/2) / dx; B entries with g, H, f folded in (see symbol_at)
  const float2 ax = f_mulf(make_float2(2.f * sx.x, 2.f * sx.y), sd.inv_dx);
  const float2 ay = f_mulf(make_float2(2.f * sy.x, 2.f * sy.y), sd.inv_dy);
  const float2 Hax = f_neg(f_mulf(sd.H, ax)), Hay = f_neg(f_mulf(sd.H, ay));
  const float2 gax = f_mulf(sd.g, ax), gay = f_mulf(sd.g, ay);
  float4 e01 = c_of(f_mulf(Hax, sx), f_mulf(Hax, cx));        // -H dxb
  float4 e02 = c_of(f_mulf(Hay, sy), f_mulf(Hay, cy));        // -H dyb
  float4 e10 = c_of(f_mulf(gax, sx), f_neg(f_mulf(gax, cx)));  // -g dxf
  float4 e20 = c_of(f_mulf(gay, sy), f_neg(f_mulf(gay, cy)));  // -g dyf
  const float2 cxcy = f_mulf(cx, cy);
  const float2 fcc = f_mulf(sd.f, cxcy);
  const float2 pr = f_mulf(fcc, f_addf(cxcy, f_mulf(sx, sy)));
  const float2 pim = f_mulf(fcc, f_subf(f_mulf(sx, cy), f_mulf(cx, sy)));
  float4 e12 = c_of(pr, pim);          // f P
  float4 e21 = c_of(f_neg(pr), pim);   // -f conj(P)
  if (adjoint) {  // B^H: (B^H)_ij = conj(B_ji)
    const float4 t01 = e01, t02 = e02, t10 = e10, t12 = e12, t20 = e20, t21 = e21;
    e01 = cconj(t10);
    e02 = cconj(t20);
    e10 = cconj(t01);
    e12 = cconj(t21);
    e20 = cconj(t02);
    e21 = cconj(t12);
  }
  float4 f[3], y1[3], y2[3];
#pragma unroll
  for (int c = 0; c < 3; ++c) f[c] = spec[k + c * nk];
  y1[0] = cadd(cmul(e01, f[1]), cmul(e02, f[2]));
  y1[1] = cadd(cmul(e10, f[0]), cmul(e12, f[2]));
  y1[2] = cadd(cmul(e20, f[0]), cmul(e21, f[1]));
  y2[0] = cadd(cmul(e01, y1[1]), cmul(e02, y1[2]));
  y2[1] = cadd(cmul(e10, y1[0]), cmul(e12, y1[2]));
  y2[2] = cadd(cmul(e20, y1[0]), cmul(e21, y1[1]));
#pragma unroll
  for (int c = 0; c < 3; ++c)
    spec[k + c * nk] = cadd(cadd(crmul(c0, f[c]), crmul(s1, y1[c])), crmul(s2, y2[c]));
}

// Map thread -> wavenumber pair.  Pairs (k, -k) with ky in [0, ny/2]; in the
// self-conjugate rows (ky = 0, and ky = ny/2 for even ny) only kx <= nx/2.
// omega(-k) = omega(k), so one pole loop serves both; the combine step takes
// each wavenumber's own symbol (for the spectral symbol the Nyquist
// derivative i k' is not the conjugate of its partner's).
__device__ __forceinline__ bool pair_of(int p, int nx, int ny, int& kx, int& ky, int& kx2, int& ky2) {
  ky = p / nx;
  kx = p - ky * nx;
  if (ky > ny / 2) return false;
  const bool selfrow = (ky == 0) || (2 * ky == ny);
  if (selfrow && kx > nx / 2) return false;
  kx2 = kx == 0 ? 0 : nx - kx;
  ky2 = ky == 0 ? 0 : ny - ky;
  return true;
}

// Orbit of wavenumber (kx, ky): fold each index to a = min(k, n - k), then,
// on a swap-symmetric grid, order the pair (a <= b).  Index: b (b + 1)/2 + a
// (triangular) or b ax + a (rectangular).
__device__ __forceinline__ int orbit_of(const OrbitParams& op, int nx, int ny, int kx, int ky) {
  int a = min(kx, nx - kx), b = min(ky, ny - ky);
  if (op.sym) {
    if (a > b) { const int t = a; a = b; b = t; }
    return b * (b + 1) / 2 + a;
  }
  return b * op.ax + a;
}
// Representative (a, b) of orbit o; a and b are themselves valid wavenumber
// indices (a <= nx/2, b <= ny/2).
__device__ __forceinline__ void orbit_rep(const OrbitParams& op, int o, int& a, int& b) {
  if (op.sym) {
    b = (int)((sqrtf(8.0f * (float)o + 1.0f) - 1.0f) * 0.5f);
    while (b > 0 && b * (b + 1) / 2 > o) --b;
    while ((b + 1) * (b + 2) / 2 <= o) ++b;
    a = o - b * (b + 1) / 2;
  } else {
    b = o / op.ax;
    a = o - b * op.ax;
  }
}

// ---------------------------------------------------------------------------
// FP64 fused pole loop.
// Table (per scalar term, 6 doubles): h n, A_re, A_im, B_re, B_im, 0 with
// A = c1_n h mu, B = c2_n.

__device__ __forceinline__ double rcp_seed(double d) {
  double r;
  asm("rcp.approx.ftz.f64 %0, %1;" : "=d"(r) : "d"(d));
  return r;
}

constexpr int kChunk = 256;  // terms staged in shared memory at a time

// ---------------------------------------------------------------------------
// Double-float fused pole loop.
// A value v is carried as an unevaluated sum hi + lo of two FP32 numbers.
// Error-free transformations (Knuth TwoSum, Dekker TwoProduct via FMA); the
// _rn intrinsics keep the compiler from contracting or reassociating them.

__device__ __forceinline__ void two_sum(float a, float b, float& s, float& e) {
  s = __fadd_rn(a, b);
  const float bb = __fsub_rn(s, a);
  e = __fadd_rn(__fsub_rn(a, __fsub_rn(s, bb)), __fsub_rn(b, bb));
}
__device__ __forceinline__ void fast_two_sum(float a, float b, float& s, float& e) {  // |a| >= |b| or a == 0
  s = __fadd_rn(a, b);
  e = __fsub_rn(b, __fsub_rn(s, a));
}
__device__ __forceinline__ float rcp_approx_f32(float x) {
  float r;
  asm("rcp.approx.ftz.f32 %0, %1;" : "=f"(r) : "f"(x));
  return r;
}


// One scalar REXII term in FP64: acc += (A + B y) / (q + y^2), y = x + h n.
// Table entry (3 double2): (h n, A_re), (A_im, B_re), (B_im, 0), A = c1 h mu, B = c2.
__device__ __forceinline__ void fp64_term(const double2* e, double x, double q, double& accr, double& acci) {
  const double2 e0 = e[0], e1 = e[1], e2 = e[2];
  const double y = x + e0.x;
  const double d = fma(y, y, q);
  const double r0 = rcp_seed(d);
  // 1/d = r0 / (1 - e) with e = 1 - d r0; r0 (1 + e + e^2) leaves a relative
  // error of order e^3 (a Newton-Raphson step plus its next term)
  const double er = fma(-d, r0, 1.0);
  const double r = fma(r0, fma(er, er, er), r0);
  accr = fma(fma(e1.y, y, e0.y), r, accr);
  acci = fma(fma(e2.x, y, e1.x), r, acci);
}

// acc += (a + b y) / d for one real component of a term, every quantity an
// FP32 (hi, lo) pair: a = (a_h, a_l), b = (b_h, b_l), y = (y_h, y_l),
// d = (d_h, d_l); r0 is an FP32 approximation of 1 / d_h (within one unit in
// the last place).  The quotient's high word is T_h = n_h r0 and its low word
// the remainder (n - T_h d) r0: n_h - T_h d_h is of order 2^-23 n_h and the
// FMA forms it to FP32 precision, so the low word is correct to about 2^-46
// of the quotient without a refined reciprocal.  The low word goes straight
// into the accumulator's low word (two roundings there per term).
__device__ __forceinline__ void df_quot_acc(float b_h, float b_l, float a_h, float a_l, float y_h, float y_l,
                                            float d_h, float d_l, float r0, float& acc_h, float& acc_l) {
  const float t_h = __fmul_rn(b_h, y_h);
  const float t_l = __fmaf_rn(b_h, y_h, -t_h);
  float n_h, n_e;
  two_sum(a_h, t_h, n_h, n_e);
  const float n_l = __fadd_rn(__fadd_rn(n_e, t_l), __fmaf_rn(b_h, y_l, __fmaf_rn(b_l, y_h, a_l)));
  const float T_h = __fmul_rn(n_h, r0);
  const float rem = __fmaf_rn(-T_h, d_l, __fadd_rn(__fmaf_rn(-T_h, d_h, n_h), n_l));
  float s, e;
  two_sum(acc_h, T_h, s, e);
  acc_h = s;
  acc_l = __fmaf_rn(rem, r0, __fadd_rn(acc_l, e));
}

// The accumulators' low words take two FP32 roundings per term and are not
// renormalised by the term itself; every kRenorm terms a FastTwoSum folds
// them back below half a unit of the high word, so that a low word never
// exceeds about kRenorm units of the partial sum's last place.
constexpr int kRenorm = 16;
__device__ __forceinline__ void df_renorm(float& h, float& l) { fast_two_sum(h, l, h, l); }

// One scalar REXII term in double-float arithmetic (see pole_fft.cu).
// x is split as X_hi (a multiple of the table's grid G) + X_lo + X_lo2 (FP32).
// acc += (A + B y) / (q + y^2) with every quantity an FP32 (hi, lo) pair.
// Table entry (3 float4): [hn_hi, Ar_hi, Ai_hi, Br_hi], [Bi_hi, Ar_lo, Ai_lo, Br_lo], [Bi_lo, hn_lo, hn_lo2, 0]
// (h n = hn_hi + hn_lo + hn_lo2, hn_hi on the grid G).
// EXACT_HN: every h n of the table lies on the grid G (hn_lo = 0, e.g. h = 0.5
// or 1), so only X_lo sits below the grid; otherwise hn_lo (up to G/2) joins
// X_lo by an error-free TwoSum first, which keeps (y_h, y_l) a normalised pair
// (a low word of order G would make the dropped y_l^2 and the FP32 rounding
// of the low words visible at the 1e-7 level).
template <bool EXACT_HN>
__device__ __forceinline__ void df_term(const float4* ent, float X_hi, float X_lo, float X_lo2, float q_hi,
                                        float q_lo, float& ar_h, float& ar_l, float& ai_h, float& ai_l) {
  const float4 e0 = ent[0], e1 = ent[1], e2 = ent[2];
  // y = x + h n with x = X_hi + X_lo + X_lo2: the grid-aligned high parts add
  // exactly, X_lo joins by an error-free FastTwoSum, the rest is far below it
  float y_h, y_l;
  if (EXACT_HN) {  // hn_lo = hn_lo2 = 0 in such a table
    fast_two_sum(__fadd_rn(X_hi, e0.x), X_lo, y_h, y_l);
    y_l = __fadd_rn(y_l, X_lo2);
  } else {
    float s_h, s_e;
    two_sum(X_lo, e2.y, s_h, s_e);  // |s_h| <= G <= |X_hi + hn_hi| unless that is 0
    fast_two_sum(__fadd_rn(X_hi, e0.x), s_h, y_h, y_l);
    y_l = __fadd_rn(y_l, __fadd_rn(__fadd_rn(X_lo2, s_e), e2.z));  // e2.z: what hn_lo leaves of h n
  }
  // d = q + y^2: both parts are >= 0, so ordering them by size makes the
  // (error-free) FastTwoSum apply
  const float p_h = __fmul_rn(y_h, y_h);
  const float p_l = __fmaf_rn(y_h, y_h, -p_h);
  float d_h, d_e;
  fast_two_sum(fmaxf(q_hi, p_h), fminf(q_hi, p_h), d_h, d_e);
  const float d_l = __fadd_rn(__fadd_rn(d_e, p_l), __fmaf_rn(2.0f * y_h, y_l, q_lo));
  const float r0 = rcp_approx_f32(d_h);
  // real and imaginary parts: A = (Ar, Ai), B = (Br, Bi)
  df_quot_acc(e0.w, e1.w, e0.y, e1.y, y_h, y_l, d_h, d_l, r0, ar_h, ar_l);
  df_quot_acc(e1.x, e2.x, e0.z, e1.z, y_h, y_l, d_h, d_l, r0, ai_h, ai_l);
}

// acc += terms [0, cnt) of a staged table chunk for PPT values of x, with the
// accumulators renormalised every kRenorm terms and at the end.
template <bool EXACT_HN, int PPT>
__device__ __forceinline__ void df_terms(const float4* st, int cnt, const float (&X_hi)[PPT],
                                         const float (&X_lo)[PPT], const float (&X_lo2)[PPT], float q_hi,
                                         float q_lo, float (&ar_h)[PPT], float (&ar_l)[PPT], float (&ai_h)[PPT],
                                         float (&ai_l)[PPT]) {
  int t = 0;
  for (; t + kRenorm <= cnt; t += kRenorm) {
#pragma unroll 4
    for (int k = 0; k < kRenorm; ++k)
#pragma unroll
      for (int u = 0; u < PPT; ++u)
        df_term<EXACT_HN>(st + 3 * (t + k), X_hi[u], X_lo[u], X_lo2[u], q_hi, q_lo, ar_h[u], ar_l[u], ai_h[u],
                          ai_l[u]);
#pragma unroll
    for (int u = 0; u < PPT; ++u) {
      df_renorm(ar_h[u], ar_l[u]);
      df_renorm(ai_h[u], ai_l[u]);
    }
  }
  for (; t < cnt; ++t)
#pragma unroll
    for (int u = 0; u < PPT; ++u)
      df_term<EXACT_HN>(st + 3 * t, X_hi[u], X_lo[u], X_lo2[u], q_hi, q_lo, ar_h[u], ar_l[u], ai_h[u], ai_l[u]);
#pragma unroll
  for (int u = 0; u < PPT; ++u) {
    df_renorm(ar_h[u], ar_l[u]);
    df_renorm(ai_h[u], ai_l[u]);
  }
}


}  // namespace rexi
