// Fourier-path pole kernels: every REXII term for every wavenumber.
//
// For constant depth each Fourier mode k evolves under the 3x3 symbol B(k)
// of the C-grid operator, whose eigenvalues are 0 and +-i omega(k) (its
// characteristic polynomial is z^3 + omega^2 z).  A shifted solve
// (alpha I + tau B)^{-1} therefore reduces to scalar work on those
// eigenvalues, and the sum over all REXII terms of eq. modifiedRexi,
//   R+ = REXII(i x) = sum_n (c1_n h mu + c2_n (x + h n)) / ((h mu)^2 + (x + h n)^2),
// x = tau omega(k), is accumulated in registers.  The conjugate symmetry of
// the coefficients (remark before eq. modifiedRexiMatrixReducedSum) gives
// REXII(-ix) = conj(R+), and with Bt = B / omega
//   r(tau B) = R0 I + Im(R+) Bt + (R0 - Re R+) Bt^2,   R0 = REXII(0),
// which is exact on all three eigenvalues (Bt^3 = -Bt).  No per-term field is
// materialised.  R+ depends on k only through omega(k), so it is summed once
// per orbit of omega's symmetries (see OrbitParams) and a separate pass
// applies r(tau B) at every wavenumber with its own symbol.
//
// Forms:
//  * pole_orbit_fp64 / pole_fused_fp64 -- FP64 registers; 1/d by the
//    rcp.approx seed plus a Newton-Raphson step with its next term in FP64.
//  * pole_orbit_mixed -- the same sum in double-float
//    arithmetic (pairs of FP32 values with Dekker/Knuth error-free
//    transformations: TwoSum, TwoProduct by FMA), FP64 only for the
//    per-orbit setup.  FP32 runs ~58x faster than FP64 on this GPU.
//    (pole_fused_fp64 is the earlier one-pair-per-thread form with the
//    combine fused, kept for the allocation-free step.)
//  * pole_orbit_combine (FP64) / pole_orbit_combine_df (double-float, real
//    input, half spectrum) -- r(tau B) at every wavenumber from per-orbit
//    scalars.
//  * pole_plain_terms / pole_plain_reduce -- the paper's GPU structure
//    (Section 4.1): per REXII term n the two shifted 3x3 solves
//    g1 = (alpha_n I + tau B)^{-1} f, g2 = (alpha_{-n} I - tau B)^{-1} g1,
//    g3 = Gamma_n (C2 g1 + (C1 - C2 alpha_{-n}) g2) written to HBM for a chunk
//    of terms, then a separate reduction pass over the chunk.
#include <algorithm>

#include "dfloat.cuh"
#include "internal.h"
#include "pole_common.cuh"

namespace rexi {


__global__ void __launch_bounds__(128) pole_fused_fp64_kernel(double2* spec, SymbolParams sp,
                                                              const double* __restrict__ table,
                                                              FusedScalars fs, int npairs) {
  __shared__ double2 st[kChunk * 3];
  const int p = blockIdx.x * blockDim.x + threadIdx.x;
  int kx = 0, ky = 0, kx2 = 0, ky2 = 0;
  const bool active = p < npairs && pair_of(p, sp.nx, sp.ny, kx, ky, kx2, ky2);
  Symbol S = symbol_at(sp, active ? kx : 0, active ? ky : 0);
  const double x = fs.tau * S.omega;
  double accr = 0.0, acci = 0.0;
  const double q = fs.q;
  const double2* tb = reinterpret_cast<const double2*>(table);
  for (int t0 = 0; t0 < fs.nterms; t0 += kChunk) {
    const int cnt = min(kChunk, fs.nterms - t0);
    __syncthreads();
    for (int i = threadIdx.x; i < cnt * 3; i += blockDim.x) st[i] = tb[(size_t)t0 * 3 + i];
    __syncthreads();
#pragma unroll 4
    for (int t = 0; t < cnt; ++t) fp64_term(st + 3 * t, x, q, accr, acci);
  }
  if (!active) return;
  const double2 R0 = make_double2(fs.R0re, fs.R0im);
  const double2 Rp = make_double2(accr, acci);
  const size_t fstride = (size_t)sp.nx * sp.ny;
  const bool adj = fs.adjoint != 0;
  combine(spec, (size_t)ky * sp.nx + kx, fstride, S, sp, false, adj, R0, Rp);
  if (kx2 != kx || ky2 != ky)
    combine(spec, (size_t)ky2 * sp.nx + kx2, fstride, symbol_at(sp, kx2, ky2), sp, false, adj, R0, Rp);
}

static int pairs_count(int nx, int ny) { return nx * (ny / 2 + 1); }

cudaError_t pole_fused_fp64(double2* spec, const SymbolParams& sp, const double* table,
                            const FusedScalars& fs, cudaStream_t s) {
  const int np = pairs_count(sp.nx, sp.ny);
  const int tpb = 128;
  pole_fused_fp64_kernel<<<(np + tpb - 1) / tpb, tpb, 0, s>>>(spec, sp, table, fs, np);
  return cudaGetLastError();
}

// ---------------------------------------------------------------------------
// Orbit form: one pole sum per orbit of omega's symmetry group (up to 8
// wavenumbers on a square grid, 4 otherwise, against 2 for the pair form),
// the terms split into `slices` ranges over blockIdx.y so that small grids
// still fill the GPU; each (slice, orbit) writes its partial R+ in FP64 and
// the combine pass sums the slices in a fixed order (deterministic).

OrbitParams orbit_params(const SymbolParams& sp) {
  OrbitParams op;
  op.ax = sp.nx / 2 + 1;
  op.ay = sp.ny / 2 + 1;
  op.sym = (sp.nx == sp.ny && sp.inv_dx == sp.inv_dy) ? 1 : 0;
  op.norb = op.sym ? op.ax * (op.ax + 1) / 2 : op.ax * op.ay;
  return op;
}

int orbit_slice_cap(int norb) {
  // as many slices as 64 MB of partial sums hold, at least 8 and at most 64
  const long long c = (64ll << 20) / (16ll * std::max(norb, 1));
  return (int)std::min<long long>(64, std::max<long long>(8, c));
}

constexpr int kOrbitThreads = 128;
#ifndef REXI_ORBIT_PPT
#define REXI_ORBIT_PPT 2
#endif
constexpr int kOrbitPPT = REXI_ORBIT_PPT;  // orbits per thread in the double-float pole sum

__device__ __forceinline__ void slice_range(const FusedScalars& fs, int slices, int& t_begin, int& t_end) {
  const int per = (fs.nterms + slices - 1) / slices;
  t_begin = min(fs.nterms, (int)blockIdx.y * per);
  t_end = min(fs.nterms, t_begin + per);
}

__global__ void __launch_bounds__(kOrbitThreads) pole_orbit_fp64_kernel(double2* __restrict__ part, SymbolParams sp,
                                                                        OrbitParams op,
                                                                        const double* __restrict__ table,
                                                                        FusedScalars fs, int slices) {
  __shared__ double2 st[kChunk * 3];
  const int o = blockIdx.x * blockDim.x + threadIdx.x;
  int a = 0, b = 0;
  if (o < op.norb) orbit_rep(op, o, a, b);
  const double x = fs.tau * symbol_at(sp, a, b).omega;
  const double q = fs.q;
  double accr = 0.0, acci = 0.0;
  int t_begin, t_end;
  slice_range(fs, slices, t_begin, t_end);
  const double2* tb = reinterpret_cast<const double2*>(table);
  for (int t0 = t_begin; t0 < t_end; t0 += kChunk) {
    const int cnt = min(kChunk, t_end - t0);
    __syncthreads();
    for (int i = threadIdx.x; i < cnt * 3; i += blockDim.x) st[i] = tb[(size_t)t0 * 3 + i];
    __syncthreads();
#pragma unroll 4
    for (int t = 0; t < cnt; ++t) fp64_term(st + 3 * t, x, q, accr, acci);
  }
  if (o < op.norb) part[(size_t)blockIdx.y * op.norb + o] = make_double2(accr, acci);
}

// PPT orbits per thread share each staged term's shared-memory loads.
template <int PPT, bool EXACT_HN>
__global__ void __launch_bounds__(kOrbitThreads) pole_orbit_mixed_kernel(double2* __restrict__ part, SymbolParams sp,
                                                                         OrbitParams op,
                                                                         const float4* __restrict__ table,
                                                                         FusedScalars fs, double grid,
                                                                         double inv_grid, float q_hi, float q_lo,
                                                                         int slices) {
  __shared__ float4 st[kChunk * 3];
  float X_hi[PPT], X_lo[PPT], X_lo2[PPT], ar_h[PPT], ar_l[PPT], ai_h[PPT], ai_l[PPT];
  int o[PPT];
#pragma unroll
  for (int u = 0; u < PPT; ++u) {
    o[u] = (blockIdx.x * PPT + u) * blockDim.x + threadIdx.x;
    int a = 0, b = 0;
    if (o[u] < op.norb) orbit_rep(op, o[u], a, b);
    const double x = fs.tau * symbol_at(sp, a, b).omega;
    const double xg = rint(x * inv_grid) * grid;  // grid a power of 2: x * (1/grid) is exact
    X_hi[u] = (float)xg;
    X_lo[u] = (float)(x - xg);
    X_lo2[u] = (float)((x - xg) - (double)X_lo[u]);
    ar_h[u] = ar_l[u] = ai_h[u] = ai_l[u] = 0.f;
  }
  int t_begin, t_end;
  slice_range(fs, slices, t_begin, t_end);
  for (int t0 = t_begin; t0 < t_end; t0 += kChunk) {
    const int cnt = min(kChunk, t_end - t0);
    __syncthreads();
    for (int i = threadIdx.x; i < cnt * 3; i += blockDim.x) st[i] = table[(size_t)t0 * 3 + i];
    __syncthreads();
    df_terms<EXACT_HN, PPT>(st, cnt, X_hi, X_lo, X_lo2, q_hi, q_lo, ar_h, ar_l, ai_h, ai_l);
  }
#pragma unroll
  for (int u = 0; u < PPT; ++u)
    if (o[u] < op.norb)
      part[(size_t)blockIdx.y * op.norb + o[u]] =
          make_double2((double)ar_h[u] + (double)ar_l[u], (double)ai_h[u] + (double)ai_l[u]);
}

// Per orbit: R+ = sum of the slices' partial sums (fixed order), then the
// combine scalars at the representative's omega (FP64, or double-float pairs
// of the real s1 and s2 for the double-float combine, where R0 is real).
struct OrbitScalarsDF {
  float2 s1, s2;
};

__device__ __forceinline__ float2 df_split(double v) {
  const float h = (float)v;
  return make_float2(h, (float)(v - (double)h));
}

template <bool DF>
__global__ void __launch_bounds__(256) pole_orbit_finalize_kernel(const double2* __restrict__ part, int slices,
                                                                  SymbolParams sp, OrbitParams op, double2 R0,
                                                                  void* __restrict__ fin) {
  const int o = blockIdx.x * blockDim.x + threadIdx.x;
  if (o >= op.norb) return;
  double2 Rp = part[o];
  for (int s = 1; s < slices; ++s) {
    const double2 v = part[(size_t)s * op.norb + o];
    Rp.x += v.x;
    Rp.y += v.y;
  }
  int a, b;
  orbit_rep(op, o, a, b);
  const OrbitScalars sc = orbit_scalars(symbol_at(sp, a, b).omega, R0, Rp);
  if (DF) {
    OrbitScalarsDF d;
    d.s1 = df_split(sc.s1);
    d.s2 = df_split(sc.s2re);
    static_cast<OrbitScalarsDF*>(fin)[o] = d;
  } else {
    static_cast<OrbitScalars*>(fin)[o] = sc;
  }
}

__global__ void __launch_bounds__(256) pole_orbit_combine_kernel(double2* spec,
                                                                 const OrbitScalars* __restrict__ fin,
                                                                 SymbolParams sp, OrbitParams op, double2 R0,
                                                                 int adjoint, int row_len) {
  const size_t nk = (size_t)row_len * sp.ny;
  const size_t k = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (k >= nk) return;
  const int ky = (int)(k / row_len), kx = (int)(k - (size_t)ky * row_len);
  const OrbitScalars o = fin[orbit_of(op, sp.nx, sp.ny, kx, ky)];
  combine_scaled(spec, k, nk, symbol_entries(sp, kx, ky, adjoint != 0), R0, o, adjoint != 0);
}

// Double-float combine on a double-float half spectrum (see combine_df_at).
__global__ void __launch_bounds__(256) pole_orbit_combine_df_kernel(float4* spec,
                                                                    const OrbitScalarsDF* __restrict__ fin,
                                                                    SymbolDF sd, int nx, int ny, OrbitParams op,
                                                                    float2 c0, int adjoint, int row_len) {
  const size_t nk = (size_t)row_len * ny;
  const size_t k = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (k >= nk) return;
  const int ky = (int)(k / row_len), kx = (int)(k - (size_t)ky * row_len);
  const OrbitScalarsDF o = fin[orbit_of(op, nx, ny, kx, ky)];
  combine_df_at(spec, k, nk, kx, ky, sd, c0, o.s1, o.s2, adjoint != 0);
}

namespace {
struct OrbitOccupancy {
  int sms = 0, fp64_blocks = 0, mixed_blocks = 0;
};
OrbitOccupancy orbit_occupancy() {
  static OrbitOccupancy occ;  // per process: the library serves one device model
  if (occ.sms == 0) {
    int dev = 0, sms = 0, b64 = 0, bmx = 0;
    if (cudaGetDevice(&dev) != cudaSuccess ||
        cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess ||
        cudaOccupancyMaxActiveBlocksPerMultiprocessor(&b64, pole_orbit_fp64_kernel, kOrbitThreads, 0) != cudaSuccess ||
        cudaOccupancyMaxActiveBlocksPerMultiprocessor(&bmx, pole_orbit_mixed_kernel<kOrbitPPT, true>, kOrbitThreads, 0) !=
            cudaSuccess) {
      cudaGetLastError();
      return OrbitOccupancy{152, 8, 8};
    }
    occ.sms = sms;
    occ.fp64_blocks = std::max(b64, 1);
    occ.mixed_blocks = std::max(bmx, 1);
  }
  return occ;
}
}  // namespace

int pole_orbit_slices(int form, int norb, int nterms, int cap) {
  if (nterms <= 1) return 1;
  const OrbitOccupancy occ = orbit_occupancy();
  const long long resident = (long long)occ.sms * (form == REXI_FORM_MIXED ? occ.mixed_blocks : occ.fp64_blocks);
  const int per_block = kOrbitThreads * (form == REXI_FORM_MIXED ? kOrbitPPT : 1);
  const long long bx = (norb + per_block - 1) / per_block;
  // per block: its terms plus a fixed cost (symbol, FP64 setup, staging, the
  // write) of about 48 terms; blocks run in waves of `resident`
  double best = 0.0;
  int best_s = 1;
  for (int s = 1; s <= std::min(cap, nterms); ++s) {
    const long long waves = (bx * s + resident - 1) / resident;
    const double t = (double)waves * ((double)((nterms + s - 1) / s) + 48.0);
    if (s == 1 || t < best * 0.98) {
      best = t;
      best_s = s;
    }
  }
  return best_s;
}

cudaError_t pole_orbits_fp64(double2* part, int slices, const SymbolParams& sp, const OrbitParams& op,
                             const double* table, const FusedScalars& fs, cudaStream_t s) {
  dim3 grid((unsigned)((op.norb + kOrbitThreads - 1) / kOrbitThreads), (unsigned)slices);
  pole_orbit_fp64_kernel<<<grid, kOrbitThreads, 0, s>>>(part, sp, op, table, fs, slices);
  return cudaGetLastError();
}

cudaError_t pole_orbits_mixed(double2* part, int slices, const SymbolParams& sp, const OrbitParams& op,
                              const float* table, const FusedScalars& fs, double grid_step, cudaStream_t s) {
  const float q_hi = (float)fs.q;
  const float q_lo = (float)(fs.q - (double)q_hi);
  const double inv_step = 1.0 / grid_step;  // exact: the split grid is a power of 2
  const int per_block = kOrbitThreads * kOrbitPPT;
  dim3 grid((unsigned)((op.norb + per_block - 1) / per_block), (unsigned)slices);
  if (fs.exact_hn)
    pole_orbit_mixed_kernel<kOrbitPPT, true><<<grid, kOrbitThreads, 0, s>>>(
        part, sp, op, reinterpret_cast<const float4*>(table), fs, grid_step, inv_step, q_hi, q_lo, slices);
  else
    pole_orbit_mixed_kernel<kOrbitPPT, false><<<grid, kOrbitThreads, 0, s>>>(
        part, sp, op, reinterpret_cast<const float4*>(table), fs, grid_step, inv_step, q_hi, q_lo, slices);
  return cudaGetLastError();
}

cudaError_t pole_orbit_combine(double2* spec, const double2* part, int slices, void* fin, const SymbolParams& sp,
                               const OrbitParams& op, const FusedScalars& fs, int row_len, cudaStream_t s) {
  const double2 R0 = make_double2(fs.R0re, fs.R0im);
  OrbitScalars* F = static_cast<OrbitScalars*>(fin);
  pole_orbit_finalize_kernel<false><<<(unsigned)((op.norb + 255) / 256), 256, 0, s>>>(part, slices, sp, op, R0, F);
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return e;
  const size_t nk = (size_t)row_len * sp.ny;
  pole_orbit_combine_kernel<<<(unsigned)((nk + 255) / 256), 256, 0, s>>>(spec, F, sp, op, R0, fs.adjoint, row_len);
  return cudaGetLastError();
}

// Complex input, mixed form: the FP64 per-orbit scalars applied in
// double-float arithmetic on the FP64 full spectrum (see combine_dfc_at).
__global__ void __launch_bounds__(256) pole_orbit_combine_dfc_kernel(double2* spec,
                                                                     const OrbitScalars* __restrict__ fin,
                                                                     SymbolDF sd, int nx, int ny, OrbitParams op,
                                                                     float4 c0, int adjoint) {
  const size_t nk = (size_t)nx * ny;
  const size_t k = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (k >= nk) return;
  const int ky = (int)(k / nx), kx = (int)(k - (size_t)ky * nx);
  const OrbitScalars o = fin[orbit_of(op, nx, ny, kx, ky)];
  float4 s2 = c_of(df_from_double(o.s2re), df_from_double(o.s2im));
  if (adjoint) s2 = cconj(s2);
  combine_dfc_at(spec, k, nk, kx, ky, sd, c0, df_from_double(o.s1), s2, adjoint != 0);
}

cudaError_t pole_orbit_combine_dfc(double2* spec, const double2* part, int slices, void* fin, const SymbolParams& sp,
                                   const float4* half_x_df, const float4* half_y_df, const OrbitParams& op,
                                   const FusedScalars& fs, cudaStream_t s) {
  if (sp.spectral) return cudaErrorInvalidValue;  // the C grid only
  const double2 R0 = make_double2(fs.R0re, fs.R0im);
  OrbitScalars* F = static_cast<OrbitScalars*>(fin);
  pole_orbit_finalize_kernel<false><<<(unsigned)((op.norb + 255) / 256), 256, 0, s>>>(part, slices, sp, op, R0, F);
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return e;
  SymbolDF sd;
  sd.g = df_split_host(sp.g);
  sd.H = df_split_host(sp.H);
  sd.f = df_split_host(sp.f);
  sd.inv_dx = df_split_host(sp.inv_dx);
  sd.inv_dy = df_split_host(sp.inv_dy);
  sd.half_x = half_x_df;
  sd.half_y = half_y_df;
  const float2 c0r = df_split_host(fs.R0re), c0i = df_split_host(fs.adjoint ? -fs.R0im : fs.R0im);
  const float4 c0 = make_float4(c0r.x, c0r.y, c0i.x, c0i.y);
  const size_t nk = (size_t)sp.nx * sp.ny;
  pole_orbit_combine_dfc_kernel<<<(unsigned)((nk + 255) / 256), 256, 0, s>>>(spec, F, sd, sp.nx, sp.ny, op, c0,
                                                                             fs.adjoint);
  return cudaGetLastError();
}

// Scalar operator: every field at wavenumber k is multiplied by phase R(k).
__global__ void __launch_bounds__(256) pole_orbit_combine_scalar_kernel(double2* spec,
                                                                        const double2* __restrict__ part,
                                                                        int slices, int nx, int ny, OrbitParams op,
                                                                        double2 phase, int adjoint) {
  const size_t nk = (size_t)nx * ny;
  const size_t k = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (k >= nk) return;
  const int ky = (int)(k / nx), kx = (int)(k - (size_t)ky * nx);
  const int o = orbit_of(op, nx, ny, kx, ky);
  double2 R = part[o];
  for (int sl = 1; sl < slices; ++sl) {
    const double2 v = part[(size_t)sl * op.norb + o];
    R.x += v.x;
    R.y += v.y;
  }
  double2 m = cm(phase, R);
  if (adjoint) m = cj(m);
#pragma unroll
  for (int c = 0; c < 3; ++c) spec[k + c * nk] = cm(m, spec[k + c * nk]);
}

cudaError_t pole_orbit_combine_scalar(double2* spec, const double2* part, int slices, const SymbolParams& sp,
                                      const OrbitParams& op, double2 phase, int adjoint, cudaStream_t s) {
  if (sp.spectral != 2) return cudaErrorInvalidValue;
  const size_t nk = (size_t)sp.nx * sp.ny;
  pole_orbit_combine_scalar_kernel<<<(unsigned)((nk + 255) / 256), 256, 0, s>>>(spec, part, slices, sp.nx, sp.ny,
                                                                                op, phase, adjoint);
  return cudaGetLastError();
}

cudaError_t pole_orbit_combine_df(void* spec_df, const double2* part, int slices, void* fin, const SymbolParams& sp,
                                  const float4* half_x_df, const float4* half_y_df, const OrbitParams& op,
                                  const FusedScalars& fs, int row_len, cudaStream_t s) {
  if (fs.R0im != 0.0 || sp.spectral) return cudaErrorInvalidValue;  // real c0, s2 and the C-grid only
  const double2 R0 = make_double2(fs.R0re, 0.0);
  pole_orbit_finalize_kernel<true><<<(unsigned)((op.norb + 255) / 256), 256, 0, s>>>(part, slices, sp, op, R0, fin);
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return e;
  SymbolDF sd;
  sd.g = df_split_host(sp.g);
  sd.H = df_split_host(sp.H);
  sd.f = df_split_host(sp.f);
  sd.inv_dx = df_split_host(sp.inv_dx);
  sd.inv_dy = df_split_host(sp.inv_dy);
  sd.half_x = half_x_df;
  sd.half_y = half_y_df;
  const size_t nk = (size_t)row_len * sp.ny;
  pole_orbit_combine_df_kernel<<<(unsigned)((nk + 255) / 256), 256, 0, s>>>(
      static_cast<float4*>(spec_df), static_cast<const OrbitScalarsDF*>(fin), sd, sp.nx, sp.ny, op, df_split_host(fs.R0re),
      fs.adjoint, row_len);
  return cudaGetLastError();
}

size_t orbit_scalars_bytes(int norb) { return (size_t)norb * sizeof(OrbitScalars); }

// ---------------------------------------------------------------------------
// Plain form (paper-style): materialise g3 per (term, k), then reduce.
// Table per term (4 double2): alpha_n, alpha_{-n}, Gamma C2, Gamma (C1 - C2 alpha_{-n}).
// (alpha I + s tau B)^{-1} v = v/alpha - s tau B v / D + tau^2 B^2 v / (alpha D),
// D = alpha^2 + tau^2 omega^2, s = +1 or -1, because B^3 = -omega^2 B.

__device__ __forceinline__ double2 cdiv(double2 a, double2 b) {
  const double den = b.x * b.x + b.y * b.y;
  return make_double2((a.x * b.x + a.y * b.y) / den, (a.y * b.x - a.x * b.y) / den);
}

__device__ __forceinline__ void shifted_solve(const Symbol& S, const SymbolParams& sp, bool adjoint,
                                              double2 alpha, double sgn, double tau, const double2 v[3],
                                              double2 out[3]) {
  double2 b1[3], b2[3];
  apply_B(S, sp, false, adjoint, v, b1);
  apply_B(S, sp, false, adjoint, b1, b2);
  const double tw2 = tau * tau * S.omega * S.omega;
  const double2 D = make_double2(alpha.x * alpha.x - alpha.y * alpha.y + tw2, 2.0 * alpha.x * alpha.y);
  const double2 one = make_double2(1.0, 0.0);
  const double2 ia = cdiv(one, alpha);
  const double2 iD = cdiv(one, D);
  const double2 k1 = cr(-sgn * tau, iD);
  const double2 k2 = cr(tau * tau, cm(ia, iD));
#pragma unroll
  for (int c = 0; c < 3; ++c) out[c] = ca(ca(cm(ia, v[c]), cm(k1, b1[c])), cm(k2, b2[c]));
}

__global__ void __launch_bounds__(256) pole_plain_terms_kernel(const double2* __restrict__ spec,
                                                               double2* __restrict__ chunk,
                                                               SymbolParams sp,
                                                               const double2* __restrict__ table,
                                                               PlainScalars ps) {
  const size_t nk = (size_t)sp.nx * sp.ny;
  const size_t k = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
  const int t = blockIdx.y;
  if (k >= nk || t >= ps.nterms) return;
  const int ky = (int)(k / sp.nx), kx = (int)(k - (size_t)ky * sp.nx);
  Symbol S = symbol_at(sp, kx, ky);
  const bool adj = ps.adjoint != 0;
  double2 alpha_n = table[4 * t], alpha_mn = table[4 * t + 1];
  double2 gC2 = table[4 * t + 2], gK = table[4 * t + 3];
  if (adj) {  // (r(tau B))^H: conjugated shifts and coefficients with B^H
    alpha_n = cj(alpha_n); alpha_mn = cj(alpha_mn); gC2 = cj(gC2); gK = cj(gK);
  }
  double2 f[3], g1[3], g2[3];
#pragma unroll
  for (int c = 0; c < 3; ++c) f[c] = spec[k + c * nk];
  shifted_solve(S, sp, adj, alpha_n, +1.0, ps.tau, f, g1);
  shifted_solve(S, sp, adj, alpha_mn, -1.0, ps.tau, g1, g2);
  double2* out = chunk + (size_t)t * 3 * nk;
#pragma unroll
  for (int c = 0; c < 3; ++c) out[k + c * nk] = ca(cm(gC2, g1[c]), cm(gK, g2[c]));
}

__global__ void __launch_bounds__(256) pole_plain_reduce_kernel(const double2* __restrict__ chunk,
                                                                double2* __restrict__ acc,
                                                                long long nk3, int nterms, int first) {
  const long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= nk3) return;
  double2 s = first ? make_double2(0.0, 0.0) : acc[i];
  for (int t = 0; t < nterms; ++t) {
    const double2 v = chunk[(size_t)t * nk3 + i];
    s.x += v.x;
    s.y += v.y;
  }
  acc[i] = s;
}

cudaError_t pole_plain_terms(const double2* spec, double2* chunk, const SymbolParams& sp,
                             const double2* table, const PlainScalars& ps, cudaStream_t s) {
  const size_t nk = (size_t)sp.nx * sp.ny;
  dim3 grid((unsigned)((nk + 255) / 256), ps.nterms);
  pole_plain_terms_kernel<<<grid, 256, 0, s>>>(spec, chunk, sp, table, ps);
  return cudaGetLastError();
}

cudaError_t pole_plain_reduce(const double2* chunk, double2* acc, long long nk3, int nterms, int first,
                              cudaStream_t s) {
  pole_plain_reduce_kernel<<<(unsigned)((nk3 + 255) / 256), 256, 0, s>>>(chunk, acc, nk3, nterms, first);
  return cudaGetLastError();
}

}  // namespace rexi
