// Batched serving launch: many independent constant-depth instances (own grid
// size, own time step, hence own pole count) advanced together.
//
// The pole sum depends on a wavenumber only through omega(k), so it is
// evaluated once per orbit of omega's symmetries (k -> -k per axis, and
// kx <-> ky on square grids; see OrbitParams).  Work is split into items of
// `threads * orbits_per_thread` orbits of one instance; an item costs
// (orbits x scalar terms).  Items are sorted by cost, largest first, and one
// persistent kernel (a few CTAs per SM) pulls them from an atomic counter, so
// that small and large instances fill the GPU together instead of one small
// launch after another; it writes R+ per orbit, and one combine launch over
// every wavenumber of every instance applies r(tau B).  The forward and
// inverse FFTs run once per distinct grid size over all instances of that
// size (they are packed next to each other).  The whole sequence is captured
// once in a CUDA graph on a stream owned by the batch and replayed.  The
// persistent kernel's CTA size and orbits per thread are chosen by timing the
// candidates (rexi_batch_autotune).  The per-instance mode launches the
// single-instance kernels instance by instance, for comparison.
#include <math.h>
#include <string.h>

#include <algorithm>
#include <map>
#include <vector>

#include "internal.h"
#include "pole_common.cuh"

namespace rexi {
namespace {

struct InstDesc {
  long long spec_off;  // first element of this instance's spectrum (field 0)
  long long orb_off;   // first entry of this instance's per-orbit combine scalars
  int nx, ny, nterms, pad;
  int ax, ay, sym, norb;  // OrbitParams of the instance's grid
  long long half_off;     // real input: first element of the instance's half spectrum (dense per size group)
  int half_ok, pad2;      // 1: even nx, real transforms along x available
  const float4* halfdf_x;  // half angles as double-float pairs
  const float4* halfdf_y;
  double inv_dx, inv_dy, tau, q, R0re, R0im, grid, inv_grid;  // grid: a power of 2 (inv_grid exact)
  float q_hi, q_lo;
  int exact_hn;  // mixed table: every h n on the split grid
  long long table_off;  // first table entry (3 x 16 bytes per term)
  const double2* half_x;
  const double2* half_y;
};

struct WorkItem {
  int inst, orbit_begin;
};

struct SizeGroup {
  int nx, ny;
  std::vector<int> insts;  // packed consecutively
  FftPlan1D fx, fy, fxh;   // fxh: half-length x plan (real input), if half_ok
  bool half_ok = false;
  long long first_off;     // element offset of the group's first state
};

}  // namespace
}  // namespace rexi

struct rexi_batch_s {
  int n = 0, form = REXI_FORM_FP64;
  double Lx = 1, Ly = 1, g = 1, f = 1, H = 1, tol = 1e-10, h = 0.5;
  std::vector<int> nx, ny, M;
  std::vector<double> dt, rho;
  std::vector<long long> offsets;  // per instance, complex128 elements; offsets[n] = total
  std::vector<rexi::SizeGroup> groups;
  std::map<int, std::pair<double2*, double2*>> axis_tables;  // n -> (twiddles, half angles), device
  std::map<int, float4*> axis_twf;                             // n -> double-float twiddles (mixed form)
  std::map<int, float4*> axis_halfdf;                          // n -> half angles as double-float pairs
  // device data owned by the batch
  void* d_tables = nullptr;      // coefficient tables of all instances
  rexi::InstDesc* d_desc = nullptr;
  rexi::WorkItem* d_items = nullptr;
  int n_items = 0;
  int item_orbits = 0;           // orbits per work item the items were built for
  int* d_blk = nullptr;          // first combine block of each instance (n + 1 entries)
  int combine_blocks = 0;
  long long total_orbits = 0;
  std::vector<rexi::InstDesc> h_desc;
  long long total_terms_orbits = 0;
  // launch configuration of the persistent kernel
  int threads = 128, ppt = 1, ctas = 0;
  // graph replay
  cudaStream_t own = nullptr;
  cudaEvent_t ev_in = nullptr, ev_out = nullptr;
  cudaGraphExec_t exec = nullptr;
  const void* g_in = nullptr;
  void* g_out = nullptr;
  void* g_ws = nullptr;
  int g_real = -1, g_threads = 0, g_ppt = 0;
  int64_t launches = 0;
};

namespace rexi {
namespace {

// ---- persistent kernel ------------------------------------------------------

template <int FORM, int PPT>
__global__ void batch_pole_kernel(OrbitScalars* orb, const InstDesc* __restrict__ desc,
                                  const WorkItem* __restrict__ items, int n_items, unsigned* counter,
                                  const void* __restrict__ tables, double g, double f, double H) {
  __shared__ float4 st[kChunk * 3];  // 48 bytes per term, both forms
  __shared__ int s_item;
  __shared__ InstDesc D;
  for (;;) {
    __syncthreads();
    if (threadIdx.x == 0) s_item = (int)atomicAdd(counter, 1u);
    __syncthreads();
    const int it = s_item;
    if (it >= n_items) return;
    if (threadIdx.x == 0) D = desc[items[it].inst];
    __syncthreads();
    SymbolParams sp;
    sp.nx = D.nx;
    sp.ny = D.ny;
    sp.inv_dx = D.inv_dx;
    sp.inv_dy = D.inv_dy;
    sp.g = g;
    sp.f = f;
    sp.H = H;
    sp.half_x = D.half_x;
    sp.half_y = D.half_y;
    OrbitParams op;
    op.ax = D.ax;
    op.ay = D.ay;
    op.sym = D.sym;
    op.norb = D.norb;
    int o[PPT];
    double x[PPT], om[PPT];
#pragma unroll
    for (int u = 0; u < PPT; ++u) {
      o[u] = items[it].orbit_begin + u * blockDim.x + threadIdx.x;
      int a = 0, b = 0;
      if (o[u] < D.norb) orbit_rep(op, o[u], a, b);
      om[u] = symbol_at(sp, a, b).omega;
      x[u] = D.tau * om[u];
    }
    double ar[PPT], ai[PPT];
    float arh[PPT], arl[PPT], aih[PPT], ail[PPT], Xh[PPT], Xl[PPT], Xl2[PPT];
#pragma unroll
    for (int u = 0; u < PPT; ++u) {
      ar[u] = ai[u] = 0.0;
      arh[u] = arl[u] = aih[u] = ail[u] = 0.f;
      const double xg = rint(x[u] * D.inv_grid) * D.grid;
      Xh[u] = (float)xg;
      Xl[u] = (float)(x[u] - xg);
      Xl2[u] = (float)((x[u] - xg) - (double)Xl[u]);
    }
    const float4* tb = reinterpret_cast<const float4*>(tables) + D.table_off * 3;
    for (int t0 = 0; t0 < D.nterms; t0 += kChunk) {
      const int cnt = min(kChunk, D.nterms - t0);
      __syncthreads();
      for (int i = threadIdx.x; i < cnt * 3; i += blockDim.x) st[i] = tb[(size_t)t0 * 3 + i];
      __syncthreads();
      if (FORM == REXI_FORM_FP64) {
        const double2* sd = reinterpret_cast<const double2*>(st);
#pragma unroll 2
        for (int t = 0; t < cnt; ++t)
#pragma unroll
          for (int u = 0; u < PPT; ++u) fp64_term(sd + 3 * t, x[u], D.q, ar[u], ai[u]);
      } else if (D.exact_hn) {
        df_terms<true, PPT>(st, cnt, Xh, Xl, Xl2, D.q_hi, D.q_lo, arh, arl, aih, ail);
      } else {
        df_terms<false, PPT>(st, cnt, Xh, Xl, Xl2, D.q_hi, D.q_lo, arh, arl, aih, ail);
      }
    }
#pragma unroll
    for (int u = 0; u < PPT; ++u) {
      if (o[u] >= D.norb) continue;
      const double2 Rp = FORM == REXI_FORM_FP64
                             ? make_double2(ar[u], ai[u])
                             : make_double2((double)arh[u] + (double)arl[u], (double)aih[u] + (double)ail[u]);
      orb[D.orb_off + o[u]] = orbit_scalars(om[u], make_double2(D.R0re, D.R0im), Rp);
    }
  }
}

// r(tau B) at every wavenumber of every instance from its orbit's scalars.
// Instance i owns combine blocks [blk[i], blk[i + 1]) (enough for its full
// spectrum).  Real input on an even-nx grid: the half spectrum at half_off
// (double-float pairs for the mixed form, df = 1), r(0) through its real part.
__global__ void __launch_bounds__(256) batch_combine_kernel(double2* spec, const OrbitScalars* __restrict__ orb,
                                                            const InstDesc* __restrict__ desc,
                                                            const int* __restrict__ blk, int n, double g, double f,
                                                            double H, int adjoint, int real_input, int df,
                                                            float2 g_df, float2 f_df, float2 H_df) {
  int lo = 0, hi = n - 1;  // last instance with blk[i] <= blockIdx.x
  while (lo < hi) {
    const int mid = (lo + hi + 1) / 2;
    if (blk[mid] <= (int)blockIdx.x) lo = mid;
    else hi = mid - 1;
  }
  const InstDesc& D = desc[lo];
  const int k = ((int)blockIdx.x - blk[lo]) * blockDim.x + threadIdx.x;
  const bool half = real_input && D.half_ok;
  const int row_len = half ? D.nx / 2 + 1 : D.nx;
  const int nk = row_len * D.ny;
  if (k >= nk) return;
  SymbolParams sp;
  sp.nx = D.nx;
  sp.ny = D.ny;
  sp.inv_dx = D.inv_dx;
  sp.inv_dy = D.inv_dy;
  sp.g = g;
  sp.f = f;
  sp.H = H;
  sp.half_x = D.half_x;
  sp.half_y = D.half_y;
  OrbitParams op;
  op.ax = D.ax;
  op.ay = D.ay;
  op.sym = D.sym;
  op.norb = D.norb;
  const int ky = k / row_len, kx = k - ky * row_len;
  OrbitScalars o = orb[D.orb_off + orbit_of(op, D.nx, D.ny, kx, ky)];
  if (!half) {
    combine_scaled(spec + D.spec_off, (size_t)k, (size_t)nk, symbol_entries(sp, kx, ky, adjoint != 0),
                   make_double2(D.R0re, D.R0im), o, adjoint != 0);
  } else if (df) {
    SymbolDF sd;
    sd.g = g_df;
    sd.H = H_df;
    sd.f = f_df;
    sd.inv_dx = df_from_double(D.inv_dx);
    sd.inv_dy = df_from_double(D.inv_dy);
    sd.half_x = D.halfdf_x;
    sd.half_y = D.halfdf_y;
    combine_df_at(reinterpret_cast<float4*>(spec + D.half_off), (size_t)k, (size_t)nk, kx, ky, sd,
                  df_from_double(D.R0re), df_from_double(o.s1), df_from_double(o.s2re), adjoint != 0);
  } else {
    o.s2im = 0.0;
    combine_scaled(spec + D.half_off, (size_t)k, (size_t)nk, symbol_entries(sp, kx, ky, adjoint != 0),
                   make_double2(D.R0re, 0.0), o, adjoint != 0);
  }
}

template <int FORM, int PPT>
cudaError_t launch_persistent(rexi_batch_s* b, OrbitScalars* orb, unsigned* counter, int threads, cudaStream_t s) {
  auto kern = batch_pole_kernel<FORM, PPT>;
  int per_sm = 0;
  cudaError_t e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kern, threads, 0);
  if (e != cudaSuccess) return e;
  int dev = 0, sms = 0;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  const int ctas = std::max(1, std::min(per_sm * sms, b->n_items));
  b->ctas = ctas;
  kern<<<ctas, threads, 0, s>>>(orb, b->d_desc, b->d_items, b->n_items, counter, b->d_tables, b->g, b->f, b->H);
  return cudaGetLastError();
}

cudaError_t launch_pole(rexi_batch_s* b, OrbitScalars* orb, unsigned* counter, cudaStream_t s) {
  if (b->form == REXI_FORM_FP64)
    return b->ppt == 2 ? launch_persistent<REXI_FORM_FP64, 2>(b, orb, counter, b->threads, s)
                       : launch_persistent<REXI_FORM_FP64, 1>(b, orb, counter, b->threads, s);
  return b->ppt == 2 ? launch_persistent<REXI_FORM_MIXED, 2>(b, orb, counter, b->threads, s)
                     : launch_persistent<REXI_FORM_MIXED, 1>(b, orb, counter, b->threads, s);
}

cudaError_t launch_combine(rexi_batch_s* b, double2* spec, const OrbitScalars* orb, int real_input, cudaStream_t s) {
  batch_combine_kernel<<<b->combine_blocks, 256, 0, s>>>(spec, orb, b->d_desc, b->d_blk, b->n, b->g, b->f, b->H, 0,
                                                         real_input, b->form == REXI_FORM_MIXED ? 1 : 0,
                                                         df_split_host(b->g), df_split_host(b->f), df_split_host(b->H));
  return cudaGetLastError();
}

size_t al256(size_t v) { return (v + 255) / 256 * 256; }

// Workspace: [counter (256 B)][packed spectrum][per-orbit R+ of every instance]
size_t batch_spec_bytes(const rexi_batch_s* b) { return al256((size_t)b->offsets[b->n] * sizeof(double2)); }
// The orbit region also serves the per-instance mode, one instance at a
// time: its term slices' partial sums, then its combine scalars.
size_t per_instance_part_bytes(const InstDesc& D) {
  return al256((size_t)orbit_slice_cap(D.norb) * D.norb * sizeof(double2));
}
size_t batch_orb_bytes(const rexi_batch_s* b) {
  size_t m = orbit_scalars_bytes((int)b->total_orbits);
  for (const auto& D : b->h_desc) m = std::max(m, per_instance_part_bytes(D) + orbit_scalars_bytes(D.norb));
  return m;
}
size_t batch_ws_bytes(const rexi_batch_s* b) { return 256 + batch_spec_bytes(b) + al256(batch_orb_bytes(b)); }

// (Re)build the work items for the current item size, largest cost first.
cudaError_t build_items(rexi_batch_s* b) {
  const int item_orbits = b->threads * b->ppt;
  if (item_orbits == b->item_orbits && b->d_items) return cudaSuccess;
  struct Cost {
    long long cost;
    WorkItem w;
  };
  std::vector<Cost> v;
  for (int i = 0; i < b->n; ++i) {
    const int no = b->h_desc[i].norb;
    for (int p = 0; p < no; p += item_orbits) {
      const long long orbits = std::min(item_orbits, no - p);
      v.push_back({orbits * (long long)b->h_desc[i].nterms, {i, p}});
    }
  }
  std::stable_sort(v.begin(), v.end(), [](const Cost& a, const Cost& c) { return a.cost > c.cost; });
  std::vector<WorkItem> items(v.size());
  for (size_t k = 0; k < v.size(); ++k) items[k] = v[k].w;
  if (b->d_items) cudaFree(b->d_items);
  b->d_items = nullptr;
  cudaError_t e = cudaMalloc(&b->d_items, items.size() * sizeof(WorkItem));
  if (e != cudaSuccess) return e;
  e = cudaMemcpy(b->d_items, items.data(), items.size() * sizeof(WorkItem), cudaMemcpyHostToDevice);
  b->n_items = (int)items.size();
  b->item_orbits = item_orbits;
  return e;
}

// FP64 transforms for the FP64 form, double-float ones for the mixed form.
cudaError_t fft_any(const rexi_batch_s* b, const double2* in, double2* out, int nfields, const FftPlan1D& px,
                    const FftPlan1D& py, int sign, double scale, int zero_imag_in, int real_out, cudaStream_t s) {
  return b->form == REXI_FORM_MIXED ? fft2d_df(in, out, nfields, px, py, sign, scale, zero_imag_in, real_out, s)
                                    : fft2d(in, out, nfields, px, py, sign, scale, zero_imag_in, real_out, s);
}

// The whole persistent-mode step on stream s.
cudaError_t enqueue_persistent(rexi_batch_s* b, const double2* in, double2* out, int real_input, char* ws,
                               cudaStream_t s) {
  unsigned* counter = reinterpret_cast<unsigned*>(ws);
  double2* spec = reinterpret_cast<double2*>(ws + 256);
  OrbitScalars* orb = reinterpret_cast<OrbitScalars*>(ws + 256 + batch_spec_bytes(b));
  cudaError_t e = cudaMemsetAsync(counter, 0, sizeof(unsigned), s);
  const int df = b->form == REXI_FORM_MIXED ? 2 : 0;  // real transforms: double-float half spectrum
  for (auto& G : b->groups) {
    if (e != cudaSuccess) return e;
    const int nf = 3 * (int)G.insts.size();
    if (real_input && G.half_ok)
      e = fft2d_r2c(in + G.first_off, spec + G.first_off, nf, G.fx, G.fxh, G.fy, df, s);
    else
      e = fft_any(b, in + G.first_off, spec + G.first_off, nf, G.fx, G.fy, -1, 1.0, real_input, 0, s);
  }
  if (e != cudaSuccess) return e;
  e = launch_pole(b, orb, counter, s);
  if (e == cudaSuccess) e = launch_combine(b, spec, orb, real_input, s);
  for (auto& G : b->groups) {
    if (e != cudaSuccess) return e;
    const int nf = 3 * (int)G.insts.size();
    const double scale = 1.0 / ((double)G.nx * G.ny);
    if (real_input && G.half_ok)
      e = fft2d_c2r(spec + G.first_off, out + G.first_off, nf, G.fx, G.fxh, G.fy, scale, df, s);
    else
      e = fft_any(b, spec + G.first_off, out + G.first_off, nf, G.fx, G.fy, +1, scale, 0, real_input, s);
  }
  return e;
}

void reset_graph(rexi_batch_s* b) {
  if (b->exec) cudaGraphExecDestroy(b->exec);
  b->exec = nullptr;
}

}  // namespace
}  // namespace rexi

using namespace rexi;

extern "C" {

void rexi_batch_destroy(rexi_batch_t b) {
  if (!b) return;
  if (b->own) cudaStreamSynchronize(b->own);
  reset_graph(b);
  if (b->own) cudaStreamDestroy(b->own);
  if (b->ev_in) cudaEventDestroy(b->ev_in);
  if (b->ev_out) cudaEventDestroy(b->ev_out);
  for (auto& kv : b->axis_twf) cudaFree(kv.second);
  for (auto& kv : b->axis_halfdf) cudaFree(kv.second);
  for (auto& kv : b->axis_tables) {
    cudaFree(kv.second.first);
    cudaFree(kv.second.second);
  }
  cudaFree(b->d_tables);
  cudaFree(b->d_desc);
  cudaFree(b->d_items);
  cudaFree(b->d_blk);
  delete b;
}

rexi_status rexi_batch_create(rexi_batch_t* out, int32_t n, const int32_t* nx, const int32_t* ny, const double* dt,
                              double Lx, double Ly, double g, double f, double H, double tol, int32_t form,
                              double h) {
  set_last_error("");
  if (!out || n < 1 || !nx || !ny || !dt) {
    set_last_error("rexi_batch_create: NULL argument or n < 1");
    return REXI_EINVAL;
  }
  *out = nullptr;
  if (!(Lx > 0 && Ly > 0 && g > 0 && H > 0 && isfinite(f)) || !valid_h(h) || !valid_tol(tol) ||
      (form != REXI_FORM_FP64 && form != REXI_FORM_MIXED)) {
    set_last_error("rexi_batch_create: bad physics, h, tol or form (FP64 or MIXED)");
    return REXI_EINVAL;
  }
  rexi_batch_s* b = new rexi_batch_s();
  b->n = n;
  b->form = form;
  b->Lx = Lx; b->Ly = Ly; b->g = g; b->f = f; b->H = H; b->tol = tol; b->h = h;
  auto bail = [&](rexi_status st, const char* msg) {
    set_last_error(msg);
    rexi_batch_destroy(b);
    return st;
  };
  std::map<std::pair<int, int>, int> gidx;
  for (int i = 0; i < n; ++i) {
    FftPlan1D px, py;
    if (!fft_factor(nx[i], &px) || !fft_factor(ny[i], &py) || !(dt[i] >= 0.0) || !isfinite(dt[i]))
      return bail(REXI_EINVAL, "rexi_batch_create: an instance has an unsupported grid or a bad dt");
    b->nx.push_back(nx[i]);
    b->ny.push_back(ny[i]);
    b->dt.push_back(dt[i]);
    auto key = std::make_pair(nx[i], ny[i]);
    if (!gidx.count(key)) {
      gidx[key] = (int)b->groups.size();
      SizeGroup G;
      G.nx = nx[i];
      G.ny = ny[i];
      G.fx = px;
      G.fy = py;
      b->groups.push_back(G);
    }
    b->groups[gidx[key]].insts.push_back(i);
  }
  // axis tables per distinct length
  for (auto& G : b->groups) {
    auto ensure_len = [&](int len) -> bool {
      if (b->axis_tables.count(len)) return true;
      std::vector<double2> tw(len), half(len);
      for (int t = 0; t < len; ++t) {
        const double a = 2.0 * M_PI * t / len, c = M_PI * t / len;
        tw[t] = make_double2(cos(a), -sin(a));
        half[t] = make_double2(cos(c), sin(c));
      }
      double2 *dtw = nullptr, *dhalf = nullptr;
      if (cudaMalloc(&dtw, len * sizeof(double2)) != cudaSuccess ||
          cudaMalloc(&dhalf, len * sizeof(double2)) != cudaSuccess) {
        cudaFree(dtw);
        return false;
      }
      b->axis_tables[len] = {dtw, dhalf};
      cudaMemcpy(dtw, tw.data(), len * sizeof(double2), cudaMemcpyHostToDevice);
      cudaMemcpy(dhalf, half.data(), len * sizeof(double2), cudaMemcpyHostToDevice);
      FftPlan1D fl;
      if (!fft_factor(len, &fl)) return false;
      std::vector<float4> twf(2 * (size_t)len), hdf(len);
      df_twiddles(tw.data(), fl, twf.data());
      split_twiddles(half.data(), len, hdf.data());
      float4 *dtwf = nullptr, *dhdf = nullptr;
      if (cudaMalloc(&dtwf, 2 * (size_t)len * sizeof(float4)) != cudaSuccess) return false;
      b->axis_twf[len] = dtwf;
      if (cudaMalloc(&dhdf, len * sizeof(float4)) != cudaSuccess) return false;
      b->axis_halfdf[len] = dhdf;
      cudaMemcpy(dtwf, twf.data(), 2 * (size_t)len * sizeof(float4), cudaMemcpyHostToDevice);
      cudaMemcpy(dhdf, hdf.data(), len * sizeof(float4), cudaMemcpyHostToDevice);
      return true;
    };
    if (!ensure_len(G.nx) || !ensure_len(G.ny))
      return bail(REXI_ENOMEM, "rexi_batch_create: table allocation failed");
    if (G.nx % 2 == 0 && fft_factor(G.nx / 2, &G.fxh)) {  // real transforms along x
      if (!ensure_len(G.nx / 2)) return bail(REXI_ENOMEM, "rexi_batch_create: table allocation failed");
      G.fxh.tw = b->axis_tables[G.nx / 2].first;
      G.fxh.twf = b->axis_twf[G.nx / 2];
      G.half_ok = true;
    }
    G.fx.tw = b->axis_tables[G.nx].first;
    G.fy.tw = b->axis_tables[G.ny].first;
    G.fx.twf = b->axis_twf[G.nx];
    G.fy.twf = b->axis_twf[G.ny];
  }
  // packed layout, group by group
  b->offsets.assign(n + 1, 0);
  long long off = 0;
  for (auto& G : b->groups) {
    G.first_off = off;
    for (int i : G.insts) {
      b->offsets[i] = off;
      off += 3LL * G.nx * G.ny;
    }
  }
  b->offsets[n] = off;
  // per-instance rho, pole count and coefficient tables
  b->h_desc.resize(n);
  std::vector<float> tab;  // 12 floats = 48 bytes per term (FP64 tables reinterpret the same bytes)
  const double mu = table_mu(), hmu = h * mu, q = hmu * hmu;
  for (int i = 0; i < n; ++i) {
    const int X = b->nx[i], Y = b->ny[i];
    const double dx = Lx / X, dy = Ly / Y;
    const double2* hx = nullptr;
    const double2* hy = nullptr;
    double best = 0.0;
    for (int ky = 0; ky < Y; ++ky) {
      const double sy = sin(M_PI * ky / Y), cy = cos(M_PI * ky / Y);
      for (int kx = 0; kx < X; ++kx) {
        const double sx = sin(M_PI * kx / X), cx = cos(M_PI * kx / X);
        best = std::max(best, g * H * (4 * sx * sx / (dx * dx) + 4 * sy * sy / (dy * dy)) + f * f * cx * cx * cy * cy);
      }
    }
    const double rho = sqrt(best);
    const int M = pole_count(dt[i] * rho, h, tol);
    if (M < 0) return bail(REXI_EINVAL, "rexi_batch_create: pole-count rule rejected an instance");
    b->rho.push_back(rho);
    b->M.push_back(M);
    TermSet ts;
    rexii_terms(M, h, &ts);
    const int N = M + kL, nterms = 2 * N + 1;
    InstDesc& D = b->h_desc[i];
    memset(&D, 0, sizeof(D));
    D.spec_off = b->offsets[i];
    D.nx = X;
    D.ny = Y;
    D.nterms = nterms;
    D.inv_dx = 1.0 / dx;
    D.inv_dy = 1.0 / dy;
    D.tau = dt[i];
    D.q = q;
    D.q_hi = (float)q;
    D.q_lo = (float)(q - (double)D.q_hi);
    D.table_off = (long long)(tab.size() / 12);
    hx = b->axis_tables[X].second;
    hy = b->axis_tables[Y].second;
    D.half_x = hx;
    D.half_y = hy;
    const double span = dt[i] * rho + h * N + 4.0;
    if (form == REXI_FORM_MIXED && span > 4.0e6)
      return bail(REXI_EINVAL, "rexi_batch_create: dt*rho too large for the mixed form");
    int gexp = 0;
    while (ldexp(1.0, 23 - gexp) > span && gexp < 60) ++gexp;
    D.grid = ldexp(1.0, -(gexp - 1));
    D.inv_grid = ldexp(1.0, gexp - 1);
    D.exact_hn = 1;
    double R0r = 0, R0i = 0;
    for (int nn = -N; nn <= N; ++nn) {
      const int k = nn + N;
      const double hn = h * nn, d = q + hn * hn;
      const double Ar = ts.c1re[k] * hmu, Ai = ts.c1im[k] * hmu, Br = ts.c2re[k], Bi = ts.c2im[k];
      R0r += (Ar + Br * hn) / d;
      R0i += (Ai + Bi * hn) / d;
      float e[12];
      if (form == REXI_FORM_FP64) {
        const double dd[6] = {hn, Ar, Ai, Br, Bi, 0.0};
        memcpy(e, dd, sizeof(dd));
      } else {
        auto split = [](double v, float& hi, float& lo) {
          hi = (float)v;
          lo = (float)(v - (double)hi);
        };
        const double hg = rint(hn / D.grid) * D.grid;
        float Arh, Arl, Aih, Ail, Brh, Brl, Bih, Bil;
        split(Ar, Arh, Arl);
        split(Ai, Aih, Ail);
        split(Br, Brh, Brl);
        split(Bi, Bih, Bil);
        const float hl = (float)(hn - hg);
        const float v[12] = {(float)hg, Arh, Aih, Brh, Bih, Arl, Ail, Brl, Bil, hl, (float)((hn - hg) - (double)hl),
                             0.f};
        if (hn != hg) D.exact_hn = 0;
        memcpy(e, v, sizeof(v));
      }
      tab.insert(tab.end(), e, e + 12);
    }
    D.R0re = R0r;
    D.R0im = R0i;
    SymbolParams spi;
    spi.nx = X;
    spi.ny = Y;
    spi.inv_dx = D.inv_dx;
    spi.inv_dy = D.inv_dy;
    const OrbitParams op = orbit_params(spi);
    D.ax = op.ax;
    D.ay = op.ay;
    D.sym = op.sym;
    D.norb = op.norb;
    D.orb_off = b->total_orbits;
    b->total_orbits += op.norb;
    b->total_terms_orbits += (long long)op.norb * nterms;
  }
  // real input: the half spectra of a size group lie densely from the group's
  // first element, field after field (the layout of the real transforms)
  for (auto& G : b->groups) {
    const long long field = (long long)G.ny * (G.nx / 2 + 1);
    for (size_t q = 0; q < G.insts.size(); ++q) {
      InstDesc& D = b->h_desc[G.insts[q]];
      D.half_ok = G.half_ok ? 1 : 0;
      D.half_off = G.first_off + 3 * (long long)q * field;
      D.halfdf_x = b->axis_halfdf[G.nx];
      D.halfdf_y = b->axis_halfdf[G.ny];
    }
  }
  std::vector<int> blk(n + 1, 0);
  for (int i = 0; i < n; ++i) blk[i + 1] = blk[i] + (b->nx[i] * b->ny[i] + 255) / 256;
  b->combine_blocks = blk[n];
  if (cudaMalloc(&b->d_tables, tab.size() * sizeof(float)) != cudaSuccess ||
      cudaMalloc(&b->d_desc, n * sizeof(InstDesc)) != cudaSuccess ||
      cudaMalloc(&b->d_blk, (n + 1) * sizeof(int)) != cudaSuccess)
    return bail(REXI_ENOMEM, "rexi_batch_create: device allocation failed");
  cudaMemcpy(b->d_blk, blk.data(), (n + 1) * sizeof(int), cudaMemcpyHostToDevice);
  cudaMemcpy(b->d_tables, tab.data(), tab.size() * sizeof(float), cudaMemcpyHostToDevice);
  cudaMemcpy(b->d_desc, b->h_desc.data(), n * sizeof(InstDesc), cudaMemcpyHostToDevice);
  if (build_items(b) != cudaSuccess) return bail(REXI_ENOMEM, "rexi_batch_create: work list allocation failed");
  if (cudaStreamCreateWithFlags(&b->own, cudaStreamNonBlocking) != cudaSuccess ||
      cudaEventCreateWithFlags(&b->ev_in, cudaEventDisableTiming) != cudaSuccess ||
      cudaEventCreateWithFlags(&b->ev_out, cudaEventDisableTiming) != cudaSuccess)
    return bail(REXI_ECUDA, "rexi_batch_create: stream or event creation failed");
  *out = b;
  return REXI_OK;
}

rexi_status rexi_batch_layout(rexi_batch_t b, int64_t* offsets, int32_t* M_out, size_t* workspace_bytes) {
  set_last_error("");
  if (!b) return REXI_EINVAL;
  if (offsets)
    for (int i = 0; i <= b->n; ++i) offsets[i] = b->offsets[i];
  if (M_out)
    for (int i = 0; i < b->n; ++i) M_out[i] = b->M[i];
  if (workspace_bytes) *workspace_bytes = batch_ws_bytes(b);
  return REXI_OK;
}

rexi_status rexi_batch_step(rexi_batch_t b, const void* in, void* out, int32_t real_input, void* ws, size_t ws_bytes,
                            int32_t mode, void* stream) {
  set_last_error("");
  if (!b || !in || !out || !ws) {
    set_last_error("rexi_batch_step: NULL argument");
    return REXI_EINVAL;
  }
  if (((uintptr_t)in | (uintptr_t)out) & 15 || (uintptr_t)ws & 255) {
    set_last_error("rexi_batch_step: misaligned buffer");
    return REXI_EINVAL;
  }
  if (ws_bytes < batch_ws_bytes(b)) {
    set_last_error("rexi_batch_step: workspace too small");
    return REXI_ENOMEM;
  }
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  const double2* in2 = static_cast<const double2*>(in);
  double2* out2 = static_cast<double2*>(out);
  char* wsc = static_cast<char*>(ws);
  cudaError_t e = cudaSuccess;
  if (mode == REXI_BATCH_PER_INSTANCE) {
    double2* spec = reinterpret_cast<double2*>(wsc + 256);
    char* orb = wsc + 256 + batch_spec_bytes(b);
    for (int i = 0; i < b->n && e == cudaSuccess; ++i) {
      const InstDesc& D = b->h_desc[i];
      FftPlan1D fx, fy;
      fft_factor(D.nx, &fx);
      fft_factor(D.ny, &fy);
      fx.tw = b->axis_tables[D.nx].first;
      fy.tw = b->axis_tables[D.ny].first;
      fx.twf = b->axis_twf[D.nx];
      fy.twf = b->axis_twf[D.ny];
      double2* sp_i = spec + D.spec_off;
      // real input: the instance's half spectrum in its own slot, as rexi_step lays it out
      const bool half = real_input && D.half_ok;
      const int df = b->form == REXI_FORM_MIXED ? 2 : 0;
      FftPlan1D fxh;
      if (half) {
        fft_factor(D.nx / 2, &fxh);
        fxh.tw = b->axis_tables[D.nx / 2].first;
        fxh.twf = b->axis_twf[D.nx / 2];
        e = fft2d_r2c(in2 + D.spec_off, sp_i, 3, fx, fxh, fy, df, s);
      } else {
        e = fft_any(b, in2 + D.spec_off, sp_i, 3, fx, fy, -1, 1.0, real_input, 0, s);
      }
      SymbolParams sp;
      sp.nx = D.nx; sp.ny = D.ny; sp.inv_dx = D.inv_dx; sp.inv_dy = D.inv_dy;
      sp.g = b->g; sp.f = b->f; sp.H = b->H; sp.half_x = D.half_x; sp.half_y = D.half_y;
      FusedScalars fs;
      fs.tau = D.tau; fs.q = D.q; fs.R0re = D.R0re; fs.R0im = half ? 0.0 : D.R0im; fs.nterms = D.nterms;
      fs.adjoint = 0;
      fs.exact_hn = D.exact_hn;  // the instance's table: whether every h n lies on its split grid
      const float* tab = static_cast<const float*>(b->d_tables) + D.table_off * 12;
      // the single-instance kernels, term slices as rexi_step chooses them
      OrbitParams op;
      op.ax = D.ax; op.ay = D.ay; op.sym = D.sym; op.norb = D.norb;
      const int slices = pole_orbit_slices(b->form, op.norb, D.nterms, orbit_slice_cap(op.norb));
      double2* part = reinterpret_cast<double2*>(orb);
      if (e == cudaSuccess)
        e = b->form == REXI_FORM_FP64
                ? pole_orbits_fp64(part, slices, sp, op, reinterpret_cast<const double*>(tab), fs, s)
                : pole_orbits_mixed(part, slices, sp, op, tab, fs, D.grid, s);
      void* fin = orb + per_instance_part_bytes(D);
      const double scale = 1.0 / ((double)D.nx * D.ny);
      if (e == cudaSuccess) {
        if (half && df)
          e = pole_orbit_combine_df(sp_i, part, slices, fin, sp, D.halfdf_x, D.halfdf_y, op, fs, D.nx / 2 + 1, s);
        else
          e = pole_orbit_combine(sp_i, part, slices, fin, sp, op, fs, half ? D.nx / 2 + 1 : D.nx, s);
      }
      if (e == cudaSuccess)
        e = half ? fft2d_c2r(sp_i, out2 + D.spec_off, 3, fx, fxh, fy, scale, df, s)
                 : fft_any(b, sp_i, out2 + D.spec_off, 3, fx, fy, +1, scale, 0, real_input, s);
      b->launches += 7;
    }
  } else if (mode == REXI_BATCH_PERSISTENT) {
    const bool same = b->exec && b->g_in == in && b->g_out == out && b->g_ws == ws && b->g_real == real_input &&
                      b->g_threads == b->threads && b->g_ppt == b->ppt;
    if (!same) {
      reset_graph(b);
      if ((e = build_items(b)) != cudaSuccess) {
        set_last_error(cudaGetErrorString(e));
        return REXI_ECUDA;
      }
      cudaGraph_t graph = nullptr;
      e = cudaStreamBeginCapture(b->own, cudaStreamCaptureModeThreadLocal);
      if (e == cudaSuccess) {
        cudaError_t e2 = enqueue_persistent(b, in2, out2, real_input, wsc, b->own);
        e = cudaStreamEndCapture(b->own, &graph);
        if (e2 != cudaSuccess) e = e2;
      }
      if (e == cudaSuccess) e = cudaGraphInstantiate(&b->exec, graph, 0);
      if (graph) cudaGraphDestroy(graph);
      if (e != cudaSuccess) {
        set_last_error(cudaGetErrorString(e));
        return REXI_ECUDA;
      }
      b->g_in = in; b->g_out = out; b->g_ws = ws; b->g_real = real_input;
      b->g_threads = b->threads; b->g_ppt = b->ppt;
    }
    // order the graph after the caller's stream and the caller's stream after the graph
    e = cudaEventRecord(b->ev_in, s);
    if (e == cudaSuccess) e = cudaStreamWaitEvent(b->own, b->ev_in, 0);
    if (e == cudaSuccess) e = cudaGraphLaunch(b->exec, b->own);
    if (e == cudaSuccess) e = cudaEventRecord(b->ev_out, b->own);
    if (e == cudaSuccess) e = cudaStreamWaitEvent(s, b->ev_out, 0);
    b->launches += 2 + 4 * (int64_t)b->groups.size();
  } else {
    set_last_error("rexi_batch_step: unknown mode");
    return REXI_EINVAL;
  }
  if (e != cudaSuccess) {
    set_last_error(cudaGetErrorString(e));
    return REXI_ECUDA;
  }
  return REXI_OK;
}

rexi_status rexi_batch_autotune(rexi_batch_t b, const void* in, void* out, int32_t real_input, void* ws,
                                size_t ws_bytes, void* stream, int32_t* threads_out, int32_t* ppt_out,
                                double* best_ms_out) {
  set_last_error("");
  if (!b) return REXI_EINVAL;
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  cudaEvent_t e0, e1;
  cudaEventCreate(&e0);
  cudaEventCreate(&e1);
  const int cand_t[3] = {64, 128, 256};
  const int cand_p[2] = {1, 2};
  double best = 1e300;
  int bt = b->threads, bp = b->ppt;
  rexi_status st = REXI_OK;
  for (int ti : cand_t) {
    for (int pi : cand_p) {
      b->threads = ti;
      b->ppt = pi;
      // first call captures the graph; time the next two replays
      st = rexi_batch_step(b, in, out, real_input, ws, ws_bytes, REXI_BATCH_PERSISTENT, stream);
      if (st != REXI_OK) break;
      cudaEventRecord(e0, s);
      for (int r = 0; r < 2 && st == REXI_OK; ++r)
        st = rexi_batch_step(b, in, out, real_input, ws, ws_bytes, REXI_BATCH_PERSISTENT, stream);
      cudaEventRecord(e1, s);
      cudaEventSynchronize(e1);
      float ms = 0.f;
      cudaEventElapsedTime(&ms, e0, e1);
      if (st != REXI_OK) break;
      if (ms / 2 < best) {
        best = ms / 2;
        bt = ti;
        bp = pi;
      }
    }
    if (st != REXI_OK) break;
  }
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  b->threads = bt;
  b->ppt = bp;
  if (threads_out) *threads_out = bt;
  if (ppt_out) *ppt_out = bp;
  if (best_ms_out) *best_ms_out = best;
  return st;
}

rexi_status rexi_batch_info(rexi_batch_t b, int32_t* threads, int32_t* ppt, int32_t* ctas, int32_t* n_items,
                            int64_t* terms_orbits, int64_t* launches) {
  if (!b) return REXI_EINVAL;
  if (threads) *threads = b->threads;
  if (ppt) *ppt = b->ppt;
  if (ctas) *ctas = b->ctas;
  if (n_items) *n_items = b->n_items;
  if (terms_orbits) *terms_orbits = b->total_terms_orbits;
  if (launches) *launches = b->launches;
  return REXI_OK;
}

}  // extern "C"
