// Periodic 2-D FFT in FP64 for the Fourier (constant-depth) path.
//
// A self-sorting Stockham transform (the radix-R formulation in which stage s
// reads x[j + r n/R] and writes X[(j / Ns) Ns R + j % Ns + r Ns], Ns the
// product of the radices of the earlier stages) run entirely in shared
// memory: one pass over HBM for the rows (x direction) and one for the
// columns (y direction, a CTA owns W adjacent columns so each row segment it
// touches is W * 16 contiguous bytes).  Radix 8, 4 and 2 use register
// butterflies; any other prime factor (3, 5, 7, ... <= 127) uses a direct
// DFT in which each thread computes one output.  Twiddles come from a host
// table w[t] = exp(-2 pi i t / n) built in FP64; the inverse uses conj(w).
#include <algorithm>

#include "internal.h"

namespace rexi {

struct StageList {
  int n;
  int nstages;
  int radix[kMaxStages];
};

__device__ __forceinline__ double2 cmul(double2 a, double2 b) {
  return make_double2(fma(a.x, b.x, -a.y * b.y), fma(a.x, b.y, a.y * b.x));
}
__device__ __forceinline__ double2 cadd(double2 a, double2 b) { return make_double2(a.x + b.x, a.y + b.y); }
__device__ __forceinline__ double2 csub(double2 a, double2 b) { return make_double2(a.x - b.x, a.y - b.y); }
// multiply by SIGN * i
template <int SIGN>
__device__ __forceinline__ double2 mul_si(double2 a) {
  return SIGN < 0 ? make_double2(a.y, -a.x) : make_double2(-a.y, a.x);
}

template <int SIGN>
__device__ __forceinline__ double2 tw_load(const double2* tw, int idx) {
  double2 w = __ldg(tw + idx);
  if (SIGN > 0) w.y = -w.y;
  return w;
}

// 2-, 4- and 8-point DFTs X_k = sum_r v_r e^{SIGN 2 pi i r k / R}, in place.
template <int SIGN>
__device__ __forceinline__ void dft2(double2* v) {
  double2 a = v[0], b = v[1];
  v[0] = cadd(a, b);
  v[1] = csub(a, b);
}
template <int SIGN>
__device__ __forceinline__ void dft4(double2* v) {
  double2 t0 = cadd(v[0], v[2]), t1 = csub(v[0], v[2]);
  double2 t2 = cadd(v[1], v[3]), t3 = mul_si<SIGN>(csub(v[1], v[3]));
  v[0] = cadd(t0, t2);
  v[2] = csub(t0, t2);
  v[1] = cadd(t1, t3);
  v[3] = csub(t1, t3);
}
template <int SIGN>
__device__ __forceinline__ void dft8(double2* v) {
  // X_{2m} = DFT4(v_r + v_{r+4}),  X_{2m+1} = DFT4((v_r - v_{r+4}) W^r),  W = e^{SIGN i pi/4}
  const double h = 0.70710678118654752440;
  double2 a[4], b[4];
#pragma unroll
  for (int r = 0; r < 4; ++r) {
    a[r] = cadd(v[r], v[r + 4]);
    b[r] = csub(v[r], v[r + 4]);
  }
  // b1 *= h (1 + SIGN i), b2 *= SIGN i, b3 *= h (-1 + SIGN i)
  {
    double2 z = b[1];
    b[1] = SIGN < 0 ? make_double2(h * (z.x + z.y), h * (z.y - z.x))
                    : make_double2(h * (z.x - z.y), h * (z.y + z.x));
    b[2] = mul_si<SIGN>(b[2]);
    z = b[3];
    b[3] = SIGN < 0 ? make_double2(h * (z.y - z.x), -h * (z.x + z.y))
                    : make_double2(-h * (z.x + z.y), h * (z.x - z.y));
  }
  dft4<SIGN>(a);
  dft4<SIGN>(b);
#pragma unroll
  for (int m = 0; m < 4; ++m) {
    v[2 * m] = a[m];
    v[2 * m + 1] = b[m];
  }
}

// One radix-R stage with register butterflies (R in {2, 4, 8}).
// Element t of sequence b lives at b * sstride + t * estride.
template <int SIGN, int R>
__device__ __forceinline__ void stage_pow2(const double2* src, double2* dst, int n, int Ns, int nseq,
                                           int sstride, int estride, bool seq_fastest,
                                           const double2* tw) {
  const int nb = n / R;
  const int total = nb * nseq;
  const int twstep = n / (Ns * R);
  for (int idx = threadIdx.x; idx < total; idx += blockDim.x) {
    int b, j;
    if (seq_fastest) {
      b = idx % nseq;
      j = idx / nseq;
    } else {
      b = idx / nb;
      j = idx % nb;
    }
    const double2* s = src + b * sstride;
    double2 v[R];
#pragma unroll
    for (int r = 0; r < R; ++r) v[r] = s[(j + r * nb) * estride];
    const int jm = j % Ns;
    if (jm != 0) {
#pragma unroll
      for (int r = 1; r < R; ++r) v[r] = cmul(v[r], tw_load<SIGN>(tw, r * jm * twstep));
    }
    if (R == 2) dft2<SIGN>(v);
    if (R == 4) dft4<SIGN>(v);
    if (R == 8) dft8<SIGN>(v);
    double2* d = dst + b * sstride;
    const int base = (j - jm) * R + jm;
#pragma unroll
    for (int r = 0; r < R; ++r) d[(base + r * Ns) * estride] = v[r];
  }
}

// One radix-R stage for an arbitrary prime R: each thread produces one output
// X[o] = sum_r x[j + r n/R] w^{r (j % Ns) n/(Ns R) + ((r k) mod R) n/R}.
template <int SIGN>
__device__ __forceinline__ void stage_generic(const double2* src, double2* dst, int n, int R, int Ns,
                                              int nseq, int sstride, int estride, bool seq_fastest,
                                              const double2* tw) {
  const int nb = n / R;
  const int total = n * nseq;
  const int twstep = n / (Ns * R);
  for (int idx = threadIdx.x; idx < total; idx += blockDim.x) {
    int b, o;
    if (seq_fastest) {
      b = idx % nseq;
      o = idx / nseq;
    } else {
      b = idx / n;
      o = idx % n;
    }
    const int k = (o / Ns) % R;
    const int jm = o % Ns;
    const int j = (o / (Ns * R)) * Ns + jm;
    const double2* s = src + b * sstride;
    double2 acc = make_double2(0.0, 0.0);
    int rk = 0;  // (r k) mod R
    for (int r = 0; r < R; ++r) {
      int t = r * jm * twstep + rk * nb;
      if (t >= n) t -= n;
      acc = cadd(acc, cmul(s[(j + r * nb) * estride], tw_load<SIGN>(tw, t)));
      rk += k;
      if (rk >= R) rk -= R;
    }
    dst[b * sstride + o * estride] = acc;
  }
}

// Runs all stages; returns the buffer holding the result.
template <int SIGN>
__device__ double2* run_stages(double2* b0, double2* b1, const StageList& st, int nseq, int sstride,
                               int estride, bool seq_fastest, const double2* tw) {
  double2* src = b0;
  double2* dst = b1;
  int Ns = 1;
  for (int s = 0; s < st.nstages; ++s) {
    const int R = st.radix[s];
    if (R == 8)
      stage_pow2<SIGN, 8>(src, dst, st.n, Ns, nseq, sstride, estride, seq_fastest, tw);
    else if (R == 4)
      stage_pow2<SIGN, 4>(src, dst, st.n, Ns, nseq, sstride, estride, seq_fastest, tw);
    else if (R == 2)
      stage_pow2<SIGN, 2>(src, dst, st.n, Ns, nseq, sstride, estride, seq_fastest, tw);
    else
      stage_generic<SIGN>(src, dst, st.n, R, Ns, nseq, sstride, estride, seq_fastest, tw);
    __syncthreads();
    Ns *= R;
    double2* t = src;
    src = dst;
    dst = t;
  }
  return src;
}

// Rows: `rpc` rows of length n per CTA.  `in` and `out` may alias (each CTA
// reads all of its rows before writing them).
template <int SIGN>
__global__ void __launch_bounds__(256) fft_rows_kernel(const double2* in, double2* out, int nrows,
                                                       int rpc, StageList st, const double2* tw,
                                                       double scale, int zero_imag_in,
                                                       int real_out) {
  extern __shared__ double2 smem[];
  const int n = st.n;
  double2* b0 = smem;
  double2* b1 = smem + (size_t)rpc * n;
  const long long row0 = (long long)blockIdx.x * rpc;
  const int nr = (int)min((long long)rpc, nrows - row0);
  const double2* g_in = in + row0 * n;
  for (int i = threadIdx.x; i < rpc * n; i += blockDim.x) {
    double2 v = make_double2(0.0, 0.0);
    if (i < nr * n) {
      v = g_in[i];
      if (zero_imag_in) v.y = 0.0;
    }
    b0[i] = v;
  }
  __syncthreads();
  double2* res = run_stages<SIGN>(b0, b1, st, rpc, n, 1, false, tw);
  double2* g_out = out + row0 * n;
  for (int i = threadIdx.x; i < nr * n; i += blockDim.x) {
    double2 v = res[i];
    v.x *= scale;
    v.y = real_out ? 0.0 : v.y * scale;
    g_out[i] = v;
  }
}

// Columns: W adjacent columns of one field per CTA (blockIdx.y = field).
template <int SIGN>
__global__ void __launch_bounds__(256) fft_cols_kernel(const double2* in, double2* out, int nx,
                                                       int W, StageList st, const double2* tw,
                                                       double scale, int zero_imag_in,
                                                       int real_out) {
  extern __shared__ double2 smem[];
  const int ny = st.n;
  double2* b0 = smem;
  double2* b1 = smem + (size_t)W * ny;
  const int x0 = blockIdx.x * W;
  const int w = min(W, nx - x0);
  const size_t field_off = (size_t)blockIdx.y * nx * ny;
  const double2* g_in = in + field_off + x0;
  for (int i = threadIdx.x; i < ny * W; i += blockDim.x) {
    const int t = i / W, c = i - t * W;
    double2 v = make_double2(0.0, 0.0);
    if (c < w) {
      v = g_in[(size_t)t * nx + c];
      if (zero_imag_in) v.y = 0.0;
    }
    b0[i] = v;
  }
  __syncthreads();
  double2* res = run_stages<SIGN>(b0, b1, st, W, 1, W, true, tw);
  double2* g_out = out + field_off + x0;
  for (int i = threadIdx.x; i < ny * W; i += blockDim.x) {
    const int t = i / W, c = i - t * W;
    if (c < w) {
      double2 v = res[i];
      v.x *= scale;
      v.y = real_out ? 0.0 : v.y * scale;
      g_out[(size_t)t * nx + c] = v;
    }
  }
}

bool fft_factor(int n, FftPlan1D* p) {
  if (n < 2 || n > 4096) return false;
  p->n = n;
  p->nstages = 0;
  int m = n;
  // powers of two: as many radix-8 stages as possible, then one 4 or 2
  while (m % 8 == 0 && p->nstages < kMaxStages) {
    p->radix[p->nstages++] = 8;
    m /= 8;
  }
  if (m % 4 == 0) {
    p->radix[p->nstages++] = 4;
    m /= 4;
  }
  if (m % 2 == 0) {
    p->radix[p->nstages++] = 2;
    m /= 2;
  }
  for (int q = 3; q <= kMaxRadix && m > 1; q += 2) {
    while (m % q == 0) {
      if (p->nstages >= kMaxStages) return false;
      p->radix[p->nstages++] = q;
      m /= q;
    }
  }
  return m == 1;
}

static StageList to_stages(const FftPlan1D& p) {
  StageList s;
  s.n = p.n;
  s.nstages = p.nstages;
  for (int i = 0; i < kMaxStages; ++i) s.radix[i] = i < p.nstages ? p.radix[i] : 0;
  return s;
}

static int rows_per_cta(int n) {
  int r = 1;
  while (r < 16 && r * n * 2 <= 1024) r *= 2;
  return r;
}
static int cols_per_cta(int n) {
  int w = 16;
  while (w > 1 && 2 * (size_t)w * n * sizeof(double2) > 128 * 1024) w /= 2;
  return w;
}

template <typename K>
static cudaError_t allow_smem(K kernel, size_t bytes) {
  if (bytes <= 48 * 1024) return cudaSuccess;
  return cudaFuncSetAttribute(kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)bytes);
}

template <int SIGN>
static cudaError_t fft2d_impl(const double2* in, double2* out, int nfields, const FftPlan1D& px,
                              const FftPlan1D& py, double scale, int zero_imag_in, int real_out,
                              cudaStream_t s) {
  const int nx = px.n, ny = py.n;
  cudaError_t e;
  {
    const int rpc = rows_per_cta(nx);
    const int nrows = nfields * ny;
    const size_t sm = 2 * (size_t)rpc * nx * sizeof(double2);
    if ((e = allow_smem(fft_rows_kernel<SIGN>, sm)) != cudaSuccess) return e;
    dim3 grid((nrows + rpc - 1) / rpc);
    fft_rows_kernel<SIGN><<<grid, 256, sm, s>>>(in, out, nrows, rpc, to_stages(px), px.tw, 1.0,
                                                zero_imag_in, 0);
    if ((e = cudaGetLastError()) != cudaSuccess) return e;
  }
  {
    const int W = cols_per_cta(ny);
    const size_t sm = 2 * (size_t)W * ny * sizeof(double2);
    if ((e = allow_smem(fft_cols_kernel<SIGN>, sm)) != cudaSuccess) return e;
    dim3 grid((nx + W - 1) / W, nfields);
    fft_cols_kernel<SIGN><<<grid, 256, sm, s>>>(out, out, nx, W, to_stages(py), py.tw, scale, 0,
                                                real_out);
    if ((e = cudaGetLastError()) != cudaSuccess) return e;
  }
  return cudaSuccess;
}

cudaError_t fft2d(const double2* in, double2* out, int nfields, const FftPlan1D& px,
                  const FftPlan1D& py, int sign, double scale, int zero_imag_in, int real_out,
                  cudaStream_t s) {
  if (sign < 0) return fft2d_impl<-1>(in, out, nfields, px, py, scale, zero_imag_in, real_out, s);
  return fft2d_impl<+1>(in, out, nfields, px, py, scale, zero_imag_in, real_out, s);
}

}  // namespace rexi
