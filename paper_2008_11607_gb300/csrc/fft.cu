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
//
// The stages are templates over the complex value type: double2 (FP64) or
// float4 = (re_hi, re_lo, im_hi, im_lo), a double-float complex number whose
// arithmetic runs on the FP32 pipes with error-free transformations (Knuth's
// TwoSum, Dekker's FastTwoSum, the FMA TwoProduct; about 48 significant
// bits), for the mixed form: GB300 issues FP32 operations 58x faster than
// FP64 ones.  The double-float transform reads and writes FP64 in HBM and
// keeps the 16-byte double-float values between its row and column passes.
#include <algorithm>
#include <type_traits>

#include "dfloat.cuh"
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
__device__ __forceinline__ float4 mul_si(float4 a) {
  return SIGN < 0 ? make_float4(a.z, a.w, -a.x, -a.y) : make_float4(-a.z, -a.w, a.x, a.y);
}
// (p + q) * h and (p - q) * h for the 8-point butterfly, h = 1/sqrt(2)
constexpr double kHalfSqrt2 = 0.70710678118654752440;
__device__ __forceinline__ double hmul_sum(double p, double q, int sgn) { return kHalfSqrt2 * (p + sgn * q); }
__device__ __forceinline__ float2 hmul_sum(float2 p, float2 q, int sgn) {
  constexpr float hh = (float)kHalfSqrt2;
  constexpr float hl = (float)(kHalfSqrt2 - (double)hh);
  const float2 t = f_add(p.x, p.y, sgn * q.x, sgn * q.y);
  const float2 m = f_mul(t.x, t.y, hh, hl);
  return f_fast(m.x, m.y);
}
__device__ __forceinline__ double re_of(double2 v) { return v.x; }
__device__ __forceinline__ double im_of(double2 v) { return v.y; }
__device__ __forceinline__ float2 re_of(float4 v) { return make_float2(v.x, v.y); }
__device__ __forceinline__ float2 im_of(float4 v) { return make_float2(v.z, v.w); }
__device__ __forceinline__ double2 cpack(double re, double im) { return make_double2(re, im); }
__device__ __forceinline__ float4 cpack(float2 re, float2 im) { return make_float4(re.x, re.y, im.x, im.y); }
__device__ __forceinline__ double neg(double v) { return -v; }
__device__ __forceinline__ float2 neg(float2 v) { return make_float2(-v.x, -v.y); }

template <int SIGN>
__device__ __forceinline__ double2 tw_load(const double2* tw, int idx) {
  double2 w = __ldg(tw + idx);
  if (SIGN > 0) w.y = -w.y;
  return w;
}
template <int SIGN>
__device__ __forceinline__ float4 tw_load(const float4* tw, int idx) {
  float4 w = __ldg(tw + idx);
  if (SIGN > 0) {
    w.z = -w.z;
    w.w = -w.w;
  }
  return w;
}
template <typename T>
__device__ __forceinline__ T czero() {
  return T{};
}

// 2-, 4- and 8-point DFTs X_k = sum_r v_r e^{SIGN 2 pi i r k / R}, in place.
template <int SIGN, typename T>
__device__ __forceinline__ void dft2(T* v) {
  T a = v[0], b = v[1];
  v[0] = cadd(a, b);
  v[1] = csub(a, b);
}
template <int SIGN, typename T>
__device__ __forceinline__ void dft4(T* v) {
  T t0 = cadd(v[0], v[2]), t1 = csub(v[0], v[2]);
  T t2 = cadd(v[1], v[3]), t3 = mul_si<SIGN>(csub(v[1], v[3]));
  v[0] = cadd(t0, t2);
  v[2] = csub(t0, t2);
  v[1] = cadd(t1, t3);
  v[3] = csub(t1, t3);
}
template <int SIGN, typename T>
__device__ __forceinline__ void dft8(T* v) {
  // X_{2m} = DFT4(v_r + v_{r+4}),  X_{2m+1} = DFT4((v_r - v_{r+4}) W^r),  W = e^{SIGN i pi/4}
  T a[4], b[4];
#pragma unroll
  for (int r = 0; r < 4; ++r) {
    a[r] = cadd(v[r], v[r + 4]);
    b[r] = csub(v[r], v[r + 4]);
  }
  // b1 *= h (1 + SIGN i), b2 *= SIGN i, b3 *= h (-1 + SIGN i)
  {
    T z = b[1];
    b[1] = SIGN < 0 ? cpack(hmul_sum(re_of(z), im_of(z), 1), hmul_sum(im_of(z), re_of(z), -1))
                    : cpack(hmul_sum(re_of(z), im_of(z), -1), hmul_sum(im_of(z), re_of(z), 1));
    b[2] = mul_si<SIGN>(b[2]);
    z = b[3];
    b[3] = SIGN < 0 ? cpack(hmul_sum(im_of(z), re_of(z), -1), neg(hmul_sum(re_of(z), im_of(z), 1)))
                    : cpack(neg(hmul_sum(re_of(z), im_of(z), 1)), hmul_sum(re_of(z), im_of(z), -1));
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
// Element t of sequence b lives at b * sstride + t * estride.  `tws`
// (nullable): this stage's twiddles grouped by butterfly, tws[jm (R - 1) +
// r - 1] = w^{r jm n / (Ns R)}, so that a butterfly's R - 1 twiddles are
// adjacent (one or two cache lines instead of R - 1); else the full table tw.
template <int SIGN, int R, typename T>
__device__ __forceinline__ void stage_pow2(const T* src, T* dst, int n, int Ns, int nseq, int sstride, int estride,
                                           bool seq_fastest, const T* tw, const T* tws) {
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
    const T* s = src + b * sstride;
    T v[R];
#pragma unroll
    for (int r = 0; r < R; ++r) v[r] = s[(j + r * nb) * estride];
    const int jm = j % Ns;
    if (jm != 0) {
      if (tws) {
#pragma unroll
        for (int r = 1; r < R; ++r) v[r] = cmul(v[r], tw_load<SIGN>(tws, jm * (R - 1) + r - 1));
      } else {
#pragma unroll
        for (int r = 1; r < R; ++r) v[r] = cmul(v[r], tw_load<SIGN>(tw, r * jm * twstep));
      }
    }
    if (R == 2) dft2<SIGN>(v);
    if (R == 4) dft4<SIGN>(v);
    if (R == 8) dft8<SIGN>(v);
    T* d = dst + b * sstride;
    const int base = (j - jm) * R + jm;
#pragma unroll
    for (int r = 0; r < R; ++r) d[(base + r * Ns) * estride] = v[r];
  }
}

// One radix-R stage for an arbitrary prime R: each thread produces one output
// X[o] = sum_r x[j + r n/R] w^{r (j % Ns) n/(Ns R) + ((r k) mod R) n/R}.
template <int SIGN, typename T>
__device__ __forceinline__ void stage_generic(const T* src, T* dst, int n, int R, int Ns, int nseq, int sstride,
                                              int estride, bool seq_fastest, const T* tw) {
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
    const T* s = src + b * sstride;
    T acc = czero<T>();
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

// Runs all stages; returns the buffer holding the result.  Double-float
// tables carry the per-stage grouping after the n entries of w (df_twiddles).
template <int SIGN, typename T>
__device__ T* run_stages(T* b0, T* b1, const StageList& st, int nseq, int sstride, int estride, bool seq_fastest,
                         const T* tw) {
  constexpr bool STAGED = std::is_same<T, float4>::value;
  T* src = b0;
  T* dst = b1;
  int Ns = 1, off = st.n;
  for (int s = 0; s < st.nstages; ++s) {
    const int R = st.radix[s];
    const T* tws = STAGED ? tw + off : nullptr;
    if (R == 8)
      stage_pow2<SIGN, 8>(src, dst, st.n, Ns, nseq, sstride, estride, seq_fastest, tw, tws);
    else if (R == 4)
      stage_pow2<SIGN, 4>(src, dst, st.n, Ns, nseq, sstride, estride, seq_fastest, tw, tws);
    else if (R == 2)
      stage_pow2<SIGN, 2>(src, dst, st.n, Ns, nseq, sstride, estride, seq_fastest, tw, tws);
    else
      stage_generic<SIGN>(src, dst, st.n, R, Ns, nseq, sstride, estride, seq_fastest, tw);
    __syncthreads();
    off += Ns * (R - 1);
    Ns *= R;
    T* t = src;
    src = dst;
    dst = t;
  }
  return src;
}

// Conversions at the HBM boundary of a pass: FP64 in and out; double-float
// values between the passes of the double-float transform.
__device__ __forceinline__ void cvt(double2 v, int zero_imag, double2* o) {
  if (zero_imag) v.y = 0.0;
  *o = v;
}
__device__ __forceinline__ void cvt(double2 v, int zero_imag, float4* o) {
  const float2 re = df_from_double(v.x);
  const float2 im = zero_imag ? make_float2(0.f, 0.f) : df_from_double(v.y);
  *o = make_float4(re.x, re.y, im.x, im.y);
}
__device__ __forceinline__ void cvt(float4 v, int zero_imag, float4* o) {
  if (zero_imag) v.z = v.w = 0.f;
  *o = v;
}
// scale: FP64 (FP64 values) or the same as a double-float pair (double-float values)
__device__ __forceinline__ void out_cvt(double2 v, double scale, float2, int real_out, double2* o) {
  *o = make_double2(v.x * scale, real_out ? 0.0 : v.y * scale);
}
__device__ __forceinline__ void out_cvt(float4 v, double, float2 sdf, int real_out, double2* o) {
  const double re = df_to_double(f_mulf(make_float2(v.x, v.y), sdf));
  *o = make_double2(re, real_out ? 0.0 : df_to_double(f_mulf(make_float2(v.z, v.w), sdf)));
}
// between passes: scale 1, complex (the caller passes scale = 1, real_out = 0)
__device__ __forceinline__ void out_cvt(float4 v, double, float2, int, float4* o) { *o = v; }

// Rows: `rpc` rows of length n per CTA.  `in` and `out` may alias (each CTA
// reads all of its rows before writing them).  T: arithmetic type; TI, TO:
// value types in HBM.
template <int SIGN, typename T, typename TI, typename TO>
__global__ void __launch_bounds__(256) fft_rows_kernel(const TI* in, TO* out, int nrows, int rpc, StageList st,
                                                       const T* tw, double scale, float2 sdf, int zero_imag_in,
                                                       int real_out) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  T* smem = reinterpret_cast<T*>(smem_raw);
  const int n = st.n;
  T* b0 = smem;
  T* b1 = smem + (size_t)rpc * n;
  const long long row0 = (long long)blockIdx.x * rpc;
  const int nr = (int)min((long long)rpc, nrows - row0);
  const TI* g_in = in + row0 * n;
  for (int i = threadIdx.x; i < rpc * n; i += blockDim.x) {
    T v = czero<T>();
    if (i < nr * n) cvt(g_in[i], zero_imag_in, &v);
    b0[i] = v;
  }
  __syncthreads();
  T* res = run_stages<SIGN>(b0, b1, st, rpc, n, 1, false, tw);
  TO* g_out = out + row0 * n;
  for (int i = threadIdx.x; i < nr * n; i += blockDim.x) out_cvt(res[i], scale, sdf, real_out, g_out + i);
}

// Columns: W adjacent columns of one field per CTA (blockIdx.y = field).
template <int SIGN, typename T, typename TI, typename TO>
__global__ void __launch_bounds__(512) fft_cols_kernel(const TI* in, TO* out, int nx, int W, StageList st,
                                                       const T* tw, double scale, float2 sdf, int zero_imag_in,
                                                       int real_out) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  T* smem = reinterpret_cast<T*>(smem_raw);
  const int ny = st.n;
  T* b0 = smem;
  T* b1 = smem + (size_t)W * ny;
  const int x0 = blockIdx.x * W;
  const int w = min(W, nx - x0);
  const size_t field_off = (size_t)blockIdx.y * nx * ny;
  const TI* g_in = in + field_off + x0;
#pragma unroll 8
  for (int i = threadIdx.x; i < ny * W; i += blockDim.x) {
    const int t = i / W, c = i - t * W;
    T v = czero<T>();
    if (c < w) cvt(g_in[(size_t)t * nx + c], zero_imag_in, &v);
    b0[i] = v;
  }
  __syncthreads();
  T* res = run_stages<SIGN>(b0, b1, st, W, 1, W, true, tw);
  TO* g_out = out + field_off + x0;
  for (int i = threadIdx.x; i < ny * W; i += blockDim.x) {
    const int t = i / W, c = i - t * W;
    if (c < w) out_cvt(res[i], scale, sdf, real_out, g_out + (size_t)t * nx + c);
  }
}

// ---------------------------------------------------------------------------
// Real input along x.  A real row x[0..n) (n = 2m) is transformed as the
// m-point complex sequence z[t] = x[2t] + i x[2t+1]: with Z = DFT_m(z), the
// DFTs of the even and odd samples are E[k] = (Z[k] + conj Z[m-k])/2 and
// O[k] = -i (Z[k] - conj Z[m-k])/2, and X[k] = E[k] + w^k O[k], w = e^{-2 pi i/n},
// for k = 0..m (the other half of X is its conjugate mirror).  The inverse
// forms Z[k] = (X[k] + conj X[m-k]) + i w^{-k} (X[k] - conj X[m-k]) for
// k < m, and the unnormalised inverse m-point transform of Z is n (x[2t] +
// i x[2t+1]).  Only half of the spectrum is transformed along y and handled
// by the pole step.

__device__ __forceinline__ double2 conj_of(double2 a) { return make_double2(a.x, -a.y); }
__device__ __forceinline__ float4 conj_of(float4 a) { return make_float4(a.x, a.y, -a.z, -a.w); }
__device__ __forceinline__ double2 half_of(double2 a) { return make_double2(0.5 * a.x, 0.5 * a.y); }
__device__ __forceinline__ float4 half_of(float4 a) {  // exact: scaling by a power of two
  return make_float4(0.5f * a.x, 0.5f * a.y, 0.5f * a.z, 0.5f * a.w);
}
__device__ __forceinline__ void real_pair(const double2* g, double2* v) { *v = make_double2(g[0].x, g[1].x); }
__device__ __forceinline__ void real_pair(const double2* g, float4* v) {
  cvt(make_double2(g[0].x, g[1].x), 0, v);
}
// scaled real and imaginary parts as FP64
__device__ __forceinline__ double2 to_d2(double2 v, double scale, float2) {
  return make_double2(v.x * scale, v.y * scale);
}
__device__ __forceinline__ double2 to_d2(float4 v, double, float2 sdf) {
  return make_double2(df_to_double(f_mulf(make_float2(v.x, v.y), sdf)),
                      df_to_double(f_mulf(make_float2(v.z, v.w), sdf)));
}

// Forward, rows: `rpc` real rows of length 2m per CTA -> m + 1 spectrum values each.
template <typename T, typename TO>
__global__ void __launch_bounds__(256) fft_rows_r2c_kernel(const double2* in, TO* out, int nrows, int rpc,
                                                           StageList st, const T* tw_half, const T* tw_full) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  T* smem = reinterpret_cast<T*>(smem_raw);
  const int m = st.n, n = 2 * m;
  T* b0 = smem;
  T* b1 = smem + (size_t)rpc * m;
  const long long row0 = (long long)blockIdx.x * rpc;
  const int nr = (int)min((long long)rpc, nrows - row0);
  const double2* g_in = in + row0 * n;
#pragma unroll 4
  for (int i = threadIdx.x; i < rpc * m; i += blockDim.x) {
    T v = czero<T>();
    if (i < nr * m) real_pair(g_in + 2 * (size_t)i, &v);
    b0[i] = v;
  }
  __syncthreads();
  const T* res = run_stages<-1>(b0, b1, st, rpc, m, 1, false, tw_half);
  TO* g_out = out + row0 * (m + 1);
  for (int i = threadIdx.x; i < nr * (m + 1); i += blockDim.x) {
    const int r = i / (m + 1), k = i - r * (m + 1);
    const T* zr = res + (size_t)r * m;
    const T zk = zr[k == m ? 0 : k];
    const T zc = conj_of(zr[k == 0 ? 0 : m - k]);
    const T e = half_of(cadd(zk, zc));
    const T o = half_of(mul_si<-1>(csub(zk, zc)));
    const T x = cadd(e, cmul(o, tw_load<-1>(tw_full, k)));
    out_cvt(x, 1.0, make_float2(1.f, 0.f), 0, g_out + i);
  }
}

// Inverse, rows: m + 1 spectrum values per row -> 2m real values (imaginary 0), scaled.
template <typename T, typename TI>
__global__ void __launch_bounds__(256) fft_rows_c2r_kernel(const TI* in, double2* out, int nrows, int rpc,
                                                           StageList st, const T* tw_half, const T* tw_full,
                                                           double scale, float2 sdf) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  T* smem = reinterpret_cast<T*>(smem_raw);
  const int m = st.n, n = 2 * m;
  T* b0 = smem;
  T* b1 = smem + (size_t)rpc * m;
  const long long row0 = (long long)blockIdx.x * rpc;
  const int nr = (int)min((long long)rpc, nrows - row0);
  // each thread forms Z[k] from X[k] and X[m - k] (the second read of a row
  // hits the cache lines of the first)
  const TI* g_in = in + row0 * (m + 1);
#pragma unroll 4
  for (int i = threadIdx.x; i < rpc * m; i += blockDim.x) {
    T v = czero<T>();
    if (i < nr * m) {
      const int r = i / m, k = i - r * m;
      T a, b;
      cvt(g_in[(size_t)r * (m + 1) + k], 0, &a);
      cvt(g_in[(size_t)r * (m + 1) + (m - k)], 0, &b);
      const T bc = conj_of(b);
      const T e = cadd(a, bc);
      const T o = cmul(csub(a, bc), tw_load<+1>(tw_full, k));
      v = cadd(e, mul_si<+1>(o));
    }
    b0[i] = v;
  }
  __syncthreads();
  const T* res = run_stages<+1>(b0, b1, st, rpc, m, 1, false, tw_half);
  double2* g_out = out + row0 * n;
  for (int i = threadIdx.x; i < nr * m; i += blockDim.x) {
    const double2 z = to_d2(res[i], scale, sdf);
    g_out[2 * (size_t)i] = make_double2(z.x, 0.0);
    g_out[2 * (size_t)i + 1] = make_double2(z.y, 0.0);
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

// Threads of a real-row CTA: one radix-8 butterfly per thread per stage.
static int rows_threads(int rpc, int m) { return std::min(256, std::max(64, rpc * m / 8)); }

static int rows_per_cta(int n) {
  int r = 1;
  while (r < 16 && r * n * 2 <= 1024) r *= 2;
  return r;
}
// Columns per CTA: the two stage buffers of W columns fit in kColsSmemKB of
// shared memory (64 KB: a 2048-point column per CTA, three CTAs per SM).
#ifndef REXI_COLS_SMEM_KB
#define REXI_COLS_SMEM_KB 64
#endif
constexpr size_t kColsSmemKB = REXI_COLS_SMEM_KB;
static int cols_per_cta(int n) {
  int w = 16;
  while (w > 1 && 2 * (size_t)w * n * sizeof(double2) > kColsSmemKB * 1024) w /= 2;
  return w;
}
// Threads of a column CTA: a large tile (one CTA per SM by its shared memory)
// gets 512 threads, one radix-8 butterfly each per stage.
static int cols_threads(int W, int n) { return (size_t)W * n >= 4096 ? 512 : 256; }

template <typename K>
static cudaError_t allow_smem(K kernel, size_t bytes) {
  if (bytes <= 48 * 1024) return cudaSuccess;
  return cudaFuncSetAttribute(kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)bytes);
}

// FP64 transform (T = double2), or double-float arithmetic (T = float4) with
// double-float values between the passes (in `out`, 16 bytes per value like FP64).
template <int SIGN, typename T>
static cudaError_t fft2d_impl(const double2* in, double2* out, int nfields, const FftPlan1D& px,
                              const FftPlan1D& py, const T* twx, const T* twy, double scale, int zero_imag_in,
                              int real_out, cudaStream_t s) {
  constexpr bool DF = sizeof(T) == sizeof(float4) && !std::is_same<T, double2>::value;
  using TM = typename std::conditional<DF, float4, double2>::type;  // between the passes
  const int nx = px.n, ny = py.n;
  TM* mid = reinterpret_cast<TM*>(out);
  cudaError_t e;
  {
    const int rpc = rows_per_cta(nx);
    const int nrows = nfields * ny;
    const size_t sm = 2 * (size_t)rpc * nx * sizeof(T);
    auto k = fft_rows_kernel<SIGN, T, double2, TM>;
    if ((e = allow_smem(k, sm)) != cudaSuccess) return e;
    dim3 grid((nrows + rpc - 1) / rpc);
    k<<<grid, 256, sm, s>>>(in, mid, nrows, rpc, to_stages(px), twx, 1.0, df_split_host(1.0), zero_imag_in, 0);
    if ((e = cudaGetLastError()) != cudaSuccess) return e;
  }
  {
    const int W = cols_per_cta(ny);
    const size_t sm = 2 * (size_t)W * ny * sizeof(T);
    auto k = fft_cols_kernel<SIGN, T, TM, double2>;
    if ((e = allow_smem(k, sm)) != cudaSuccess) return e;
    dim3 grid((nx + W - 1) / W, nfields);
    k<<<grid, cols_threads(W, ny), sm, s>>>(mid, out, nx, W, to_stages(py), twy, scale, df_split_host(scale), 0,
                                            real_out);
    if ((e = cudaGetLastError()) != cudaSuccess) return e;
  }
  return cudaSuccess;
}

// Real-input transforms: forward rows (half-length complex + split), then
// columns of the half spectrum; inverse columns, then rows (merge +
// half-length complex).  T: arithmetic type, TM: value type of the
// intermediate in HBM.
template <typename T, typename TS>
static cudaError_t fft2d_r2c_impl(const double2* in, double2* spec, int nfields, const FftPlan1D& px,
                                  const FftPlan1D& pxh, const FftPlan1D& py, const T* twx, const T* twxh,
                                  const T* twy, cudaStream_t s) {
  constexpr bool DF = !std::is_same<T, double2>::value;
  using TM = typename std::conditional<DF, float4, double2>::type;
  const int m = pxh.n, ny = py.n;
  TM* mid = reinterpret_cast<TM*>(spec);
  cudaError_t e;
  {
    const int rpc = rows_per_cta(m);
    const int nrows = nfields * ny;
    const size_t sm = 2 * (size_t)rpc * m * sizeof(T);
    auto k = fft_rows_r2c_kernel<T, TM>;
    if ((e = allow_smem(k, sm)) != cudaSuccess) return e;
    k<<<(nrows + rpc - 1) / rpc, rows_threads(rpc, m), sm, s>>>(in, mid, nrows, rpc, to_stages(pxh), twxh, twx);
    if ((e = cudaGetLastError()) != cudaSuccess) return e;
  }
  {
    const int W = cols_per_cta(ny);
    const size_t sm = 2 * (size_t)W * ny * sizeof(T);
    auto k = fft_cols_kernel<-1, T, TM, TS>;
    if ((e = allow_smem(k, sm)) != cudaSuccess) return e;
    dim3 grid((m + 1 + W - 1) / W, nfields);
    k<<<grid, cols_threads(W, ny), sm, s>>>(mid, reinterpret_cast<TS*>(spec), m + 1, W, to_stages(py), twy, 1.0,
                                            df_split_host(1.0), 0, 0);
    if ((e = cudaGetLastError()) != cudaSuccess) return e;
  }
  (void)px;
  return cudaSuccess;
}

template <typename T, typename TS>
static cudaError_t fft2d_c2r_impl(double2* spec, double2* out, int nfields, const FftPlan1D& px,
                                  const FftPlan1D& pxh, const FftPlan1D& py, const T* twx, const T* twxh,
                                  const T* twy, double scale, cudaStream_t s) {
  constexpr bool DF = !std::is_same<T, double2>::value;
  using TM = typename std::conditional<DF, float4, double2>::type;
  const int m = pxh.n, ny = py.n;
  TM* mid = reinterpret_cast<TM*>(spec);
  cudaError_t e;
  {
    const int W = cols_per_cta(ny);
    const size_t sm = 2 * (size_t)W * ny * sizeof(T);
    auto k = fft_cols_kernel<+1, T, TS, TM>;
    if ((e = allow_smem(k, sm)) != cudaSuccess) return e;
    dim3 grid((m + 1 + W - 1) / W, nfields);
    k<<<grid, cols_threads(W, ny), sm, s>>>(reinterpret_cast<const TS*>(spec), mid, m + 1, W, to_stages(py), twy,
                                            1.0, df_split_host(1.0), 0, 0);
    if ((e = cudaGetLastError()) != cudaSuccess) return e;
  }
  {
    const int rpc = rows_per_cta(m);
    const int nrows = nfields * ny;
    const size_t sm = 2 * (size_t)rpc * m * sizeof(T);
    auto k = fft_rows_c2r_kernel<T, TM>;
    if ((e = allow_smem(k, sm)) != cudaSuccess) return e;
    k<<<(nrows + rpc - 1) / rpc, rows_threads(rpc, m), sm, s>>>(mid, out, nrows, rpc, to_stages(pxh), twxh, twx, scale,
                                              df_split_host(scale));
    if ((e = cudaGetLastError()) != cudaSuccess) return e;
  }
  (void)px;
  return cudaSuccess;
}

bool fft_df_ready(const FftPlan1D& px, const FftPlan1D& pxh, const FftPlan1D& py) {
  return px.twf && pxh.twf && py.twf;
}

cudaError_t fft2d_r2c(const double2* in, double2* spec, int nfields, const FftPlan1D& px, const FftPlan1D& pxh,
                      const FftPlan1D& py, int df, cudaStream_t s) {
  if (df == 2 && fft_df_ready(px, pxh, py))
    return fft2d_r2c_impl<float4, float4>(in, spec, nfields, px, pxh, py, px.twf, pxh.twf, py.twf, s);
  if (df && fft_df_ready(px, pxh, py))
    return fft2d_r2c_impl<float4, double2>(in, spec, nfields, px, pxh, py, px.twf, pxh.twf, py.twf, s);
  return fft2d_r2c_impl<double2, double2>(in, spec, nfields, px, pxh, py, px.tw, pxh.tw, py.tw, s);
}

cudaError_t fft2d_c2r(double2* spec, double2* out, int nfields, const FftPlan1D& px, const FftPlan1D& pxh,
                      const FftPlan1D& py, double scale, int df, cudaStream_t s) {
  if (df == 2 && fft_df_ready(px, pxh, py))
    return fft2d_c2r_impl<float4, float4>(spec, out, nfields, px, pxh, py, px.twf, pxh.twf, py.twf, scale, s);
  if (df && fft_df_ready(px, pxh, py))
    return fft2d_c2r_impl<float4, double2>(spec, out, nfields, px, pxh, py, px.twf, pxh.twf, py.twf, scale, s);
  return fft2d_c2r_impl<double2, double2>(spec, out, nfields, px, pxh, py, px.tw, pxh.tw, py.tw, scale, s);
}

cudaError_t fft2d(const double2* in, double2* out, int nfields, const FftPlan1D& px,
                  const FftPlan1D& py, int sign, double scale, int zero_imag_in, int real_out,
                  cudaStream_t s) {
  if (sign < 0) return fft2d_impl<-1>(in, out, nfields, px, py, px.tw, py.tw, scale, zero_imag_in, real_out, s);
  return fft2d_impl<+1>(in, out, nfields, px, py, px.tw, py.tw, scale, zero_imag_in, real_out, s);
}

cudaError_t fft2d_df(const double2* in, double2* out, int nfields, const FftPlan1D& px, const FftPlan1D& py,
                     int sign, double scale, int zero_imag_in, int real_out, cudaStream_t s) {
  if (!px.twf || !py.twf) return fft2d(in, out, nfields, px, py, sign, scale, zero_imag_in, real_out, s);
  if (sign < 0) return fft2d_impl<-1>(in, out, nfields, px, py, px.twf, py.twf, scale, zero_imag_in, real_out, s);
  return fft2d_impl<+1>(in, out, nfields, px, py, px.twf, py.twf, scale, zero_imag_in, real_out, s);
}

// Double-float FFT twiddles: out[0, n) = w[t] split into pairs, then for each
// stage s (radix R, Ns the product of the earlier radices) the Ns (R - 1)
// values w[r jm n / (Ns R)], jm < Ns, r = 1..R-1, in the order
// [jm (R - 1) + r - 1] (run_stages); the stages' counts sum to n - 1, so out
// holds 2n entries (the last one unused).
void df_twiddles(const double2* tw, const FftPlan1D& p, float4* out) {
  const int n = p.n;
  split_twiddles(tw, n, out);
  int off = n, Ns = 1;
  for (int s = 0; s < p.nstages; ++s) {
    const int R = p.radix[s], twstep = n / (Ns * R);
    for (int jm = 0; jm < Ns; ++jm)
      for (int r = 1; r < R; ++r) split_twiddles(tw + (size_t)r * jm * twstep, 1, out + off + jm * (R - 1) + r - 1);
    off += Ns * (R - 1);
    Ns *= R;
  }
  out[2 * n - 1] = make_float4(0.f, 0.f, 0.f, 0.f);
}

void split_twiddles(const double2* tw, int n, float4* out) {
  for (int t = 0; t < n; ++t) {
    const float rh = (float)tw[t].x, ih = (float)tw[t].y;
    out[t] = make_float4(rh, (float)(tw[t].x - (double)rh), ih, (float)(tw[t].y - (double)ih));
  }
}

}  // namespace rexi
