// rexi_alu_probe: arithmetic throughput probe used to measure the FP32 and
// FP64 fused multiply-add rates that bound the pole-sum kernels (a
// measurement utility; the paper has no counterpart).
//
// Every thread runs kChains (16) independent multiply-add recurrences
// acc = acc * m + c (m slightly below 1, so the values settle at c / (1 - m)
// and never become subnormal or overflow) for `iters` rounds, so the pipes see
// kChains independent operations per round and per thread.  One value per
// thread is folded and written only when it matches an impossible sentinel,
// which keeps the work observable to the compiler without memory traffic.
#include <stdint.h>

#include "internal.h"

namespace {

constexpr int kChains = 16;  // enough independent work to cover the FP64 pipe's latency too
constexpr int kThreads = 256;

template <typename T>
__global__ void __launch_bounds__(kThreads) alu_probe_kernel(int iters, T m, T c, T* out) {
  T acc[kChains];
#pragma unroll
  for (int i = 0; i < kChains; ++i) acc[i] = (T)(threadIdx.x + i) * (T)1e-3;
  for (int it = 0; it < iters; ++it) {
#pragma unroll
    for (int u = 0; u < 16; ++u) {
#pragma unroll
      for (int i = 0; i < kChains; ++i) acc[i] = fma(acc[i], m, c);
    }
  }
  T s = 0;
#pragma unroll
  for (int i = 0; i < kChains; ++i) s += acc[i];
  if (s == (T)-1.0) out[blockIdx.x * blockDim.x + threadIdx.x] = s;
}

// Packed FP32: each fma.rn.f32x2 does two FP32 multiply-adds (the two halves of
// a 64-bit register), kChains packed chains per thread.
__device__ __forceinline__ unsigned long long fma_f32x2(unsigned long long a, unsigned long long b,
                                                       unsigned long long c) {
  unsigned long long d;
  asm("fma.rn.f32x2 %0, %1, %2, %3;" : "=l"(d) : "l"(a), "l"(b), "l"(c));
  return d;
}
__device__ __forceinline__ unsigned long long pack2(float lo, float hi) {
  return (unsigned long long)__float_as_uint(lo) | ((unsigned long long)__float_as_uint(hi) << 32);
}

__global__ void __launch_bounds__(kThreads) alu_probe_f32x2_kernel(int iters, float m, float c, float* out) {
  unsigned long long acc[kChains];
#pragma unroll
  for (int i = 0; i < kChains; ++i) acc[i] = pack2((float)(threadIdx.x + i) * 1e-3f, (float)(threadIdx.x + 2 * i) * 1e-3f);
  const unsigned long long mm = pack2(m, m), cc = pack2(c, c);
  for (int it = 0; it < iters; ++it) {
#pragma unroll
    for (int u = 0; u < 16; ++u) {
#pragma unroll
      for (int i = 0; i < kChains; ++i) acc[i] = fma_f32x2(acc[i], mm, cc);
    }
  }
  float s = 0.f;
#pragma unroll
  for (int i = 0; i < kChains; ++i) s += __uint_as_float((unsigned)acc[i]) + __uint_as_float((unsigned)(acc[i] >> 32));
  if (s == -1.0f) out[blockIdx.x * blockDim.x + threadIdx.x] = s;
}

}  // namespace

// kind 0: FP32 (fmaf), kind 1: FP64 (fma), kind 2: packed FP32 (fma.rn.f32x2,
// two multiply-adds per instruction, so twice the flops of kind 0 per call).  blocks x 256 threads, each
// thread 16 * 16 * iters multiply-adds (2 flops each).  out_dev: at least
// blocks * 256 values of the kind's type (written only in the impossible
// sentinel case).  Asynchronous on `stream`; the caller times it.
extern "C" rexi_status rexi_alu_probe(int32_t kind, int32_t blocks, int32_t iters, void* out_dev, void* stream) {
  rexi::set_last_error("");
  if (kind < 0 || kind > 2 || blocks < 1 || iters < 1 || !out_dev) {
    rexi::set_last_error("rexi_alu_probe: kind must be 0, 1 or 2, blocks and iters >= 1, out non-NULL");
    return REXI_EINVAL;
  }
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  if (kind == 0)
    alu_probe_kernel<float><<<blocks, kThreads, 0, s>>>(iters, 0.9999999f, 1e-7f, static_cast<float*>(out_dev));
  else if (kind == 1)
    alu_probe_kernel<double><<<blocks, kThreads, 0, s>>>(iters, 0.9999999, 1e-7, static_cast<double*>(out_dev));
  else
    alu_probe_f32x2_kernel<<<blocks, kThreads, 0, s>>>(iters, 0.9999999f, 1e-7f, static_cast<float*>(out_dev));
  const cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) {
    rexi::set_last_error(cudaGetErrorString(e));
    return REXI_ECUDA;
  }
  return REXI_OK;
}
