// Reading the per-tile partial sums that the blocks of a grid publish for the
// last block to finish (each block: store its partial, __threadfence, then an
// atomicAdd on a counter; the block that draws the last ticket sums them).
#pragma once

#include <cuda_runtime.h>

namespace rexi {

// Relaxed loads at GPU scope: they bypass the L1 cache (which another SM's
// stores do not update) and, unlike a loop of volatile loads, several can be
// in flight at once.
__device__ __forceinline__ double ld_partial(const double* p) {
  double v;
  asm volatile("ld.relaxed.gpu.global.f64 %0, [%1];" : "=d"(v) : "l"(p) : "memory");
  return v;
}
__device__ __forceinline__ double2 ld_partial(const double2* p) {
  double2 v;
  asm volatile("ld.relaxed.gpu.global.v2.f64 {%0, %1}, [%2];" : "=d"(v.x), "=d"(v.y) : "l"(p) : "memory");
  return v;
}
__device__ __forceinline__ float2 ld_partial(const float2* p) {
  float2 v;
  asm volatile("ld.relaxed.gpu.global.v2.f32 {%0, %1}, [%2];" : "=f"(v.x), "=f"(v.y) : "l"(p) : "memory");
  return v;
}

// s + partials[first] + partials[first + stride] + ... (indices below n),
// added in ascending index order.  The loads go out eight at a time before
// their sums, so a thread waits for one L2 round trip per eight partials
// instead of one per partial; the order of the additions, and so the result,
// is that of the plain loop.
template <typename T, typename Add>
__device__ __forceinline__ T strided_partial_sum(const T* partials, int n, int first, int stride, T s, Add add) {
  int i = first;
  for (; i + 7 * stride < n; i += 8 * stride) {
    T v[8];
#pragma unroll
    for (int k = 0; k < 8; ++k) v[k] = ld_partial(partials + i + k * stride);
#pragma unroll
    for (int k = 0; k < 8; ++k) s = add(s, v[k]);
  }
  for (; i < n; i += stride) s = add(s, ld_partial(partials + i));
  return s;
}

}  // namespace rexi
