// Variable-depth (Krylov) path: declarations shared with api.cu.
#pragma once

#include <cuda_runtime.h>

#include "rexi.h"

namespace rexi {

struct KrylovSettings {
  int nx = 0, ny = 0;
  double Lx = 1, Ly = 1, g = 1, f = 1, Hmean = 1;
  const double* depth = nullptr;
  double rtol = 1e-10;
  int max_iters = 20000;
  int term_batch = 64;
  void* dev_state = nullptr;  // plan-owned device scalars (flags, counters)
};

// Optional instrumentation from the plan: phase marks (0..4 per term batch)
// and a kernel-launch counter.
struct KrylovHooks {
  void (*mark)(void* ctx, int i, cudaStream_t s) = nullptr;
  void* ctx = nullptr;
  int64_t* launches = nullptr;
};

rexi_status krylov_init(KrylovSettings* k, int nx, int ny, double Lx, double Ly, double g, double f,
                        const double* depth, double Hmean);
void krylov_destroy(KrylovSettings* k);
size_t krylov_workspace_bytes(const KrylovSettings* k, int M, int real_input, int form);
rexi_status krylov_step(KrylovSettings* k, int form, double h, int M, const void* in, void* out, double dt,
                        int real_input, int term_begin, int term_end, void* ws, size_t ws_bytes,
                        cudaStream_t s, rexi_step_info* info, bool adjoint, const KrylovHooks& hooks);

}  // namespace rexi
