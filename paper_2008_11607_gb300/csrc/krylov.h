// Variable-depth (Krylov) path: declarations shared with api.cu.
#pragma once

#include <cuda_runtime.h>

#include "rexi.h"

namespace rexi {

struct KrylovSettings {
  int nx = 0, ny = 0;
  double Lx = 1, Ly = 1, g = 1, f = 1, Hmean = 1;
  const double* depth = nullptr;
  double rtol = 1e-10;        // relative residual target per term (energy norm)
  int max_iters = 20000;      // CG iteration cap per term (per inner solve in the mixed form)
  int term_batch = 64;        // terms solved together in one launch
  double inner_rtol = 1e-4;   // mixed form: FP32 inner solve target per refinement step
  int max_outer = 30;         // mixed form: refinement steps cap
  int method = 0;             // 0: CG per REXII term; 1: one Lanczos basis shared by all poles
  double rho_bound = 0;       // upper bound of ||A||_W (the plan's own rho)
  double* pinned = nullptr;   // small pinned host buffer (convergence checks)
  cudaEvent_t ev[2] = {nullptr, nullptr};
  void* dev_state = nullptr;  // plan-owned device tables below
  double* w64 = nullptr;      // energy weight g / H (FP64)
  float* H32 = nullptr;       // depth (FP32 copy for the inner solver)
  float* w32 = nullptr;       // energy weight (FP32)
  float2* Hdf = nullptr;      // depth and energy weight as double-float pairs (shared-Krylov mixed form)
  float2* wdf = nullptr;
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
size_t krylov_grad_workspace_bytes(const KrylovSettings* k, int M, int real_input, int form, double h);
rexi_status krylov_step(KrylovSettings* k, int form, double h, int M, const void* in, void* out, double dt,
                        int real_input, int term_begin, int term_end, void* ws, size_t ws_bytes,
                        cudaStream_t s, rexi_step_info* info, bool adjoint, const KrylovHooks& hooks);
// Shared-Krylov (multi-shift Lanczos) variant of krylov_step: FP64, or
// double-float for the mixed form with real input.
size_t lanczos_workspace_bytes(const KrylovSettings* k, int M, int real_input);
rexi_status lanczos_tables(KrylovSettings* k);  // fills Hdf, wdf
// Depth gradient from two kept Lanczos bases (real input; FP64).
size_t lanczos_grad_workspace_bytes(const KrylovSettings* k, int M, double h);
rexi_status krylov_grad_depth_lanczos(KrylovSettings* k, int form, double h, int M, const void* f_in,
                                      const void* g_out,
                                      double* grad_depth, double dt, void* ws, size_t ws_bytes, cudaStream_t s,
                                      rexi_step_info* info, const KrylovHooks& hooks);
rexi_status krylov_step_lanczos(KrylovSettings* k, int form, double h, int M, const void* in, void* out, double dt,
                                int real_input, int term_begin, int term_end, void* ws, size_t ws_bytes,
                                cudaStream_t s, rexi_step_info* info, bool adjoint, const KrylovHooks& hooks);
// grad_depth += dL/dH for out = r(dt A(H)) f_in and G = dL/d out.
rexi_status krylov_grad_depth(KrylovSettings* k, int form, double h, int M, const void* f_in, const void* g_out,
                              double* grad_depth, double dt, int real_input, void* ws, size_t ws_bytes,
                              cudaStream_t s, rexi_step_info* info, const KrylovHooks& hooks);

}  // namespace rexi
