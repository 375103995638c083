// Variable-depth (Krylov) path.  Placeholder until the pole-batched solver lands.
#include "krylov.h"

namespace rexi {

rexi_status krylov_init(KrylovSettings* k, int nx, int ny, double Lx, double Ly, double g, double f,
                        const double* depth, double Hmean) {
  k->nx = nx; k->ny = ny; k->Lx = Lx; k->Ly = Ly; k->g = g; k->f = f; k->depth = depth; k->Hmean = Hmean;
  return REXI_OK;
}
void krylov_destroy(KrylovSettings*) {}
size_t krylov_workspace_bytes(const KrylovSettings*, int, int, int) { return 256; }
rexi_status krylov_step(KrylovSettings*, int, double, int, const void*, void*, double, int, int, int, void*,
                        size_t, cudaStream_t, rexi_step_info*, bool) {
  return REXI_EUNSUPPORTED;
}

}  // namespace rexi
