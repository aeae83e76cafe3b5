// kuramoto_general.cu -- Eq. 2 with a general coupling matrix K_ij.
#include "kuramoto.h"
#include "kuramoto_internal.h"

namespace sde {

sde_status kuramoto_general_alloc(KuramotoCtx *) { return SDE_OK; }
void kuramoto_general_free(KuramotoCtx *) {}
sde_status kuramoto_general_run(KuramotoCtx *, const sde_run_desc *, cudaStream_t, double *) {
  set_error("general coupling is not built yet");
  return SDE_ERR_UNSUPPORTED;
}
sde_status kuramoto_set_coupling(KuramotoCtx *, const float *, cudaStream_t) {
  set_error("general coupling is not built yet");
  return SDE_ERR_UNSUPPORTED;
}

}  // namespace sde
