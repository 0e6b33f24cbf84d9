// ens.cu -- ensemble entry points (persistent multi-grid launch).
#include "../../include/advect.h"
#include "ctx.h"

extern "C" {

advect_status advect_ensemble_create(int, const int*, const int*, const int*, const advect_coeffs*,
                                     advect_dtype, advect_ctx** out) {
  if (out) *out = nullptr;
  return ADVECT_EUNSUPPORTED;
}

advect_status advect_ensemble_forward(advect_ctx*, const void* const*, const void* const*,
                                      const void* const*, void* const*, void* const*, void* const*,
                                      advect_stream) {
  return ADVECT_EUNSUPPORTED;
}

advect_status advect_ensemble_adjoint(advect_ctx*, const void* const*, const void* const*,
                                      const void* const*, const void* const*, const void* const*,
                                      const void* const*, void* const*, void* const*, void* const*,
                                      advect_stream) {
  return ADVECT_EUNSUPPORTED;
}

}  // extern "C"
