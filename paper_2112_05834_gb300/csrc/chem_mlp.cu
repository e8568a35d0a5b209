// Learned per-cell cost and initial-step model (placeholder until the BF16 kernels land).
#include "chem_capi_internal.h"
#include "chem_mlp_internal.h"

chem_status chem_internal_mlp_predict(chem_handle h, const double*, const double*, const double*, int64_t,
                                      cudaStream_t, const float**, const double**) {
  h->err = "learned model not available";
  return CHEM_ERR_INVALID_ARG;
}

void chem_internal_release_learned(chem_handle) {}
