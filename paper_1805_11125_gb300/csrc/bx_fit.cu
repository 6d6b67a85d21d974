// bx_fit.cu -- batched quasi-Newton fits driven by the adjoint gradient.
#include "bx_model.h"

void bx_fit_free(bx_model*) {}

extern "C" int bx_fit(bx_model* m, int, const int*, const double*, const bx_fit_opts*, double*, bx_fit_result*) {
    if (!m) return bx_set_error(BX_EINVAL, "model is NULL");
    return bx_set_error(BX_EINVAL, "bx_fit: not available in this build");
}
