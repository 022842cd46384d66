// xc_vjp.cu -- adjoint (vector-Jacobian product) of the cross section.
#include "xc_batched.cuh"

namespace xc {

xc_status vjp_run(BatchedState *st, const VjpArgs &a, int64_t *launches) {
    (void)st; (void)a; (void)launches;
    set_error("adjoint not built yet");
    return XC_EUNSUPPORTED;
}

}  // namespace xc
