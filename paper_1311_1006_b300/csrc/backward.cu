// Adjoint evaluation (placeholder until the dual-strength kernels land).
#include "fmm_internal.cuh"

namespace fmm {
fmm_status run_backward(Tree& t, const double*, const double*, double*, double*, cudaStream_t) {
    (void)t;
    set_error("backward not built yet");
    return FMM_ERR_INVALID_ARG;
}
}  // namespace fmm
