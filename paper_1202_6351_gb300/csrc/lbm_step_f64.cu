// lbm_step_f64.cu -- fused step kernels for LBM_F64 storage.
#include "lbm_step_impl.cuh"

namespace lbm {
cudaError_t launch_step_f64(const Args& a, int model, bool odd, int force, bool walls, cudaStream_t s) {
    return launch_step_store<LBM_F64>(a, model, odd, force, walls, s);
}
}  // namespace lbm
