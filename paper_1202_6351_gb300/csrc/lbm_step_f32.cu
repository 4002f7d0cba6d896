// lbm_step_f32.cu -- fused step kernels for LBM_F32 storage.
#include "lbm_step_impl.cuh"

namespace lbm {
cudaError_t launch_step_f32(const Args& a, int model, bool odd, int force, bool walls, cudaStream_t s) {
    return launch_step_store<LBM_F32>(a, model, odd, force, walls, s);
}
}  // namespace lbm
