// lbm_step_bf16.cu -- fused step kernels for LBM_BF16DEV storage.
#include "lbm_step_impl.cuh"

namespace lbm {
cudaError_t launch_step_bf16(const Args& a, int model, bool odd, int force, bool walls, cudaStream_t s) {
    return launch_step_store<LBM_BF16DEV>(a, model, odd, force, walls, s);
}
}  // namespace lbm
