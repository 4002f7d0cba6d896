// lbm_step_bf16.cu -- fused step kernels for LBM_BF16DEV storage.
#include "lbm_step_impl.cuh"
#include "lbm_fused.cuh"

namespace lbm {
cudaError_t launch_step_bf16(const Args& a, int model, bool odd, int force, bool walls, cudaStream_t s) {
    return launch_step_store<LBM_BF16DEV>(a, model, odd, force, walls, s);
}
cudaError_t launch_fused_bf16(const CUtensorMap& map, const Args& a, void* out, int* err, int model, int force,
                              bool walls, cudaStream_t s) {
    return launch_fused_store<LBM_BF16DEV>(map, a, out, err, model, force, walls, s);
}
size_t fused_smem_bf16() { return FusedGeom<LBM_BF16DEV>::SMEM; }
}  // namespace lbm
