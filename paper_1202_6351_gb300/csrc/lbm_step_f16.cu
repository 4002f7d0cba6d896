// lbm_step_f16.cu -- fused step kernels for LBM_F16DEV storage.
#include "lbm_step_impl.cuh"
#include "lbm_fused.cuh"

namespace lbm {
cudaError_t launch_step_f16(const Args& a, int model, bool odd, int force, bool walls, cudaStream_t s) {
    return launch_step_store<LBM_F16DEV>(a, model, odd, force, walls, s);
}
cudaError_t launch_fused_f16(const CUtensorMap& map, const Args& a, void* out, int* err, int model, int force,
                              bool walls, cudaStream_t s) {
    return launch_fused_store<LBM_F16DEV>(map, a, out, err, model, force, walls, s);
}
size_t fused_smem_f16() { return FusedGeom<LBM_F16DEV>::SMEM; }
}  // namespace lbm
