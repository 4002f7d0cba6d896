// lbm_step_f32.cu -- fused step kernels for LBM_F32 storage.
#include "lbm_step_impl.cuh"
#include "lbm_fused.cuh"

namespace lbm {
cudaError_t launch_step_f32(const Args& a, int model, bool odd, int force, bool walls, cudaStream_t s) {
    return launch_step_store<LBM_F32>(a, model, odd, force, walls, s);
}
cudaError_t launch_fused_f32(const CUtensorMap& map, const Args& a, void* out, int* err, int model, int force,
                              bool walls, cudaStream_t s) {
    return launch_fused_store<LBM_F32>(map, a, out, err, model, force, walls, s);
}
size_t fused_smem_f32() { return FusedGeom<LBM_F32>::SMEM; }
}  // namespace lbm
