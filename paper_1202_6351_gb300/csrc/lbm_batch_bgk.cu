// lbm_batch_bgk.cu -- batch kernels (one step, and two steps per launch) for the bgk collision.
#include "lbm_batch_fused.cuh"
#include "lbm_batch_impl.cuh"

namespace lbm {
cudaError_t launch_batch_bgk(int grid, const BatchDomain* doms, const int* tiles, int ntiles, int lbx, int rows, int flip,
                            int policy, int* counter, const unsigned* rtab, int rstride, int kstep,
                            cudaStream_t s) {
    batch_kernel<LBM_BGK><<<grid, kBatchThreads, 0, s>>>(doms, tiles, ntiles, lbx, rows, flip, policy, counter, rtab, rstride, kstep);
    return cudaGetLastError();
}
int batch_blocks_per_sm_bgk() {
    int n = 0;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n, batch_kernel<LBM_BGK>, kBatchThreads, 0) != cudaSuccess) return 1;
    return n > 0 ? n : 1;
}
cudaError_t launch_batch_fused_bgk(int cls, int ntiles, const BatchDomain* doms, const BatchPair* pairs,
                                  const int* tiles, int k, const unsigned* rtab, int rstride, int kstep, int* err,
                                  cudaStream_t s) {
    return launch_batch_fused_model<LBM_BGK>(cls, ntiles, doms, pairs, tiles, k, rtab, rstride, kstep, err, s);
}
}  // namespace lbm
