// lbm_batch_fused.cuh -- two time steps per launch for a whole batch: one CTA
// per 64 x 16 tile of any lattice of the batch, each running the tile body of
// the two-step kernel (lbm_fused.cuh) for its lattice's storage kind, edges,
// force and rounding.
//
// Every lattice keeps two population arrays that trade roles at every launch
// (ping-pong): launch k of a sequence reads arr[k & 1] and writes
// arr[(k & 1) ^ 1] of every lattice, so an even number of launches ends on the
// arrays the sequence started from.  The tiles of one lattice are independent
// within a launch (each reads its halo from the input array and writes only its
// own nodes to the output array), and the lattices are independent of each
// other, so no CTA waits on another.
#pragma once

#include "lbm_batch_impl.cuh"
#include "lbm_fused.cuh"

namespace lbm {

// Per-lattice part of a two-step launch: both arrays and the tensor map of
// each (map[j] describes arr[j]).  Tensor maps read by TMA from global memory
// need 64-byte alignment.
struct alignas(64) BatchPair {
    CUtensorMap map[2];
    void* arr[2];
};

// Shared memory of the two-step batch kernel: the largest tile buffer of the
// storage kinds a batch may hold.
constexpr size_t kBatchFusedSmem =
    FusedGeom<LBM_F32>::SMEM > FusedGeom<LBM_F16DEV>::SMEM ? FusedGeom<LBM_F32>::SMEM : FusedGeom<LBM_F16DEV>::SMEM;
static_assert(FusedTile<LBM_F32>::THREADS == FusedTile<LBM_F16DEV>::THREADS &&
                  FusedGeom<LBM_F32>::TX == FusedGeom<LBM_F16DEV>::TX && FusedGeom<LBM_F32>::TY == FusedGeom<LBM_F16DEV>::TY,
              "one tile shape and CTA size for every storage kind");
constexpr int kBatchFusedThreads = FusedTile<LBM_F32>::THREADS;
// The packed FP32x2 stages of the two-step tile (lbm_fused.cuh) in the batch
// kernel, which carries every storage, edge, force and rounding path in one
// kernel.
constexpr bool kBatchPacked = false;
constexpr int kBatchFusedTX = FusedGeom<LBM_F32>::TX, kBatchFusedTY = FusedGeom<LBM_F32>::TY;

template <int MODEL, int STORE, int FORCE, bool WALLS>
__device__ __forceinline__ void batch_fused_sr(const BatchPair& P, const Args& a, int src, int* err, int x0, int y0,
                                               unsigned rb0, unsigned rb1, unsigned char* smem,
                                               unsigned long long* bar, int* ok) {
    if (a.rseed)
        fused2_tile<MODEL, STORE, FORCE, WALLS, true, kBatchPacked>(&P.map[src], a, P.arr[src], P.arr[src ^ 1], err, x0,
                                                                    y0, rb0, rb1, smem, bar, ok);
    else
        fused2_tile<MODEL, STORE, FORCE, WALLS, false, kBatchPacked>(&P.map[src], a, P.arr[src], P.arr[src ^ 1], err, x0,
                                                                     y0, 0u, 0u, smem, bar, ok);
}

template <int MODEL, int STORE>
__device__ __forceinline__ void batch_fused_store(const BatchDomain& D, const BatchPair& P, int src, int* err, int x0,
                                                  int y0, unsigned rb0, unsigned rb1, unsigned char* smem,
                                                  unsigned long long* bar, int* ok) {
    if (D.walls) {
        if (D.force) batch_fused_sr<MODEL, STORE, 1, true>(P, D.a, src, err, x0, y0, rb0, rb1, smem, bar, ok);
        else batch_fused_sr<MODEL, STORE, 0, true>(P, D.a, src, err, x0, y0, rb0, rb1, smem, bar, ok);
    } else {
        if (D.force) batch_fused_sr<MODEL, STORE, 1, false>(P, D.a, src, err, x0, y0, rb0, rb1, smem, bar, ok);
        else batch_fused_sr<MODEL, STORE, 0, false>(P, D.a, src, err, x0, y0, rb0, rb1, smem, bar, ok);
    }
}

// tiles: 3 ints per tile (lattice, tile x, tile y) of 64 x 16 nodes; launch k
// of a sequence reads arr[k & 1]; the stochastic-rounding hashes of its two
// steps are rtab[d * rstride + 2 kstep] and [... + 1].
template <int MODEL>
__global__ void __launch_bounds__(kBatchFusedThreads, FusedTile<LBM_F32>::MIN_BLOCKS)
    batch_fused_kernel(const BatchDomain* __restrict__ doms, const BatchPair* __restrict__ pairs,
                       const int* __restrict__ tiles, int k, const unsigned* __restrict__ rtab, int rstride, int kstep,
                       int* __restrict__ err) {
    extern __shared__ __align__(1024) unsigned char fused_smem[];
    __shared__ BatchDomain sdom;
    __shared__ __align__(8) unsigned long long bar;
    __shared__ int ok;
    const int t = blockIdx.x;
    const int dom = tiles[3 * t], tx = tiles[3 * t + 1], ty = tiles[3 * t + 2];
    {  // the lattice's descriptor into shared memory (every constant of the update a shared-memory operand)
        const int4* src = reinterpret_cast<const int4*>(doms + dom);
        int4* dst = reinterpret_cast<int4*>(&sdom);
        for (int c = threadIdx.x; c < kDomChunks; c += blockDim.x) dst[c] = src[c];
    }
    __syncthreads();
    const BatchDomain& D = sdom;
    const BatchPair& P = pairs[dom];
    unsigned rb0 = 0u, rb1 = 0u;
    if (D.a.rseed) {
        rb0 = rtab[dom * rstride + 2 * kstep];
        rb1 = rtab[dom * rstride + 2 * kstep + 1];
    }
    const int src = k & 1;
    const int x0 = tx * kBatchFusedTX, y0 = ty * kBatchFusedTY;
    switch (D.store) {
        case LBM_F32: batch_fused_store<MODEL, LBM_F32>(D, P, src, err, x0, y0, rb0, rb1, fused_smem, &bar, &ok); break;
        case LBM_F16DEV: batch_fused_store<MODEL, LBM_F16DEV>(D, P, src, err, x0, y0, rb0, rb1, fused_smem, &bar, &ok); break;
        default: batch_fused_store<MODEL, LBM_BF16DEV>(D, P, src, err, x0, y0, rb0, rb1, fused_smem, &bar, &ok); break;
    }
}

template <int MODEL>
static cudaError_t launch_batch_fused_model(int ntiles, const BatchDomain* doms, const BatchPair* pairs, const int* tiles,
                                            int k, const unsigned* rtab, int rstride, int kstep, int* err,
                                            cudaStream_t s) {
    static bool configured = false;
    if (!configured) {
        cudaError_t e = cudaFuncSetAttribute(batch_fused_kernel<MODEL>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                             int(kBatchFusedSmem));
        if (e != cudaSuccess) return e;
        configured = true;
    }
    if (ntiles < 1) return cudaSuccess;
    batch_fused_kernel<MODEL><<<ntiles, kBatchFusedThreads, kBatchFusedSmem, s>>>(doms, pairs, tiles, k, rtab, rstride,
                                                                                  kstep, err);
    return cudaGetLastError();
}

}  // namespace lbm
