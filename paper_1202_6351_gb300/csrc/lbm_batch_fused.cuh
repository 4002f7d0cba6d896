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
//
// The lattices fall into classes by storage kind, edges, force and rounding
// (the template arguments of the tile body).  The tile list is ordered by
// class and each class has a kernel of its own, so every kernel carries one
// tile body under its register budget, as the single-lattice kernel does; the
// kernels of one two-step launch are independent and run side by side.  Every
// class collides one node per thread: the packed FP32x2 node pairs of the
// single-lattice kernel spill here (the tile decode takes registers of its
// own) and ran slower.
#pragma once

#include <utility>

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

static_assert(FusedTile<LBM_F32>::THREADS == FusedTile<LBM_F16DEV>::THREADS &&
                  FusedGeom<LBM_F32>::TX == FusedGeom<LBM_F16DEV>::TX && FusedGeom<LBM_F32>::TY == FusedGeom<LBM_F16DEV>::TY,
              "one tile shape and CTA size for every storage kind");
constexpr int kBatchFusedThreads = FusedTile<LBM_F32>::THREADS;
constexpr int kBatchFusedTX = FusedGeom<LBM_F32>::TX, kBatchFusedTY = FusedGeom<LBM_F32>::TY;

// Class of a lattice: storage kind (FP32, FP16, BF16 deviations), any wall,
// uniform force, stochastic rounding.
constexpr int kBatchClasses = 24;
inline int batch_class(int store, bool walls, int force, bool sr) {
    const int s = store == LBM_F32 ? 0 : (store == LBM_F16DEV ? 1 : 2);
    return ((s * 2 + (walls ? 1 : 0)) * 2 + (force ? 1 : 0)) * 2 + (sr ? 1 : 0);
}

// tiles: 3 ints per tile (lattice, tile x, tile y) of 64 x 16 nodes, every
// lattice of this kernel's class; launch k of a sequence reads arr[k & 1];
// the stochastic-rounding hashes of its two steps are
// rtab[d * rstride + 2 kstep] and [... + 1].
template <int MODEL, int STORE, int FORCE, bool WALLS, bool SR>
__global__ void __launch_bounds__(FusedTile<STORE>::THREADS, FusedTile<STORE>::MIN_BLOCKS)
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
    const BatchPair& P = pairs[dom];
    const unsigned rb0 = SR ? rtab[dom * rstride + 2 * kstep] : 0u;
    const unsigned rb1 = SR ? rtab[dom * rstride + 2 * kstep + 1] : 0u;
    const int src = k & 1;
    fused2_tile<MODEL, STORE, FORCE, WALLS, SR, false>(&P.map[src], sdom.a, P.arr[src], P.arr[src ^ 1], err,
                                                       tx * kBatchFusedTX, ty * kBatchFusedTY, rb0, rb1, fused_smem,
                                                       &bar, &ok);
}

template <int MODEL, int CLS>
static cudaError_t launch_batch_class(int ntiles, const BatchDomain* doms, const BatchPair* pairs, const int* tiles,
                                      int k, const unsigned* rtab, int rstride, int kstep, int* err, cudaStream_t s) {
    constexpr int STORE = CLS / 8 == 0 ? LBM_F32 : (CLS / 8 == 1 ? LBM_F16DEV : LBM_BF16DEV);
    constexpr bool WALLS = (CLS / 4) & 1, SR = CLS & 1;
    constexpr int FORCE = (CLS / 2) & 1;
    constexpr size_t SMEM = FusedGeom<STORE>::SMEM;
    static bool configured = false;
    if (!configured) {
        cudaError_t e = cudaFuncSetAttribute(batch_fused_kernel<MODEL, STORE, FORCE, WALLS, SR>,
                                             cudaFuncAttributeMaxDynamicSharedMemorySize, int(SMEM));
        if (e != cudaSuccess) return e;
        configured = true;
    }
    if (ntiles < 1) return cudaSuccess;
    batch_fused_kernel<MODEL, STORE, FORCE, WALLS, SR><<<ntiles, kBatchFusedThreads, SMEM, s>>>(
        doms, pairs, tiles, k, rtab, rstride, kstep, err);
    return cudaGetLastError();
}

using BatchClassLaunch = cudaError_t (*)(int, const BatchDomain*, const BatchPair*, const int*, int, const unsigned*, int,
                                         int, int*, cudaStream_t);

template <int MODEL, int... C>
static cudaError_t launch_batch_fused_class(std::integer_sequence<int, C...>, int cls, int ntiles,
                                            const BatchDomain* doms, const BatchPair* pairs, const int* tiles, int k,
                                            const unsigned* rtab, int rstride, int kstep, int* err, cudaStream_t s) {
    static constexpr BatchClassLaunch table[] = {launch_batch_class<MODEL, C>...};
    if (cls < 0 || cls >= int(sizeof...(C))) return cudaErrorInvalidValue;
    return table[cls](ntiles, doms, pairs, tiles, k, rtab, rstride, kstep, err, s);
}

// The kernel of class `cls` over `ntiles` tiles of that class.
template <int MODEL>
static cudaError_t launch_batch_fused_model(int cls, int ntiles, const BatchDomain* doms, const BatchPair* pairs,
                                            const int* tiles, int k, const unsigned* rtab, int rstride, int kstep,
                                            int* err, cudaStream_t s) {
    return launch_batch_fused_class<MODEL>(std::make_integer_sequence<int, kBatchClasses>(), cls, ntiles, doms, pairs,
                                           tiles, k, rtab, rstride, kstep, err, s);
}

}  // namespace lbm
