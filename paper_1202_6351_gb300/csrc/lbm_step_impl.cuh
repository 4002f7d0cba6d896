// lbm_step_impl.cuh -- the fused D2Q9 stream-and-collide kernel, instantiated
// once per storage type by lbm_step_<store>.cu.
//
// One thread per node (variant 0; variant 1 takes two rows per thread with
// packed FP32x2 arithmetic, variant 2 four nodes of a row per thread with
// 64-bit accesses for 16-bit stores): AA-pattern load of the nine populations
// with the wall links resolved (Eq. 24, Sec. III-A, III-C), decode of the
// stored deviations to FP32/FP64, macroscopic fields (Eq. 26-27), raw moments
// (Eq. 15), source (Eq. 13-14), cascaded kernel g3..g8 (Eq. 17-22) or a
// sibling collision, back-transform (Eq. 25), encode and AA-pattern store.
// All of it in registers, one launch per time step.
#pragma once

#include "lbm_internal.h"
#include "lbm_pair.cuh"
#include "lbm_vec.cuh"

namespace lbm {

template <int MODEL, int STORE, bool ODD, int FORCE, bool WALLS, bool SR = false>
__global__ void __launch_bounds__(kStepBX * kStepBY) step_kernel(const Args a) {
    const int x = blockIdx.x * blockDim.x + threadIdx.x;
    const int y = blockIdx.y * blockDim.y + threadIdx.y;
    if (x >= a.nx || y >= a.ny) return;
    step_node_split<MODEL, STORE, ODD, FORCE, WALLS, SR>(a, x, y, SR ? round_base(a) : 0u);
}

// One node per thread from a.f into a.fo (out of place; periodic lattices,
// FP32 and FP64 storage: the adjoint's forward and recomputed steps).
template <int MODEL, int STORE, bool ODD, int FORCE, bool SR>
__global__ void __launch_bounds__(kStepBX * kStepBY) step_kernel_oop(const Args a) {
    const int x = blockIdx.x * blockDim.x + threadIdx.x;
    const int y = blockIdx.y * blockDim.y + threadIdx.y;
    if (x >= a.nx || y >= a.ny) return;
    step_node<MODEL, STORE, ODD, FORCE, false, SR, true>(a, x, y, SR ? round_base(a) : 0u);
}

// Two rows per thread (nodes (x, y) and (x, y + 1)) with packed FP32x2
// arithmetic; a pair that touches a wall edge takes the per-node wall path.
template <int MODEL, int STORE, bool ODD, int FORCE, bool WALLS>
__global__ void __launch_bounds__(kStepBX * kStepBY, 4) step_kernel_pair(const Args a) {
    const int x = blockIdx.x * blockDim.x + threadIdx.x;
    const int y = 2 * (blockIdx.y * blockDim.y + threadIdx.y);
    if (x >= a.nx || y >= a.ny) return;
    const bool two = y + 1 < a.ny;
    if (WALLS && ((x == 0) | (x == a.nx - 1) | (y == 0) | (y + 1 >= a.ny - 1))) {
        step_node_split<MODEL, STORE, ODD, FORCE, true>(a, x, y);
        if (two) step_node_split<MODEL, STORE, ODD, FORCE, true>(a, x, y + 1);
        return;
    }
    step_pair<MODEL, STORE, ODD, FORCE>(a, x, y, two);
}

// N nodes of a row per thread (16-bit stores, no per-node force field);
// vectors that need a wrapped or wall neighbour take the per-node path.
// The CTA is bx x by threads with bx a multiple of 32, so the lanes of a warp
// hold consecutive vectors of one row (step_vec exchanges elements between
// neighbouring lanes on odd steps).
// Register budget per parity, as measured: the even step keeps all nine planes
// aligned and spills at 64 registers, so it gets 80 (6 CTAs of 128 threads per
// SM); the odd step runs faster with more warps at 64 (8 CTAs per SM).  CTAs of
// 128 threads rather than 256 run the four-node kernel 3-4 % faster (FP16 on
// 4096^2: 145.5 against 140.6 GLUPS).
constexpr int kVecThreads = 128;

template <int N, int MODEL, int STORE, bool ODD, int FORCE, bool WALLS, bool SR>
__global__ void __launch_bounds__(kVecThreads, ODD ? 8 : 6) step_kernel_vec(const Args a) {
    const int x0 = N * (blockIdx.x * blockDim.x + threadIdx.x);
    const int y = blockIdx.y * blockDim.y + threadIdx.y;
    const bool inside = x0 < a.nx && y < a.ny;
    const bool vec = inside && (ODD ? (x0 >= N && x0 + N < a.nx && (!WALLS || (y > 0 && y < a.ny - 1)))
                                    : (x0 + N <= a.nx));
    const unsigned vmask = ODD ? __ballot_sync(0xffffffffu, vec) : 0u;
    if (vec) {
        step_vec<N, MODEL, STORE, ODD, FORCE, SR>(a, x0, y, vmask, threadIdx.x & 31);
    } else if (inside) {
        const int x1 = min(x0 + N, a.nx);
        const unsigned rb = SR ? round_base(a) : 0u;
        for (int x = x0; x < x1; ++x) step_node_split<MODEL, STORE, ODD, FORCE, WALLS, SR>(a, x, y, rb);
    }
}

// CTA of bx x (threads / bx) threads, bx halved (down to 32) while half of it
// still covers the `width` threads a row needs, so narrow lattices leave no
// threads idle.
static inline dim3 fit_block(int bx, int width, int threads = kStepBX * kStepBY) {
    if (bx % 32 != 0 || bx < 32 || bx > threads) bx = kStepBX < threads ? kStepBX : threads;  // lanes of a warp share a row
    while (bx > 32 && bx / 2 >= width) bx /= 2;
    return dim3(bx, threads / bx);
}

template <int N, int MODEL, int STORE, bool ODD, int FORCE, bool WALLS, bool SR>
static cudaError_t launch_vec(const Args& a, cudaStream_t s) {
    const int vecs = (a.nx + N - 1) / N;
    const dim3 block = fit_block(a.block_x > 0 ? a.block_x : kStepBX, vecs, kVecThreads);
    const dim3 grid((vecs + block.x - 1) / block.x, (a.ny + block.y - 1) / block.y);
    step_kernel_vec<N, MODEL, STORE, ODD, FORCE, WALLS, SR><<<grid, block, 0, s>>>(a);
    return cudaGetLastError();
}

template <int MODEL, int STORE, bool ODD, int FORCE, bool WALLS>
static cudaError_t launch_one(const Args& a, cudaStream_t s) {
    if (a.fo) {  // out of place: periodic FP32 / FP64 only
        if constexpr ((STORE == LBM_F32 || STORE == LBM_F64) && !WALLS) {
            const dim3 block = fit_block(a.block_x > 0 ? a.block_x : kStepBX, a.nx);
            const dim3 grid((a.nx + block.x - 1) / block.x, (a.ny + block.y - 1) / block.y);
            if (a.rseed) step_kernel_oop<MODEL, STORE, ODD, FORCE, true><<<grid, block, 0, s>>>(a);
            else step_kernel_oop<MODEL, STORE, ODD, FORCE, false><<<grid, block, 0, s>>>(a);
            return cudaGetLastError();
        }
        return cudaErrorNotSupported;
    }
    if constexpr (STORE == LBM_F32) {
        if (a.rseed) {  // stochastic rounding of FP32 stores: variant 0 only
            const dim3 block = fit_block(a.block_x > 0 ? a.block_x : kStepBX, a.nx);
            const dim3 grid((a.nx + block.x - 1) / block.x, (a.ny + block.y - 1) / block.y);
            step_kernel<MODEL, STORE, ODD, FORCE, WALLS, true><<<grid, block, 0, s>>>(a);
            return cudaGetLastError();
        }
    }
    if constexpr (STORE == LBM_F16DEV || STORE == LBM_BF16DEV) {
        if (a.rseed) {  // stochastic rounding: variants 0 and 2 (variant 1 runs variant 0)
            if constexpr (FORCE != 2) {
                if (a.variant == 2) return launch_vec<4, MODEL, STORE, ODD, FORCE, WALLS, true>(a, s);
            }
            const dim3 block = fit_block(a.block_x > 0 ? a.block_x : kStepBX, a.nx);
            const dim3 grid((a.nx + block.x - 1) / block.x, (a.ny + block.y - 1) / block.y);
            step_kernel<MODEL, STORE, ODD, FORCE, WALLS, true><<<grid, block, 0, s>>>(a);
            return cudaGetLastError();
        }
        if constexpr (FORCE != 2) {
            if (a.variant == 2) return launch_vec<4, MODEL, STORE, ODD, FORCE, WALLS, false>(a, s);
        }
    }
    const dim3 block = fit_block(a.block_x > 0 ? a.block_x : kStepBX, a.nx);
    const int bx = block.x, by = block.y;
    if constexpr (STORE != LBM_F64) {
        if (a.variant == 1) {
            const int rows = (a.ny + 1) / 2;
            const dim3 grid((a.nx + bx - 1) / bx, (rows + by - 1) / by);
            step_kernel_pair<MODEL, STORE, ODD, FORCE, WALLS><<<grid, block, 0, s>>>(a);
            return cudaGetLastError();
        }
    }
    const dim3 grid((a.nx + bx - 1) / bx, (a.ny + by - 1) / by);
    step_kernel<MODEL, STORE, ODD, FORCE, WALLS><<<grid, block, 0, s>>>(a);
    return cudaGetLastError();
}

template <int MODEL, int STORE, bool ODD, int FORCE>
static cudaError_t pick_walls(const Args& a, bool walls, cudaStream_t s) {
    return walls ? launch_one<MODEL, STORE, ODD, FORCE, true>(a, s) : launch_one<MODEL, STORE, ODD, FORCE, false>(a, s);
}

template <int MODEL, int STORE, bool ODD>
static cudaError_t pick_force(const Args& a, int force, bool walls, cudaStream_t s) {
    switch (force) {
        case 0: return pick_walls<MODEL, STORE, ODD, 0>(a, walls, s);
        case 1: return pick_walls<MODEL, STORE, ODD, 1>(a, walls, s);
        default: return pick_walls<MODEL, STORE, ODD, 2>(a, walls, s);
    }
}

template <int MODEL, int STORE>
static cudaError_t pick_parity(const Args& a, bool odd, int force, bool walls, cudaStream_t s) {
    return odd ? pick_force<MODEL, STORE, true>(a, force, walls, s) : pick_force<MODEL, STORE, false>(a, force, walls, s);
}

template <int STORE>
static cudaError_t launch_step_store(const Args& a, int model, bool odd, int force, bool walls, cudaStream_t s) {
    switch (model) {
        case LBM_CASCADED: return pick_parity<LBM_CASCADED, STORE>(a, odd, force, walls, s);
        case LBM_BGK: return pick_parity<LBM_BGK, STORE>(a, odd, force, walls, s);
        default: return pick_parity<LBM_RAWMRT, STORE>(a, odd, force, walls, s);
    }
}

}  // namespace lbm
