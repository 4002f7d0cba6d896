// lbm_batch_impl.cuh -- persistent kernel that advances many independent
// lattices by one time step in a single launch.
//
// The work list is a flat array of tiles (domain, tile x, tile y); a tile is
// the bx x by block of nodes one 256-thread CTA updates.  A resident grid of
// CTAs walks the list under one of three policies (round robin, contiguous
// chunks, or dynamic via an atomic counter); each node runs exactly the same
// step_node body as the single-domain kernel, selected at run time by the
// domain's storage kind, walls, force and AA parity.  No CTA waits on another.
#pragma once

#include "lbm_internal.h"

namespace lbm {

constexpr int kBatchThreads = 256;

enum : int { kPolicyRoundRobin = 0, kPolicyChunked = 1, kPolicyDynamic = 2 };

// 16-byte aligned and a whole number of 16-byte chunks: a CTA copies the
// descriptor of its next tile into shared memory with 16-byte asynchronous
// copies while it updates the current tile.
struct alignas(16) BatchDomain {
    Args a;
    int store;   // LBM_F32, LBM_BF16DEV or LBM_F16DEV
    int walls;   // any non-periodic edge
    int force;   // 0: none, 1: uniform
    int parity;  // AA parity of the domain's next step when the launch sequence starts
    long long t; // the domain's step count when the launch sequence starts (stochastic rounding)
};
static_assert(sizeof(BatchDomain) % 16 == 0, "BatchDomain is copied in 16-byte chunks");
constexpr int kDomChunks = int(sizeof(BatchDomain) / 16);
static_assert(kDomChunks <= 64, "two chunks per lane of one warp");

// One 16-byte global -> shared copy that bypasses the registers (cp.async),
// and the wait for all of this thread's outstanding copies.
__device__ __forceinline__ void copy16_async(void* smem, const void* gmem) {
    const unsigned s = static_cast<unsigned>(__cvta_generic_to_shared(smem));
    asm volatile("cp.async.cg.shared.global [%0], [%1], 16;\n" ::"r"(s), "l"(gmem) : "memory");
}
__device__ __forceinline__ void copy_async_wait_all() {
    asm volatile("cp.async.commit_group;\ncp.async.wait_group 0;\n" ::: "memory");
}

template <int MODEL, int STORE, bool ODD, bool SR>
__device__ __forceinline__ void batch_node_store(const BatchDomain& D, int x, int y, unsigned rb) {
    if (D.walls) {
        if (D.force) step_node_split<MODEL, STORE, ODD, 1, true, SR>(D.a, x, y, rb);
        else step_node_split<MODEL, STORE, ODD, 0, true, SR>(D.a, x, y, rb);
    } else {
        if (D.force) step_node<MODEL, STORE, ODD, 1, false, SR>(D.a, x, y, rb);
        else step_node<MODEL, STORE, ODD, 0, false, SR>(D.a, x, y, rb);
    }
}

// rb: the hash of (seed, step) of a domain with stochastic rounding (D.a.rseed).
template <int MODEL, bool ODD>
__device__ __forceinline__ void batch_node(const BatchDomain& D, int x, int y, unsigned rb) {
    switch (D.store) {
        case LBM_F32:
            if (D.a.rseed) batch_node_store<MODEL, LBM_F32, ODD, true>(D, x, y, rb);
            else batch_node_store<MODEL, LBM_F32, ODD, false>(D, x, y, 0u);
            break;
        case LBM_F16DEV:
            if (D.a.rseed) batch_node_store<MODEL, LBM_F16DEV, ODD, true>(D, x, y, rb);
            else batch_node_store<MODEL, LBM_F16DEV, ODD, false>(D, x, y, 0u);
            break;
        default:
            if (D.a.rseed) batch_node_store<MODEL, LBM_BF16DEV, ODD, true>(D, x, y, rb);
            else batch_node_store<MODEL, LBM_BF16DEV, ODD, false>(D, x, y, 0u);
            break;
    }
}

// Tile index after tile t under the CTA's policy (called by one lane).
__device__ __forceinline__ int next_tile(int t, int stride, int policy, int* counter) {
    return policy == kPolicyDynamic ? atomicAdd(counter, 1) : t + stride;
}

// Warp 0 of the CTA stages tile t (its work-list entry and the domain's
// descriptor) into buffer `buf`: lane 0 reads the entry,
// every lane copies up to two 16-byte chunks of the descriptor with cp.async
// (no registers held while the copies are in flight); the caller waits for
// them (copy_async_wait_all) and then synchronises the CTA.
__device__ __forceinline__ void stage_tile(int t, int end, const BatchDomain* __restrict__ doms,
                                           const int* __restrict__ tiles, BatchDomain* sdom, int (*stile)[4],
                                           int buf, int lane) {
    int dom = 0;
    if (lane == 0) {
        stile[buf][0] = t;
        if (t < end) {
            dom = tiles[3 * t];
            stile[buf][1] = dom;
            stile[buf][2] = tiles[3 * t + 1];
            stile[buf][3] = tiles[3 * t + 2];
        }
    }
    dom = __shfl_sync(0xffffffffu, dom, 0);
    if (__shfl_sync(0xffffffffu, t, 0) >= end) return;
    const char* src = reinterpret_cast<const char*>(doms + dom);
    char* dst = reinterpret_cast<char*>(sdom + buf);
    for (int k = lane; k < kDomChunks; k += 32) copy16_async(dst + 16 * k, src + 16 * k);
}

// tiles: 3 ints per tile (domain, tile x, tile y); bx = 1 << lbx threads along x;
// a tile is bx x (by rows) nodes and each thread updates `rows` of its rows
// (node rows ly, ly + by, ...), which spreads the tile's decode over more nodes.
// The descriptor of the tile being updated sits in shared memory (every
// constant of the update is a shared-memory operand), and warp 0 stages the
// next tile's descriptor into the other buffer while the CTA works, so the
// chain work list -> domain -> descriptor is off the critical path.
template <int MODEL>
__global__ void __launch_bounds__(kBatchThreads) batch_kernel(const BatchDomain* __restrict__ doms,
                                                              const int* __restrict__ tiles, int ntiles, int lbx,
                                                              int rows, int flip, int policy, int* counter,
                                                              const unsigned* __restrict__ rtab, int rstride,
                                                              int kstep) {
    __shared__ BatchDomain sdom[2];
    __shared__ int stile[2][4];  // tile index, domain, tile x, tile y
    const int bx = 1 << lbx, by = kBatchThreads >> lbx;
    const int lx = threadIdx.x & (bx - 1), ly = threadIdx.x >> lbx;
    const int lane = threadIdx.x & 31;
    const bool stager = threadIdx.x < 32;
    int end, stride;
    int first = 0;
    if (policy == kPolicyChunked) {
        first = int((long long)blockIdx.x * ntiles / gridDim.x);
        end = int((long long)(blockIdx.x + 1) * ntiles / gridDim.x);
        stride = 1;
    } else {
        first = blockIdx.x;
        end = ntiles;
        stride = gridDim.x;
    }
    if (stager) {
        int t = first;
        if (policy == kPolicyDynamic && lane == 0) t = atomicAdd(counter, 1);
        t = __shfl_sync(0xffffffffu, t, 0);
        stage_tile(t, end, doms, tiles, sdom, stile, 0, lane);
        copy_async_wait_all();
    }
    __syncthreads();
    for (int cur = 0;; cur ^= 1) {
        const int t = stile[cur][0];
        if (t >= end) break;
        if (stager) {  // stage the next tile into the other buffer
            int tn = 0;
            if (lane == 0) tn = next_tile(t, stride, policy, counter);
            tn = __shfl_sync(0xffffffffu, tn, 0);
            stage_tile(tn, end, doms, tiles, sdom, stile, cur ^ 1, lane);
        }
        const BatchDomain& D = sdom[cur];
        const int dom = stile[cur][1];
        const int x = stile[cur][2] * bx + lx, y0 = stile[cur][3] * by * rows + ly;
        const bool odd = ((D.parity ^ flip) & 1) != 0;
        const unsigned rb = D.a.rseed ? rtab[dom * rstride + kstep] : 0u;
        if (x < D.a.nx) {
            for (int r = 0; r < rows; ++r) {
                const int y = y0 + r * by;
                if (y >= D.a.ny) break;
                if (odd) batch_node<MODEL, true>(D, x, y, rb);
                else batch_node<MODEL, false>(D, x, y, rb);
            }
        }
        if (stager) copy_async_wait_all();
        __syncthreads();  // the next buffer is complete and every thread is done with this one
    }
}

}  // namespace lbm
