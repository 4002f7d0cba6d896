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

struct BatchDomain {
    Args a;
    int store;   // LBM_F32, LBM_BF16DEV or LBM_F16DEV
    int walls;   // any non-periodic edge
    int force;   // 0: none, 1: uniform
    int parity;  // AA parity of the domain's next step when the launch sequence starts
    long long t; // the domain's step count when the launch sequence starts (stochastic rounding)
};

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

// tiles: 3 ints per tile (domain, tile x, tile y); bx = 1 << lbx threads along x;
// a tile is bx x (by rows) nodes and each thread updates `rows` of its rows
// (node rows ly, ly + by, ...), which spreads the tile's decode over more nodes.
template <int MODEL>
__global__ void __launch_bounds__(kBatchThreads) batch_kernel(const BatchDomain* __restrict__ doms,
                                                              const int* __restrict__ tiles, int ntiles, int lbx,
                                                              int rows, int flip, int policy, int* counter,
                                                              const unsigned* __restrict__ rtab, int rstride,
                                                              int kstep) {
    __shared__ int s_next;
    const int bx = 1 << lbx, by = kBatchThreads >> lbx;
    const int lx = threadIdx.x & (bx - 1), ly = threadIdx.x >> lbx;
    int t, end, stride;
    if (policy == kPolicyChunked) {
        t = int((long long)blockIdx.x * ntiles / gridDim.x);
        end = int((long long)(blockIdx.x + 1) * ntiles / gridDim.x);
        stride = 1;
    } else {
        t = blockIdx.x;
        end = ntiles;
        stride = gridDim.x;
    }
    for (;;) {
        if (policy == kPolicyDynamic) {
            if (threadIdx.x == 0) s_next = atomicAdd(counter, 1);
            __syncthreads();
            t = s_next;
            __syncthreads();
        }
        if (t >= end) break;
        const int dom = tiles[3 * t];
        const BatchDomain& D = doms[dom];
        const int x = tiles[3 * t + 1] * bx + lx, y0 = tiles[3 * t + 2] * by * rows + ly;
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
        if (policy != kPolicyDynamic) t += stride;
    }
}

}  // namespace lbm
