// lbm_vec.cuh -- the fused update for four consecutive nodes of a row per
// thread, for the 16-bit deviation stores (FP16, BF16).
//
// With 16-bit populations the one-node-per-thread kernel issues one 16-bit
// load, one 16-bit store and their address arithmetic per population and
// node, and runs out of instruction issue long before HBM bandwidth.  Here a
// thread owns nodes x0 .. x0 + N - 1 (N = 4, x0 a multiple of N) of row y and
// moves each population plane with one 64-bit access where the AA pattern
// keeps the N values aligned:
//
//   even step: every plane is read at x0 .. x0 + N - 1 and written there (own
//              slots), so all nine planes are aligned vector loads and stores;
//   odd step:  node x reads and writes the slots (x + e_p, p) of the nine
//              planes p.  For e_p,x = 0 the N slots are aligned; for
//              e_p,x = +1 (-1) they are shifted by one column: the thread
//              reads its aligned vector and takes the one element past its
//              right (left) end from the neighbouring lane by a warp shuffle,
//              and after the collision hands the one result that falls into
//              the neighbour's vector back the same way, so that every lane
//              stores exactly its own aligned vector.  At warp and row edges
//              the element is loaded and the shifted range stored with narrow
//              stores instead.
//
// Every slot is read and written by the one thread that owns its node, as in
// the scalar kernel (the shuffles only move values between registers).  The
// arithmetic of each node is the scalar kernel's (same collide, same
// round-to-nearest-even conversions), so both kernels produce bit-identical
// states.
//
// Vectors that need a wrapped or wall neighbour (the first and last vector of
// a row and, with walls, the first and last row) and the partial vector at
// the end of a row run the scalar per-node path instead.
#pragma once

#include <cuda_bf16.h>
#include <cuda_fp16.h>
#include <cuda_runtime.h>
#include <stdint.h>

#include "lbm_device.cuh"

namespace lbm {

// Access to 16-bit deviations packed two to a 32-bit word (element 0 in the
// low half, as in memory).
template <int STORE> struct Half16;
template <> struct Half16<LBM_F16DEV> {
    static __device__ __forceinline__ float lo(uint32_t w) {
        return __half2float(__ushort_as_half(static_cast<unsigned short>(w & 0xffffu)));
    }
    static __device__ __forceinline__ float hi(uint32_t w) {
        return __half2float(__ushort_as_half(static_cast<unsigned short>(w >> 16)));
    }
    static __device__ __forceinline__ float one(unsigned short h) { return __half2float(__ushort_as_half(h)); }
    static __device__ __forceinline__ uint32_t pack(float a, float b) {
        const __half2 h = __floats2half2_rn(a, b);  // a in the low half
        return *reinterpret_cast<const uint32_t*>(&h);
    }
    static __device__ __forceinline__ unsigned short enc(float a) { return __half_as_ushort(__float2half_rn(a)); }
};
template <> struct Half16<LBM_BF16DEV> {
    static __device__ __forceinline__ float lo(uint32_t w) { return __uint_as_float(w << 16); }
    static __device__ __forceinline__ float hi(uint32_t w) { return __uint_as_float(w & 0xffff0000u); }
    static __device__ __forceinline__ float one(unsigned short h) { return __uint_as_float(uint32_t(h) << 16); }
    static __device__ __forceinline__ uint32_t pack(float a, float b) {
        const __nv_bfloat162 h = __floats2bfloat162_rn(a, b);  // a in the low half
        return *reinterpret_cast<const uint32_t*>(&h);
    }
    static __device__ __forceinline__ unsigned short enc(float a) { return __bfloat16_as_ushort(__float2bfloat16_rn(a)); }
};

// Element j of an aligned vector held as 32-bit words.
template <int STORE>
__device__ __forceinline__ float vec_elem(const uint32_t* w, int j) {
    return (j & 1) ? Half16<STORE>::hi(w[j >> 1]) : Half16<STORE>::lo(w[j >> 1]);
}

template <int N> struct VecN;
template <> struct VecN<4> {
    static __device__ __forceinline__ void load(const unsigned short* p, uint32_t* w) {
        const uint2 v = *reinterpret_cast<const uint2*>(p);
        w[0] = v.x; w[1] = v.y;
    }
    static __device__ __forceinline__ void store(unsigned short* p, const uint32_t* w) {
        *reinterpret_cast<uint2*>(p) = make_uint2(w[0], w[1]);
    }
};
// Store words w[0 .. k-1] as k 32-bit stores starting at p (4-byte aligned).
template <int K>
__device__ __forceinline__ void store_words(unsigned short* p, const uint32_t* w) {
#pragma unroll
    for (int k = 0; k < K; ++k) *reinterpret_cast<uint32_t*>(p + 2 * k) = w[k];
}

// N nodes (x0 .. x0 + N - 1, y) whose slots need no wrap in x and no
// wall link; x0 is a multiple of N.  On odd steps `vmask` has a bit for every
// lane of the warp that runs this function (the lanes of a warp hold
// consecutive vectors of one row): a lane exchanges the one element of a
// shifted plane that lies in its neighbour's aligned vector with that
// neighbour (warp shuffles), so that each lane loads and stores exactly its
// own aligned vector; a lane whose neighbour is outside `vmask` (warp or row
// edge) loads that element and stores its shifted range with narrow stores.
template <int N, int MODEL, int STORE, bool ODD, int FORCE, bool SR = false>
__device__ __forceinline__ void step_vec(const Args& a, int x0, int y, unsigned vmask, int lane) {
    using H = Half16<STORE>;
    constexpr int W = N / 2;  // words per vector
    unsigned short* __restrict__ f = static_cast<unsigned short*>(a.f);
    const int r0 = y * a.pitch;
    const int rm = (y > 0 ? y - 1 : a.ny - 1) * a.pitch, rp = (y < a.ny - 1 ? y + 1 : 0) * a.pitch;
    const bool left_ok = ODD && lane > 0 && ((vmask >> (lane - 1)) & 1u);
    const bool right_ok = ODD && lane < 31 && ((vmask >> (lane + 1)) & 1u);

    // Region of plane p: columns x0 + s .. x0 + N - 1 + s of its row, s = e_p,x
    // on odd steps and 0 on even ones.  w holds the aligned vector at x0, e the
    // region element outside it.
    uint32_t w[9][W];
    unsigned short e[9];
#pragma unroll
    for (int p = 0; p < 9; ++p) {
        const int row = ODD ? (cy(p) == 1 ? rp : (cy(p) == -1 ? rm : r0)) : r0;
        const unsigned short* base = plane_ptr(a, static_cast<const unsigned short*>(f), p) + row + x0;
        VecN<N>::load(base, w[p]);
    }
#pragma unroll
    for (int p = 0; p < 9; ++p) {
        e[p] = 0;
        if (ODD && cx(p) != 0) {
            const int row = cy(p) == 1 ? rp : (cy(p) == -1 ? rm : r0);
            const unsigned short* base = plane_ptr(a, static_cast<const unsigned short*>(f), p) + row + x0;
            if (cx(p) == 1) {  // column x0 + N: element 0 of the right neighbour's vector
                const uint32_t r = __shfl_down_sync(vmask, w[p][0], 1);
                e[p] = right_ok ? static_cast<unsigned short>(r & 0xffffu) : base[N];
            } else {  // column x0 - 1: element N - 1 of the left neighbour's vector
                const uint32_t r = __shfl_up_sync(vmask, w[p][W - 1], 1);
                e[p] = left_ok ? static_cast<unsigned short>(r >> 16) : base[-1];
            }
        }
    }

    const Coef<float> c(a);
    float Fx, Fy;
    node_force<float, FORCE>(a, x0, y, Fx, Fy);  // uniform force only (FORCE 0 or 1)

    // Outputs: region element i of plane p, packed into words as soon as both
    // halves exist.
    //   s = 0:   words (0,1) (2,3) ...                       -> ow[p][0 .. W-1]
    //   s = +-1: single 0, words (1,2) (3,4) ..., single N-1 -> os0, ow[p][0 .. W-2], os1
    // With stochastic rounding (SR) every value is encoded as soon as it exists,
    // from the offset of its own node and direction (as in store_node).
    float prev[9];
    unsigned short prevh[9];
    uint32_t ow[9][W];
    unsigned short os0[9], os1[9];
    const unsigned rbase = SR ? round_base(a) : 0u;
#pragma unroll
    for (int i = 0; i < N; ++i) {
        float d[9];
#pragma unroll
        for (int q = 0; q < 9; ++q) {
            const int p = ODD ? opp(q) : q;  // plane holding node i's input for direction q
            const int s = ODD ? cx(p) : 0;
            float v;
            if (s == 0) v = vec_elem<STORE>(w[p], i);
            else if (s == 1) v = i < N - 1 ? vec_elem<STORE>(w[p], i + 1) : H::one(e[p]);
            else v = i > 0 ? vec_elem<STORE>(w[p], i - 1) : H::one(e[p]);
            d[q] = v;
        }
        collide<MODEL, float, (FORCE != 0)>(d, Fx, Fy, c);
        const unsigned rn = SR ? round_node(a, rbase, x0 + i, y) : 0u;
#pragma unroll
        for (int q = 0; q < 9; ++q) {
            const int p = ODD ? q : opp(q);  // plane receiving node i's output for direction q
            const int s = ODD ? cx(p) : 0;
            if constexpr (SR) {
                const unsigned short hv = StochasticRound<STORE>::enc(d[q], rn + static_cast<unsigned>(q) * kRoundStride);
                const uint32_t pair = static_cast<uint32_t>(prevh[p]) | (static_cast<uint32_t>(hv) << 16);
                if (s == 0) {
                    if (i & 1) ow[p][i >> 1] = pair;
                } else {
                    if (i == 0) os0[p] = hv;
                    else if (i == N - 1) os1[p] = hv;
                    else if (!(i & 1)) ow[p][(i >> 1) - 1] = pair;
                }
                prevh[p] = hv;
            } else {
                if (s == 0) {
                    if (i & 1) ow[p][i >> 1] = H::pack(prev[p], d[q]);
                } else {
                    if (i == 0) os0[p] = H::enc(d[q]);
                    else if (i == N - 1) os1[p] = H::enc(d[q]);
                    else if (!(i & 1)) ow[p][(i >> 1) - 1] = H::pack(prev[p], d[q]);
                }
                prev[p] = d[q];
            }
        }
    }

#pragma unroll
    for (int p = 0; p < 9; ++p) {
        const int row = ODD ? (cy(p) == 1 ? rp : (cy(p) == -1 ? rm : r0)) : r0;
        unsigned short* base = plane_ptr(a, f, p) + row + x0;
        const int s = ODD ? cx(p) : 0;
        if (s == 0) {
            VecN<N>::store(base, ow[p]);
        } else if (s == 1) {
            // Region x0+1 .. x0+N.  The aligned vector at x0 is the left
            // neighbour's last element followed by region elements 0 .. N-2.
            const uint32_t r = __shfl_up_sync(vmask, static_cast<uint32_t>(os1[p]), 1);
            if (left_ok) {
                uint32_t v[W];
                v[0] = (r & 0xffffu) | (static_cast<uint32_t>(os0[p]) << 16);
#pragma unroll
                for (int k = 1; k < W; ++k) v[k] = ow[p][k - 1];
                VecN<N>::store(base, v);
            } else {
                base[1] = os0[p];
                store_words<W - 1>(base + 2, ow[p]);
            }
            if (!right_ok) base[N] = os1[p];
        } else {
            // Region x0-1 .. x0+N-2.  The aligned vector at x0 is region
            // elements 1 .. N-1 followed by the right neighbour's first element.
            const uint32_t r = __shfl_down_sync(vmask, static_cast<uint32_t>(os0[p]), 1);
            if (right_ok) {
                uint32_t v[W];
#pragma unroll
                for (int k = 0; k < W - 1; ++k) v[k] = ow[p][k];
                v[W - 1] = static_cast<uint32_t>(os1[p]) | (r << 16);
                VecN<N>::store(base, v);
            } else {
                store_words<W - 1>(base, ow[p]);
                base[N - 2] = os1[p];
            }
            if (!left_ok) base[-1] = os0[p];
        }
    }
}

}  // namespace lbm
