// lbm_pair.cuh -- the fused update for two nodes per thread with packed FP32x2
// arithmetic (sm_100+ FFMA2 / FADD2 / FMUL2).
//
// A thread takes nodes (x, y) and (x, y + 1): their loads and stores stay
// per node (coalesced along x, no shuffles), while every arithmetic operation
// of the collision works on both nodes at once.  The value type F2 carries the
// two nodes; a product is kept unevaluated (P2) so that a * b + c becomes one
// packed FMA, as the compiler would contract it for scalars.
#pragma once

#include <cuda_runtime.h>

#include "lbm_device.cuh"

namespace lbm {

struct F2 {
    float2 v;
    F2() = default;
    LBM_HD F2(float2 x) : v(x) {}
    LBM_HD F2(float s) : v(make_float2(s, s)) {}
    LBM_HD F2(double s) : F2(float(s)) {}
    LBM_HD F2(int s) : F2(float(s)) {}
};

__device__ __forceinline__ float2 neg2(float2 x) { return __fmul2_rn(x, make_float2(-1.f, -1.f)); }

struct P2 {  // the product a * b, not yet rounded
    float2 a, b;
    __device__ __forceinline__ operator F2() const { return F2(__fmul2_rn(a, b)); }
};

__device__ __forceinline__ P2 operator*(F2 x, F2 y) { return {x.v, y.v}; }
__device__ __forceinline__ P2 operator*(P2 p, F2 y) { return {F2(p).v, y.v}; }
__device__ __forceinline__ P2 operator*(F2 x, P2 p) { return {x.v, F2(p).v}; }
__device__ __forceinline__ P2 operator*(P2 p, P2 q) { return {F2(p).v, F2(q).v}; }

__device__ __forceinline__ F2 operator+(F2 x, F2 y) { return __fadd2_rn(x.v, y.v); }
__device__ __forceinline__ F2 operator+(P2 p, F2 y) { return __ffma2_rn(p.a, p.b, y.v); }
__device__ __forceinline__ F2 operator+(F2 y, P2 p) { return __ffma2_rn(p.a, p.b, y.v); }
__device__ __forceinline__ F2 operator+(P2 p, P2 q) { return __ffma2_rn(p.a, p.b, F2(q).v); }

// x - y = fma(y, -1, x) is exact in the product, so it rounds once like FSUB.
__device__ __forceinline__ F2 operator-(F2 x, F2 y) { return __ffma2_rn(y.v, make_float2(-1.f, -1.f), x.v); }
__device__ __forceinline__ F2 operator-(P2 p, F2 y) { return __ffma2_rn(p.a, p.b, neg2(y.v)); }
__device__ __forceinline__ F2 operator-(F2 y, P2 p) { return __ffma2_rn(neg2(p.a), p.b, y.v); }
__device__ __forceinline__ F2 operator-(P2 p, P2 q) { return __ffma2_rn(p.a, p.b, neg2(F2(q).v)); }
__device__ __forceinline__ F2 operator-(F2 x) { return neg2(x.v); }
__device__ __forceinline__ P2 operator-(P2 p) { return {neg2(p.a), p.b}; }

__device__ __forceinline__ F2& operator+=(F2& x, F2 y) { return x = x + y; }
__device__ __forceinline__ F2& operator+=(F2& x, P2 p) { return x = x + p; }
__device__ __forceinline__ F2& operator-=(F2& x, F2 y) { return x = x - y; }
__device__ __forceinline__ F2& operator-=(F2& x, P2 p) { return x = x - p; }

__device__ __forceinline__ F2 recip(F2 x) { return F2(make_float2(recip(x.v.x), recip(x.v.y))); }
__device__ __forceinline__ F2 rmul(F2 a, F2 b) { return F2(a * b); }  // rounded product (P2 -> F2)
__device__ __forceinline__ F2 fma_rn(F2 a, F2 b, F2 c) { return F2(__ffma2_rn(a.v, b.v, c.v)); }

template <>
__host__ __device__ inline F2 wgt<F2>(int q) { return F2(wgt<float>(q)); }

// Coefficients of both nodes (the same lattice-wide constants).
__device__ __forceinline__ Coef<F2> pair_coef(const Args& a) {
    const Coef<float> s(a);
    Coef<F2> c;
    c.c3 = s.c3; c.c4 = s.c4; c.c5 = s.c5; c.c6 = s.c6; c.c7 = s.c7; c.c8 = s.c8;
    c.w3 = s.w3; c.w4 = s.w4; c.w5 = s.w5; c.w6 = s.w6; c.w7 = s.w7; c.w8 = s.w8;
    c.rho0 = s.rho0;
    return c;
}

// Nodes (x, y) and (x, y + 1) of an interior or periodic region (no wall
// links); `two` is false when y + 1 is past the last row (its lane is idle).
template <int MODEL, int STORE, bool ODD, int FORCE>
__device__ __forceinline__ void step_pair(const Args& a, int x, int y, bool two) {
    float d0[9], d1[9];
    load_node<STORE, ODD, false>(a, x, y, d0);
    if (two) load_node<STORE, ODD, false>(a, x, y + 1, d1);
    else {
#pragma unroll
        for (int q = 0; q < 9; ++q) d1[q] = d0[q];
    }
    float fx0, fy0, fx1 = 0.f, fy1 = 0.f;
    node_force<float, FORCE>(a, x, y, fx0, fy0);
    if (FORCE != 0) {
        if (two) node_force<float, FORCE>(a, x, y + 1, fx1, fy1);
        else { fx1 = fx0; fy1 = fy0; }
    }
    F2 d[9];
#pragma unroll
    for (int q = 0; q < 9; ++q) d[q] = F2(make_float2(d0[q], d1[q]));
    const Coef<F2> c = pair_coef(a);
    collide<MODEL, F2, (FORCE != 0)>(d, F2(make_float2(fx0, fx1)), F2(make_float2(fy0, fy1)), c);
#pragma unroll
    for (int q = 0; q < 9; ++q) { d0[q] = d[q].v.x; d1[q] = d[q].v.y; }
    store_node<STORE, ODD, false>(a, x, y, d0, 0u);
    if (two) store_node<STORE, ODD, false>(a, x, y + 1, d1, 0u);
}

}  // namespace lbm
