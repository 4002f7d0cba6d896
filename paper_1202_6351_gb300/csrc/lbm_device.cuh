// lbm_device.cuh -- device-side building blocks of the fused D2Q9 update.
//
// Everything here runs per node in registers: the nine populations of a node
// are loaded (AA pattern, see below), collided with the cascaded central-moment
// operator of Sec. II (or a sibling), and stored back.  No tensor cores: the
// per-node map is a handful of signed sums and FMAs, not a dense contraction.
//
// Populations are held as deviations d_a = f_a - w_a rho0 (w = 4/9, 1/9, 1/36),
// so that the O(1) rest state never enters an FP32 subtraction; the moments of
// w_a rho0 are added back analytically (sum w = 1, sum w e_x^2 = 1/3,
// sum w e_x^2 e_y^2 = 1/9, odd moments 0).
//
// AA-pattern streaming on one array f[9][ny][pitch] (Bailey et al. layout):
//   even step: node x reads slot a of x and writes its post-collision a into
//              slot abar of x (no neighbour access);
//   odd step:  node x reads slot abar of x - e_a (the value the neighbour
//              stored there at the even step) and writes post-collision a into
//              slot a of x + e_a.
// Every slot is read and written by one thread only, so the update is in
// place.  After an even number of steps slot a of node x holds f_a(x).
// Half-way bounce-back: a link whose far end lies beyond a wall is reflected
// at the node itself, with the moving-wall term 6 w_a rho_w (e_a . U_wall)
// (Sec. III-C); a diagonal link through the corner point of two walls is
// reflected without it (see incoming_wall).
// The 16-bit stores round to nearest even or, per lattice, stochastically
// (StochasticRound, random offsets from a counter-based hash).  FP32 stores
// can round stochastically too: the collision then forms the last addition of
// Eq. (25) as an error-free sum (two_sum) and the store rounds its exact
// remainder in (round_sr32).
#pragma once

#include <cuda_bf16.h>
#include <cuda_fp16.h>
#include <stdint.h>

#include "lbm.h"

#define LBM_HD __host__ __device__ __forceinline__

namespace lbm {

// ---------------------------------------------------------------- lattice
__host__ __device__ constexpr int cx(int a) { return (a == 1 || a == 5 || a == 8) ? 1 : (a == 3 || a == 6 || a == 7) ? -1 : 0; }
__host__ __device__ constexpr int cy(int a) { return (a == 2 || a == 5 || a == 6) ? 1 : (a == 4 || a == 7 || a == 8) ? -1 : 0; }
__host__ __device__ constexpr int opp(int a) { return a == 0 ? 0 : (a < 5 ? ((a + 1) & 3) + 1 : ((a - 3) & 3) + 5); }
template <typename R>
__host__ __device__ constexpr R wgt(int a) { return a == 0 ? R(4) / R(9) : (a < 5 ? R(1) / R(9) : R(1) / R(36)); }

static_assert(opp(1) == 3 && opp(2) == 4 && opp(3) == 1 && opp(4) == 2, "opposites");
static_assert(opp(5) == 7 && opp(6) == 8 && opp(7) == 5 && opp(8) == 6, "opposites");

// ---------------------------------------------------------------- storage
template <int STORE> struct Store;
// `scale` multiplies the deviation before it is stored.  The step kernels work
// directly in stored units: the collision is homogeneous of degree one in
// (d, rho0, F) at fixed velocity (u = j / rho is scale free), so scaling rho0,
// F and the wall terms by the same factor (prepare_constants) is exact.
template <> struct Store<LBM_F64> {
    using T = double; using R = double;
    static constexpr double scale = 1.0;
    static __device__ __forceinline__ R dec(T v) { return v; }
    static __device__ __forceinline__ T enc(R v) { return v; }
};
template <> struct Store<LBM_F32> {
    using T = float; using R = float;
    static constexpr double scale = 1.0;
    static __device__ __forceinline__ R dec(T v) { return v; }
    static __device__ __forceinline__ T enc(R v) { return v; }
};
template <> struct Store<LBM_BF16DEV> {
    using T = __nv_bfloat16; using R = float;
    static constexpr double scale = 1.0;
    static __device__ __forceinline__ R dec(T v) { return __bfloat162float(v); }
    static __device__ __forceinline__ T enc(R v) { return __float2bfloat16_rn(v); }
};
// FP16 keeps 4096 x deviation: deviations of 1.5e-8 .. 16 stay normal numbers.
template <> struct Store<LBM_F16DEV> {
    using T = __half; using R = float;
    static constexpr double scale = 4096.0;
    static __device__ __forceinline__ R dec(T v) { return __half2float(v); }
    static __device__ __forceinline__ T enc(R v) { return __float2half_rn(v); }
};

inline double store_scale(int store) { return store == LBM_F16DEV ? Store<LBM_F16DEV>::scale : 1.0; }

// Stochastic rounding of a 16-bit store: r is a uniform random 32-bit word.
// Adding its top bits below the kept part of the float's significand and then
// truncating rounds |v| up with probability equal to its distance above the
// representable value below, in units of their spacing, so the stored value is
// an unbiased estimate of v: increments far smaller than the spacing survive on
// average, where round to nearest would drop them every step.
template <int STORE> struct StochasticRound;
template <> struct StochasticRound<LBM_F16DEV> {  // FP16 keeps 10 of the float's 23 fraction bits
    static __device__ __forceinline__ unsigned short enc(float v, unsigned r) {
        return __half_as_ushort(__float2half_rz(__uint_as_float(__float_as_uint(v) + (r >> 19))));
    }
};
template <> struct StochasticRound<LBM_BF16DEV> {  // BF16 keeps 7
    static __device__ __forceinline__ unsigned short enc(float v, unsigned r) {
        return static_cast<unsigned short>((__float_as_uint(v) + (r >> 16)) >> 16);
    }
};
template <int STORE>
__device__ __forceinline__ typename Store<STORE>::T enc_sr(typename Store<STORE>::R v, unsigned r) {
    if constexpr (STORE == LBM_F16DEV) return __ushort_as_half(StochasticRound<STORE>::enc(v, r));
    else if constexpr (STORE == LBM_BF16DEV) return __ushort_as_bfloat16(StochasticRound<STORE>::enc(v, r));
    else return Store<STORE>::enc(v);
}

// Error-free sum (Knuth's TwoSum): s = fl(a + b) and err with a + b = s + err
// exactly, for round-to-nearest FP32 without overflow.  The intrinsics keep
// the compiler from contracting or reassociating the operations.
LBM_HD float two_sum(float a, float b, float& err) {
#ifdef __CUDA_ARCH__
    const float s = __fadd_rn(a, b);
    const float bb = __fsub_rn(s, a);
    err = __fadd_rn(__fsub_rn(a, __fsub_rn(s, bb)), __fsub_rn(b, bb));
#else
    volatile float vs = a + b;
    const float s = vs;
    volatile float vbb = s - a;
    const float bb = vbb;
    err = (a - (s - bb)) + (b - bb);
#endif
    return s;
}

// Stochastic rounding of an FP32 value known exactly as s + e (s = fl(s + e)):
// s moves to its neighbour on the side of e with probability |e| / gap, gap
// the distance to that neighbour, so the stored value is an unbiased estimate
// of s + e.  r is a uniform random 32-bit word; its top 24 bits give
// u = k 2^-24 and u * gap is exact (gap is a power of two).  s = 0 implies
// e = 0 (a sum that rounds to zero is exact with gradual underflow), so the
// neighbour of +-0 is never taken.
__device__ __forceinline__ float round_sr32(float s, float e, unsigned r) {
    const unsigned bits = __float_as_uint(s);
    const bool away = (e > 0.f) == (s > 0.f);  // magnitude grows
    const float nb = __uint_as_float(away ? bits + 1u : bits - 1u);
    const float gap = fabsf(nb - s);
    const float u = __uint2float_rz(r >> 8) * 0x1p-24f;
    return fabsf(e) > u * gap ? nb : s;
}

// ---------------------------------------------------------------- launch arguments
// Plain-old-data, passed by value to every kernel.
// Index of the per-launch constants in Args::kf / Args::kd.
enum : int { K_C3 = 0, K_W3 = 6, K_RHO0 = 12, K_FX = 13, K_FY = 14, K_SCALE = 15, K_COUNT = 16 };
// Slot of the wall-term arrays used by a link that enters through a corner
// where two walls meet: it is bounced back with no wall-motion term.
enum : int { kCorner = 4 };

struct Args {
    void* f;                  // populations [9][ny][pitch] of the stored type
    void* fo;                 // where an out-of-place step stores its result (null: f, in place).
                              // Every slot is read and written by one thread, so a step from f into a
                              // second array of the same layout needs no other change (the adjoint
                              // recomputes its checkpoint segments this way instead of copying); only
                              // the kernels instantiated with OOP read it
    long long plane;          // pitch * ny
    int nx, ny, pitch;
    int wall[4];              // 1 if the edge (W, E, S, N) is a wall
    double wallx[5], wally[5];// 6 rho_w U_wall (x, y components) per edge; [kCorner] = 0
    double om[6];             // omega_3 .. omega_8
    double F[2];              // uniform body force
    const void* ffield;       // per-node force [2][ny][nx] (Real), or null
    double rho0;
    double scale;             // storage scale of the deviations (Store<>::scale)
    int variant;              // 0: one node per thread; 1: two rows per thread, packed FP32x2 (FP32 arithmetic);
                              // 2: four nodes per thread (16-bit); 3: two steps per launch (lbm_fused.cuh)
    int block_x;              // CTA width of the step kernels (CTA height = 256 / block_x); 0 means 128
    // The constants the step kernels use, converted once on the host into both
    // arithmetic types (GB300's FP64 rate is far too low for per-thread
    // conversions or divisions): omega_3/12, omega_4/4 .. omega_8/4 (Eq. 17-22),
    // omega_3 .. omega_8, and rho0, F_x, F_y and the wall terms in stored units.
    float kf[K_COUNT];
    double kd[K_COUNT];
    float wallxf[5], wallyf[5];
    // Stochastic rounding of the 16-bit stores (rseed != 0): the hash C0 of
    // (seed, step) for this launch is rbase, or rtable[tstep] for a launch
    // replayed from a CUDA graph (the table is filled before each replay).
    unsigned long long rseed;
    const unsigned* rtable;
    unsigned rbase;
    int tstep;
    unsigned rbase1;          // C0 of the second step of a two-step launch (rtable[tstep + 1] in a replay)
};

// Fill Args::kf, kd, wallxf, wallyf from om, rho0, F, wallx, wally (and zero
// the corner slot).
inline void prepare_constants(Args& a) {
    a.wallx[kCorner] = 0.0;
    a.wally[kCorner] = 0.0;
    a.kd[K_C3] = a.om[0] / 12.0;
    for (int k = 1; k < 6; ++k) a.kd[K_C3 + k] = a.om[k] / 4.0;
    for (int k = 0; k < 6; ++k) a.kd[K_W3 + k] = a.om[k];
    a.kd[K_RHO0] = a.rho0 * a.scale;
    a.kd[K_FX] = a.F[0] * a.scale;
    a.kd[K_FY] = a.F[1] * a.scale;
    a.kd[K_SCALE] = a.scale;
    for (int k = 0; k < K_COUNT; ++k) a.kf[k] = float(a.kd[k]);
    for (int k = 0; k < 5; ++k) {
        a.wallxf[k] = float(a.wallx[k] * a.scale);
        a.wallyf[k] = float(a.wally[k] * a.scale);
    }
}

template <typename R> __device__ __forceinline__ const R* kconst(const Args& a);
template <> __device__ __forceinline__ const float* kconst<float>(const Args& a) { return a.kf; }
template <> __device__ __forceinline__ const double* kconst<double>(const Args& a) { return a.kd; }

// Relaxation constants in the arithmetic type.
template <typename R>
struct Coef {
    R c3, c4, c5, c6, c7, c8;  // omega_3/12, omega_4/4, ..., omega_8/4 (Eq. 17-22)
    R w3, w4, w5, w6, w7, w8;  // the rates themselves (MRT, BGK)
    R rho0;
    LBM_HD Coef() {}
    // From a constants array laid out as Args::kf / Args::kd.
    LBM_HD explicit Coef(const R* k) {
        c3 = k[K_C3]; c4 = k[K_C3 + 1]; c5 = k[K_C3 + 2]; c6 = k[K_C3 + 3]; c7 = k[K_C3 + 4]; c8 = k[K_C3 + 5];
        w3 = k[K_W3]; w4 = k[K_W3 + 1]; w5 = k[K_W3 + 2]; w6 = k[K_W3 + 3]; w7 = k[K_W3 + 4]; w8 = k[K_W3 + 5];
        rho0 = k[K_RHO0];
    }
    __device__ __forceinline__ explicit Coef(const Args& a) : Coef(kconst<R>(a)) {}
};

// ---------------------------------------------------------------- walls
// Wall through which the link arriving at (x, y) in direction q comes from
// outside the lattice, or -1.  A diagonal link whose path crosses the corner
// point of two walls belongs to neither: it returns kCorner (plain bounce-back,
// no wall-motion term).  With the lid term on that link instead, the
// lid-driven cavity of Sec. III-C converges at first order only; without it,
// at the second order the paper reports there.
__device__ __forceinline__ int incoming_wall(const Args& a, int q, int x, int y) {
    int wy = -1, wx = -1;
    if (cy(q) == 1 && y == 0 && a.wall[LBM_SOUTH]) wy = LBM_SOUTH;
    if (cy(q) == -1 && y == a.ny - 1 && a.wall[LBM_NORTH]) wy = LBM_NORTH;
    if (cx(q) == 1 && x == 0 && a.wall[LBM_WEST]) wx = LBM_WEST;
    if (cx(q) == -1 && x == a.nx - 1 && a.wall[LBM_EAST]) wx = LBM_EAST;
    return wy >= 0 ? (wx >= 0 ? int(kCorner) : wy) : wx;
}
// Moving-wall term for a population entering in direction q through wall w.
// The product is rounded on its own (never fused into an FMA with a later
// addition), so every kernel that adds the term rounds it alike.
template <typename R>
__device__ __forceinline__ R wall_term(const Args& a, int q, int w) {
    if constexpr (sizeof(R) == 4) return __fmul_rn(wgt<R>(q), R(cx(q)) * a.wallxf[w] + R(cy(q)) * a.wallyf[w]);
    else return __dmul_rn(wgt<R>(q), R(cx(q)) * a.wallx[w] + R(cy(q)) * a.wally[w]);  // FP64 storage: scale 1
}
// v + wall_term, one rounded addition (the moving-wall link of Sec. III-C).
template <typename R>
__device__ __forceinline__ R add_wall_term(const Args& a, R v, int q, int w) {
    if constexpr (sizeof(R) == 4) return __fadd_rn(v, wall_term<R>(a, q, w));
    else return __dadd_rn(v, wall_term<R>(a, q, w));
}

// ---------------------------------------------------------------- AA access
// Offsets inside one population plane are 32-bit (pitch * ny < 2^31 is checked
// at creation); the plane base f + q * plane is the same for every thread.
template <typename T>
__device__ __forceinline__ const T* plane_ptr(const Args& a, const T* f, int q) { return f + q * a.plane; }
template <typename T>
__device__ __forceinline__ T* plane_ptr(const Args& a, T* f, int q) { return f + q * a.plane; }

// Load the nine pre-collision deviations of node (x, y), in stored units.
// ODD selects the parity of the step about to be taken (see the header comment).
template <int STORE, bool ODD, bool WALLS>
__device__ __forceinline__ void load_node(const Args& a, int x, int y, typename Store<STORE>::R d[9]) {
    using S = Store<STORE>;
    using T = typename S::T;
    using R = typename S::R;
    const T* __restrict__ f = static_cast<const T*>(a.f);
    const int n = y * a.pitch + x;
    if (!ODD) {
#pragma unroll
        for (int q = 0; q < 9; ++q) d[q] = S::dec(plane_ptr(a, f, q)[n]);
    } else {
        const int xm = x > 0 ? x - 1 : a.nx - 1, xp = x < a.nx - 1 ? x + 1 : 0;
        const int rm = (y > 0 ? y - 1 : a.ny - 1) * a.pitch, rp = (y < a.ny - 1 ? y + 1 : 0) * a.pitch;
        const int r0 = y * a.pitch;
#pragma unroll
        for (int q = 0; q < 9; ++q) {
            int w = -1;
            if (WALLS) w = incoming_wall(a, q, x, y);
            if (w >= 0) {
                d[q] = add_wall_term<R>(a, S::dec(plane_ptr(a, f, q)[n]), q, w);
            } else {
                const int sx = cx(q) == 1 ? xm : (cx(q) == -1 ? xp : x);
                const int sr = cy(q) == 1 ? rm : (cy(q) == -1 ? rp : r0);
                d[q] = S::dec(plane_ptr(a, f, opp(q))[sr + sx]);
            }
        }
    }
}

// ---------------------------------------------------------------- random offsets
// The offset for population q of node n (n = y nx + x) at a step is
// mix(C0 + 9 n C1) + q C1 (mod 2^32), whose top bits serve the rounding: C0 is an
// integer hash of (seed, step) and mix the "lowbias32" mixer of C. Wellons, so
// over the steps the offset of each value is uniform and independent of the
// value and of the other nodes' offsets; C1 is odd.  Without the per-node mix
// (offsets C0 + (9 n + q) C1, correlated between neighbouring nodes) a long
// FP16 Taylor-Green run on 1024^2 still lost 0.3 % of its amplitude in one decay
// time (BF16: 2.6 %); with it, 0.01 % and 0.05 %, as with a hash per value.
constexpr unsigned kRoundStride = 0x9e3779b9u;
LBM_HD unsigned mix32(unsigned x) {
    x ^= x >> 16;
    x *= 0x7feb352du;
    x ^= x >> 15;
    x *= 0x846ca68bu;
    x ^= x >> 16;
    return x;
}
// C0 for step t (computed on the host per launch, or by fill_round_table).
LBM_HD unsigned round_hash(unsigned long long seed, unsigned long long t) {
    return mix32(static_cast<unsigned>(seed) ^
                 mix32(static_cast<unsigned>(t) ^ mix32(static_cast<unsigned>(t >> 32) ^ static_cast<unsigned>(seed >> 32))));
}
__device__ __forceinline__ unsigned round_base(const Args& a) { return a.rtable ? a.rtable[a.tstep] : a.rbase; }
// mix(C0 + 9 n C1) for node (x, y); add q C1 for population q.
__device__ __forceinline__ unsigned round_node(const Args& a, unsigned base, int x, int y) {
    return mix32(base + 9u * static_cast<unsigned>(y * a.nx + x) * kRoundStride);
}

// Store the nine post-collision deviations of node (x, y).
// rb: the hash C0 of this launch's (seed, step) when SR (stochastic rounding).
// For FP32 storage with SR, err[q] is the exact remainder of d[q] (the
// collision's two_sum), which round_sr32 rounds in.
template <int STORE, bool ODD, bool WALLS, bool SR = false, bool OOP = false>
__device__ __forceinline__ void store_node(const Args& a, int x, int y, const typename Store<STORE>::R d[9],
                                           unsigned rb, const typename Store<STORE>::R* err = nullptr) {
    using S = Store<STORE>;
    using T = typename S::T;
    using R = typename S::R;
    constexpr bool SR32 = SR && STORE == LBM_F32;
    T* __restrict__ f = static_cast<T*>(OOP ? a.fo : a.f);
    const int n = y * a.pitch + x;
    const unsigned rn = SR ? round_node(a, rb, x, y) : 0u;
    auto put = [&](R v, R e, int q) -> T {
        const unsigned r = rn + static_cast<unsigned>(q) * kRoundStride;
        if constexpr (SR32) return round_sr32(v, e, r);
        else return SR ? enc_sr<STORE>(v, r) : S::enc(v);
    };
    auto enc = [&](R v, int q) -> T { return put(v, SR32 ? err[q] : R(0), q); };
    if (!ODD) {
#pragma unroll
        for (int q = 0; q < 9; ++q) plane_ptr(a, f, opp(q))[n] = enc(d[q], q);
    } else {
        const int xm = x > 0 ? x - 1 : a.nx - 1, xp = x < a.nx - 1 ? x + 1 : 0;
        const int rm = (y > 0 ? y - 1 : a.ny - 1) * a.pitch, rp = (y < a.ny - 1 ? y + 1 : 0) * a.pitch;
        const int r0 = y * a.pitch;
#pragma unroll
        for (int q = 0; q < 9; ++q) {
            int w = -1;
            if (WALLS) w = incoming_wall(a, opp(q), x, y);
            if (w >= 0) {
                if constexpr (SR32) {
                    float e2;
                    const float v = two_sum(d[q], wall_term<R>(a, opp(q), w), e2);
                    plane_ptr(a, f, opp(q))[n] = put(v, err[q] + e2, q);
                } else {
                    plane_ptr(a, f, opp(q))[n] = enc(add_wall_term<R>(a, d[q], opp(q), w), q);
                }
            } else {
                const int tx = cx(q) == 1 ? xp : (cx(q) == -1 ? xm : x);
                const int tr = cy(q) == 1 ? rp : (cy(q) == -1 ? rm : r0);
                plane_ptr(a, f, q)[tr + tx] = enc(d[q], q);
            }
        }
    }
}

// ---------------------------------------------------------------- per-node force
template <typename R, int FORCE>
__device__ __forceinline__ void node_force(const Args& a, int x, int y, R& Fx, R& Fy) {
    if (FORCE == 0) { Fx = R(0); Fy = R(0); return; }
    const R* k = kconst<R>(a);
    Fx = k[K_FX]; Fy = k[K_FY];
    if (FORCE == 2) {  // the field is kept in physical units
        const R* ff = static_cast<const R*>(a.ffield);
        const int n = y * a.nx + x;
        Fx += k[K_SCALE] * ff[n];
        Fy += k[K_SCALE] * ff[a.nx * a.ny + n];
    }
}

// ---------------------------------------------------------------- rounded products
// Which product of a sum of two products the compiler fuses into an FMA, and
// whether it fuses a product that has several uses, depends on the code
// around the inlined collision.  So wherever a sum has two inexact products,
// or a product has several uses, the collisions spell the operations out:
// rmul (a product rounded on its own) and fma_rn (one fused multiply-add).
// Every kernel variant then rounds every node alike.
LBM_HD float rmul(float a, float b) {
#ifdef __CUDA_ARCH__
    return __fmul_rn(a, b);
#else
    volatile float p = a * b;
    return p;
#endif
}
LBM_HD double rmul(double a, double b) {
#ifdef __CUDA_ARCH__
    return __dmul_rn(a, b);
#else
    volatile double p = a * b;
    return p;
#endif
}

// a * b + c as one fused multiply-add in every kernel (not left to the
// compiler's choice of which of two products to fuse into a sum).
LBM_HD float fma_rn(float a, float b, float c) {
#ifdef __CUDA_ARCH__
    return __fmaf_rn(a, b, c);
#else
    return fmaf(a, b, c);
#endif
}
LBM_HD double fma_rn(double a, double b, double c) {
#ifdef __CUDA_ARCH__
    return __fma_rn(a, b, c);
#else
    return fma(a, b, c);
#endif
}

// ---------------------------------------------------------------- moments
template <typename R>
struct Moments {
    R drho, rho, jx, jy;           // sum d, rho0 + drho, sum d e (momentum of f_bar)
    R kxx, kyy, kxy, kxxy, kxyy, kxxyy;  // raw moments of d (Eq. 15 without the rho0 w part)
};

// 1/rho: IEEE division in FP64; in FP32 the hardware reciprocal (rcp.approx,
// relative error below 2^-22), far below the FP32 storage rounding of d.
LBM_HD double recip(double x) { return 1.0 / x; }
LBM_HD float recip(float x) {
#ifdef __CUDA_ARCH__
    float r;
    asm("rcp.approx.ftz.f32 %0, %1;" : "=f"(r) : "f"(x));
    return r;
#else
    return 1.0f / x;
#endif
}

template <typename R>
LBM_HD Moments<R> moments(const R d[9], R rho0) {
    Moments<R> m;
    const R s13 = d[1] + d[3], s24 = d[2] + d[4];
    const R s56 = d[5] + d[6], s78 = d[7] + d[8];
    const R s58 = d[5] + d[8], s67 = d[6] + d[7];
    m.kxxyy = s56 + s78;
    m.kxx = s13 + m.kxxyy;
    m.kyy = s24 + m.kxxyy;
    m.drho = d[0] + s13 + m.kyy;
    m.rho = rho0 + m.drho;
    m.jx = (d[1] - d[3]) + (s58 - s67);
    m.jy = (d[2] - d[4]) + (s56 - s78);
    m.kxy = (d[5] + d[7]) - (d[6] + d[8]);
    m.kxxy = s56 - s78;
    m.kxyy = s58 - s67;
    return m;
}

// Source S_a (Eq. 14 with the m^s list before it) for force (Fx, Fy) at velocity (ux, uy).
template <typename R>
LBM_HD void source(R ux, R uy, R Fx, R Fy, R S[9]) {
    const R m1 = Fx, m2 = Fy;
    const R fxux = rmul(Fx, ux), fyuy = rmul(Fy, uy), fxuy = rmul(Fx, uy), fyux = rmul(Fy, ux);
    const R uxx = rmul(ux, ux), uyy = rmul(uy, uy);
    const R m3 = R(6) * (fxux + fyuy);
    const R m4 = R(2) * (fxux - fyuy);
    const R m5 = fxuy + fyux;
    const R m6 = fma_rn(fma_rn(R(-3), uxx, R(2)), Fy, R(-6) * rmul(fxux, uy));
    const R m7 = fma_rn(fma_rn(R(-3), uyy, R(2)), Fx, R(-6) * rmul(fyuy, ux));
    const R m8 = R(6) * fma_rn(fma_rn(R(3), uyy, R(-2)), fxux, rmul(fma_rn(R(3), uxx, R(-2)), fyuy));
    const R k = R(1.0 / 36.0);
    S[0] = k * (R(4) * (m8 - m3));
    S[1] = k * (R(6) * m1 - m3 + R(9) * m4 + R(6) * m7 - R(2) * m8);
    S[2] = k * (R(6) * m2 - m3 - R(9) * m4 + R(6) * m6 - R(2) * m8);
    S[3] = k * (-R(6) * m1 - m3 + R(9) * m4 - R(6) * m7 - R(2) * m8);
    S[4] = k * (-R(6) * m2 - m3 - R(9) * m4 - R(6) * m6 - R(2) * m8);
    S[5] = k * (fma_rn(R(6), m1 + m2, R(2) * m3) + R(9) * m5 - R(3) * (m6 + m7) + m8);
    S[6] = k * (fma_rn(R(6), m2 - m1, R(2) * m3) - R(9) * m5 - R(3) * (m6 - m7) + m8);
    S[7] = k * (fma_rn(R(-6), m1 + m2, R(2) * m3) + R(9) * m5 + R(3) * (m6 + m7) + m8);
    S[8] = k * (fma_rn(R(6), m1 - m2, R(2) * m3) - R(9) * m5 + R(3) * (m6 - m7) + m8);
}

// Add K . g (Eq. 25; g0 = g1 = g2 = 0) to d.
template <typename R>
LBM_HD void add_kernel(R d[9], R g3, R g4, R g5, R g6, R g7, R g8) {
    const R t = R(2) * g3 + g8;
    const R a = g4 - g3;             // f1, f3 share -g3 + g4
    const R b = -g3 - g4;            // f2, f4 share -g3 - g4
    d[0] += R(4) * (g8 - g3);
    d[1] += a + R(2) * (g7 - g8);
    d[3] += a - R(2) * (g7 + g8);
    d[2] += b + R(2) * (g6 - g8);
    d[4] += b - R(2) * (g6 + g8);
    const R p = g5 - g6, q = g5 + g6;
    d[5] += t + p - g7;
    d[6] += t - q + g7;
    d[7] += t + q + g7;
    d[8] += t - p - g7;
}

// The increments K . g of add_kernel as separate values (the error-free path).
template <typename R>
LBM_HD void kernel_increments(R inc[9], R g3, R g4, R g5, R g6, R g7, R g8) {
    const R t = R(2) * g3 + g8;
    const R a = g4 - g3, b = -g3 - g4;
    const R p = g5 - g6, q = g5 + g6;
    inc[0] = R(4) * (g8 - g3);
    inc[1] = a + R(2) * (g7 - g8);
    inc[3] = a - R(2) * (g7 + g8);
    inc[2] = b + R(2) * (g6 - g8);
    inc[4] = b - R(2) * (g6 + g8);
    inc[5] = t + p - g7;
    inc[6] = t - q + g7;
    inc[7] = t + q + g7;
    inc[8] = t - p - g7;
}

// d += inc, with each sum's exact remainder in err when TS (FP32 only).
template <typename R, bool TS>
LBM_HD void add_increments(R d[9], const R inc[9], R* err) {
#pragma unroll
    for (int q = 0; q < 9; ++q) {
        if constexpr (TS) d[q] = two_sum(d[q], inc[q], err[q]);
        else d[q] += inc[q];
    }
}

// ---------------------------------------------------------------- cascaded collision
// Sec. II, Eq. (13)-(25), on deviations.  FORCE = 0: no source terms.
// TS (FP32 with stochastic rounding of the store): the post-collision value
// d + (K g + S) is formed by one error-free sum whose remainder goes to err.
template <typename R, bool FORCED, bool TS = false>
LBM_HD void collide_cascaded(R d[9], R Fx, R Fy, const Coef<R>& c, R* err = nullptr) {
    const Moments<R> m = moments(d, c.rho0);
    const R inv = recip(m.rho);
    const R ux = (FORCED ? m.jx + R(0.5) * Fx : m.jx) * inv;   // Eq. (27)
    const R uy = (FORCED ? m.jy + R(0.5) * Fy : m.jy) * inv;
    const R uxx = rmul(ux, ux), uyy = rmul(uy, uy), uxy = rmul(ux, uy);
    const R r3 = rmul(c.rho0, R(1.0 / 3.0));
    // raw source moments, Eq. (13)
    R sxx = 0, syy = 0, sxy = 0, sxxy = 0, sxyy = 0, sxxyy = 0;
    if (FORCED) {
        const R fxuy = rmul(Fx, uy), fyux = rmul(Fy, ux);
        sxx = R(2) * Fx * ux; syy = R(2) * Fy * uy; sxy = fxuy + fyux;
        sxxy = fma_rn(Fy, uxx, R(2) * Fx * uxy); sxyy = fma_rn(Fx, uyy, R(2) * Fy * uxy);
        sxxyy = R(2) * uxy * (fxuy + fyux);
    }
    const R kxx_t = r3 + m.kxx, kyy_t = r3 + m.kyy;  // full kappa'_xx, kappa'_yy
    // Eq. (17)-(19)
    const R g3 = rmul(c.c3, fma_rn(m.rho, uxx + uyy, R(2.0 / 3.0) * m.drho) - (m.kxx + m.kyy) - R(0.5) * (sxx + syy));
    const R g4 = rmul(c.c4, m.rho * (uxx - uyy) - (m.kxx - m.kyy) - R(0.5) * (sxx - syy));
    const R g5 = rmul(c.c5, m.rho * uxy - m.kxy - R(0.5) * sxy);
    const R A = R(3) * g3 + g4, B = R(3) * g3 - g4;
    // Eq. (20)-(21)
    const R g6 = fma_rn(c.c6, R(2) * m.rho * uxx * uy + m.kxxy - R(2) * ux * m.kxy - uy * kxx_t - R(0.5) * sxxy,
                        R(-0.5) * uy * A) - R(2) * ux * g5;
    const R g7 = fma_rn(c.c7, R(2) * m.rho * ux * uyy + m.kxyy - R(2) * uy * m.kxy - ux * kyy_t - R(0.5) * sxyy,
                        R(-0.5) * ux * B) - R(2) * uy * g5;
    // Eq. (22)
    const R G8 = R(1.0 / 9.0) * m.drho - m.kxxyy + R(3) * m.rho * uxx * uyy
               + R(2) * fma_rn(ux, m.kxyy, rmul(uy, m.kxxy)) - uxx * kyy_t - uyy * kxx_t
               - R(4) * uxy * m.kxy - R(0.5) * sxxyy;
    const R g8 = fma_rn(c.c8, G8, R(-2) * g3) - R(0.5) * fma_rn(uyy, A, rmul(uxx, B)) - R(4) * uxy * g5
               - R(2) * fma_rn(uy, g6, rmul(ux, g7));
    if constexpr (TS) {
        R inc[9];
        kernel_increments(inc, g3, g4, g5, g6, g7, g8);
        if (FORCED) {
            R S[9];
            source(ux, uy, Fx, Fy, S);
#pragma unroll
            for (int q = 0; q < 9; ++q) inc[q] += S[q];
        }
        add_increments<R, true>(d, inc, err);
        return;
    }
    add_kernel(d, g3, g4, g5, g6, g7, g8);
    if (FORCED) {
        R S[9];
        source(ux, uy, Fx, Fy, S);
#pragma unroll
        for (int q = 0; q < 9; ++q) d[q] += S[q];
    }
}

// ---------------------------------------------------------------- SRT-BGK sibling
// d~ = d - w (d - d_eq) + (1 - w/2) S with the 2nd-order polynomial f_eq and w = omega_4.
template <typename R, bool FORCED, bool TS = false>
LBM_HD void collide_bgk(R d[9], R Fx, R Fy, const Coef<R>& c, R* err = nullptr) {
    const Moments<R> m = moments(d, c.rho0);
    const R inv = recip(m.rho);
    const R ux = (FORCED ? m.jx + R(0.5) * Fx : m.jx) * inv;
    const R uy = (FORCED ? m.jy + R(0.5) * Fy : m.jy) * inv;
    const R usq = R(1.5) * (rmul(ux, ux) + rmul(uy, uy));
    const R w = c.w4;
    R S[9];
    if (FORCED) source(ux, uy, Fx, Fy, S);
#pragma unroll
    for (int q = 0; q < 9; ++q) {
        const R eu = R(cx(q)) * ux + R(cy(q)) * uy;
        const R deq = wgt<R>(q) * (m.drho + m.rho * (fma_rn(R(4.5) * eu, eu, R(3) * eu) - usq));
        if constexpr (TS) {
            R inc = -w * (d[q] - deq);
            if (FORCED) inc += (R(1) - R(0.5) * w) * S[q];
            d[q] = two_sum(d[q], inc, err[q]);
        } else {
            d[q] = d[q] - w * (d[q] - deq);
            if (FORCED) d[q] += (R(1) - R(0.5) * w) * S[q];
        }
    }
}

// ---------------------------------------------------------------- raw-moment MRT sibling
// f~ = f - K D^-1 [L (m - m_eq) - (I - L/2) m_s], L = diag(0,0,0,omega_3..omega_8),
// basis K of Eq. (3), polynomial equilibrium moments m_eq in closed form.
template <typename R, bool FORCED, bool TS = false>
LBM_HD void collide_rawmrt(R d[9], R Fx, R Fy, const Coef<R>& c, R* err = nullptr) {
    const Moments<R> m = moments(d, c.rho0);
    const R inv = recip(m.rho);
    const R ux = (FORCED ? m.jx + R(0.5) * Fx : m.jx) * inv;
    const R uy = (FORCED ? m.jy + R(0.5) * Fy : m.jy) * inv;
    const R uxx = rmul(ux, ux), uyy = rmul(uy, uy), usq = uxx + uyy;
    // orthogonal moments of d (the rest-state part w rho0 is added to m_eq's side)
    const R tr = m.kxx + m.kyy;
    const R m3 = fma_rn(R(3), tr, R(-4) * m.drho);
    const R m4 = m.kxx - m.kyy;
    const R m5 = m.kxy;
    const R m6 = fma_rn(R(-3), m.kxxy, R(2) * m.jy);
    const R m7 = fma_rn(R(-3), m.kxyy, R(2) * m.jx);
    const R m8 = fma_rn(R(9), m.kxxyy, fma_rn(R(-6), tr, R(4) * m.drho));
    // equilibrium moments of f_eq - w rho0
    const R p3 = rmul(R(3) * m.rho, usq);  // shared by e3 and e8
    const R e3 = p3 - R(2) * m.drho;
    const R e4 = m.rho * (uxx - uyy);
    const R e5 = m.rho * ux * uy;
    const R e6 = m.rho * uy;
    const R e7 = m.rho * ux;
    const R e8 = m.drho - p3;
    R s3 = 0, s4 = 0, s5 = 0, s6 = 0, s7 = 0, s8 = 0;
    if (FORCED) {  // the m^s list before Eq. (14)
        const R fxux = rmul(Fx, ux), fyuy = rmul(Fy, uy), fxuy = rmul(Fx, uy), fyux = rmul(Fy, ux);
        s3 = R(6) * (fxux + fyuy); s4 = R(2) * (fxux - fyuy); s5 = fxuy + fyux;
        s6 = fma_rn(fma_rn(R(-3), uxx, R(2)), Fy, R(-6) * rmul(fxux, uy));
        s7 = fma_rn(fma_rn(R(-3), uyy, R(2)), Fx, R(-6) * rmul(fyuy, ux));
        s8 = R(6) * fma_rn(fma_rn(R(3), uyy, R(-2)), fxux, rmul(fma_rn(R(3), uxx, R(-2)), fyuy));
    }
    // change of each orthogonal moment divided by its norm D_b
    // -w (m - m_eq) + (1 - w/2) m_s: the source product rounded on its own, the
    // relaxation product fused into the sum
    auto relax = [](R w, R dm, R sm) { return fma_rn(-w, dm, rmul(R(1) - R(0.5) * w, sm)); };
    const R g3 = rmul(relax(c.w3, m3 - e3, s3), R(1.0 / 36.0));
    const R g4 = relax(c.w4, m4 - e4, s4) * R(0.25);
    const R g5 = relax(c.w5, m5 - e5, s5) * R(0.25);
    const R g6 = rmul(relax(c.w6, m6 - e6, s6), R(1.0 / 12.0));
    const R g7 = rmul(relax(c.w7, m7 - e7, s7), R(1.0 / 12.0));
    const R g8 = rmul(relax(c.w8, m8 - e8, s8), R(1.0 / 36.0));
    // d += K g over b = 3..8 with columns of Eq. (3), plus the momentum source F/6 on K1, K2
    R fx6 = 0, fy6 = 0;
    if (FORCED) { fx6 = rmul(Fx, R(1.0 / 6.0)); fy6 = rmul(Fy, R(1.0 / 6.0)); }
    if constexpr (TS) {
        R inc[9];
        inc[0] = R(-4) * g3 + R(4) * g8;
        inc[1] = fx6 - g3 + g4 + R(2) * g7 - R(2) * g8;
        inc[2] = fy6 - g3 - g4 + R(2) * g6 - R(2) * g8;
        inc[3] = -fx6 - g3 + g4 - R(2) * g7 - R(2) * g8;
        inc[4] = -fy6 - g3 - g4 - R(2) * g6 - R(2) * g8;
        inc[5] = fx6 + fy6 + R(2) * g3 + g5 - g6 - g7 + g8;
        inc[6] = -fx6 + fy6 + R(2) * g3 - g5 - g6 + g7 + g8;
        inc[7] = -fx6 - fy6 + R(2) * g3 + g5 + g6 + g7 + g8;
        inc[8] = fx6 - fy6 + R(2) * g3 - g5 + g6 - g7 + g8;
        add_increments<R, true>(d, inc, err);
        return;
    }
    d[0] += R(-4) * g3 + R(4) * g8;
    d[1] += fx6 - g3 + g4 + R(2) * g7 - R(2) * g8;
    d[2] += fy6 - g3 - g4 + R(2) * g6 - R(2) * g8;
    d[3] += -fx6 - g3 + g4 - R(2) * g7 - R(2) * g8;
    d[4] += -fy6 - g3 - g4 - R(2) * g6 - R(2) * g8;
    d[5] += fx6 + fy6 + R(2) * g3 + g5 - g6 - g7 + g8;
    d[6] += -fx6 + fy6 + R(2) * g3 - g5 - g6 + g7 + g8;
    d[7] += -fx6 - fy6 + R(2) * g3 + g5 + g6 + g7 + g8;
    d[8] += fx6 - fy6 + R(2) * g3 - g5 + g6 - g7 + g8;
}

template <int MODEL, typename R, bool FORCED, bool TS = false>
LBM_HD void collide(R d[9], R Fx, R Fy, const Coef<R>& c, R* err = nullptr) {
    if (MODEL == LBM_CASCADED) collide_cascaded<R, FORCED, TS>(d, Fx, Fy, c, err);
    else if (MODEL == LBM_BGK) collide_bgk<R, FORCED, TS>(d, Fx, Fy, c, err);
    else collide_rawmrt<R, FORCED, TS>(d, Fx, Fy, c, err);
}

// ---------------------------------------------------------------- one node, one step
// a1-a9: AA-pattern load, decode, force, collision, encode, AA-pattern store.
// With SR on FP32 storage the collision keeps the exact remainder of each
// post-collision value for the stochastic rounding of the store.
// OOP: store into a.fo instead of a.f (an out-of-place step).
template <int MODEL, int STORE, bool ODD, int FORCE, bool WALLS, bool SR = false, bool OOP = false>
__device__ __forceinline__ void step_node(const Args& a, int x, int y, unsigned rb) {
    using R = typename Store<STORE>::R;
    constexpr bool TS = SR && STORE == LBM_F32;
    const Coef<R> c(a);
    R d[9], err[9];
    load_node<STORE, ODD, WALLS>(a, x, y, d);
    R Fx, Fy;
    node_force<R, FORCE>(a, x, y, Fx, Fy);
    collide<MODEL, R, (FORCE != 0), TS>(d, Fx, Fy, c, err);
    store_node<STORE, ODD, WALLS, SR, OOP>(a, x, y, d, rb, err);
}

// As step_node; with walls, only nodes on the lattice edge take the wall-aware
// path (an interior node has no wall link and no wrapped neighbour).  rb as in
// store_node (ignored unless SR).
template <int MODEL, int STORE, bool ODD, int FORCE, bool WALLS, bool SR = false>
__device__ __forceinline__ void step_node_split(const Args& a, int x, int y, unsigned rb = 0u) {
    if (WALLS && ((x == 0) | (x == a.nx - 1) | (y == 0) | (y == a.ny - 1)))
        step_node<MODEL, STORE, ODD, FORCE, true, SR>(a, x, y, rb);
    else
        step_node<MODEL, STORE, ODD, FORCE, false, SR>(a, x, y, rb);
}

}  // namespace lbm
