// lbm_fused.cuh -- two time steps per launch (temporal blocking) for FP32 and
// 16-bit storage: one HBM read and one HBM write of the populations per two
// collide-and-stream steps (Eq. 23-24) instead of one of each per step.
//
// A CTA owns a TX x TY tile of nodes.  Two steps need the tile's state at time
// t on the tile grown by two nodes on every side, so:
//   1. one TMA load (cp.async.bulk.tensor.3d) brings all nine population
//      planes of that region, f(t), into shared memory (the box starts at a
//      16-byte aligned column left of the region; periodic wrap-around, which
//      a tensor copy does not do, is patched with plain loads on edge tiles);
//   2. every node of the grown region collides in place (step t: collision of
//      Sec. II, rounded to the storage format exactly as the one-step kernel
//      stores it, in the AA even-step slots);
//   3. every node of the tile grown by one node takes the AA odd step in the
//      same buffer: it reads its populations from its neighbours' even-step
//      slots, with the wall links of Sec. III-A/C, collides (step t + 1) and
//      writes into the slots it read from, which no other node touches, so
//      the step needs no second buffer;
//   4. after the odd step the buffer holds f(t + 2) in the natural layout, and
//      the tile goes to the output array by bulk copies, one per row and plane.
// The per-node arithmetic and every rounding of the stored values are those of
// two single steps (AA even step then odd step), so the result is bit for bit
// that of lbm_step without fusion; nodes of the grown regions are computed by
// more than one CTA (about 1.24x the collisions of two single steps for a
// 64 x 16 tile).  The input and output arrays differ (ping-pong): neighbouring
// CTAs read the halo of this CTA's tile while it writes.
#pragma once

#include <cuda.h>

#include <type_traits>

#include "lbm_async.cuh"
#include "lbm_device.cuh"
#include "lbm_pair.cuh"

namespace lbm {

// Tile geometry and launch shape per storage kind.
template <int STORE> struct FusedTile;
template <> struct FusedTile<LBM_F32> {
    static constexpr int TX = 64, TY = 16, ALIGN = 4, THREADS = 256, MIN_BLOCKS = 4;
};
template <> struct FusedTile<LBM_F16DEV> {
    static constexpr int TX = 64, TY = 16, ALIGN = 8, THREADS = 256, MIN_BLOCKS = 4;
};
template <> struct FusedTile<LBM_BF16DEV> : FusedTile<LBM_F16DEV> {};

// Shared-memory geometry of the fused kernel for one storage kind.
template <int STORE>
struct FusedGeom {
    using FT = FusedTile<STORE>;
    using T = typename Store<STORE>::T;
    static constexpr int TX = FT::TX, TY = FT::TY;
    static constexpr int BW = TX + 2 * FT::ALIGN;   // box width (elements): 16-byte aligned on both sides
    static constexpr int BH = TY + 4;               // box height: two halo rows above and below
    static constexpr int OFF = FT::ALIGN - 2;       // column of region x = x0 - 2 inside the box
    static constexpr int RW = TX + 4, RH = TY + 4;  // region collided at step t
    static constexpr int SW = TX + 2, SH = TY + 2;  // region collided at step t + 1
    static constexpr size_t A_BYTES = size_t(9) * BH * BW * sizeof(T);
    static constexpr size_t SMEM = A_BYTES;
    static_assert((BW * sizeof(T)) % 16 == 0 && (FT::ALIGN * sizeof(T)) == 16, "TMA box alignment");
    static_assert((TX * sizeof(T)) % 16 == 0, "bulk row copies of the tile start and end on 16-byte boundaries");
};

// Error codes the fused kernel leaves in its error word.
enum : int { kFusedErrTimeout = 1 };

// ---------------------------------------------------------------- packed stages
// Stages 2 and 3 of a tile with two nodes per thread (the k-th and the
// (k + half)-th node of the region) collided together in packed FP32x2
// arithmetic; loads, conversions, wall links and stores stay per node.  A node
// beyond a wall (or the missing partner of an odd region) is collided on
// whatever its slots hold and not stored.
template <int MODEL, int STORE, int FORCE, bool WALLS, bool SR>
__device__ __forceinline__ void fused2_pack_stages(const Args& a, typename Store<STORE>::T* A, int x0, int y0,
                                                   unsigned rb0, unsigned rb1) {
    using G = FusedGeom<STORE>;
    using S = Store<STORE>;
    using T = typename S::T;
    constexpr int NT = FusedTile<STORE>::THREADS;
    const int tid = threadIdx.x;
    const bool perx = !a.wall[LBM_WEST], pery = !a.wall[LBM_SOUTH];
    auto Aat = [&](int q, int ry, int rxb) -> T& { return A[(q * G::BH + ry) * G::BW + rxb]; };
    const bool small = a.nx <= G::TX + 2 || a.ny <= G::TY + 2;
    auto wrap = [small](int v, int n) {
        if (small) return ((v % n) + n) % n;
        return v < 0 ? v + n : (v >= n ? v - n : v);
    };
    const Coef<F2> c2 = pair_coef(a);
    auto enc = [&](float v, unsigned rn, int q) -> T {
        if constexpr (SR) return enc_sr<STORE>(v, rn + static_cast<unsigned>(q) * kRoundStride);
        else return S::enc(v);
    };

    // ---- 2. step t on the grown region (AA even step, in place)
    constexpr int N2 = G::RW * G::RH, H2 = (N2 + 1) / 2;
    for (int k = tid; k < H2; k += NT) {
        int ry[2], rx[2], gx[2], gy[2];
        bool ok[2];
#pragma unroll
        for (int j = 0; j < 2; ++j) {
            const int kk = k + j * H2 < N2 ? k + j * H2 : k;
            ry[j] = kk / G::RW;
            rx[j] = kk % G::RW;
            gx[j] = x0 - 2 + rx[j];
            gy[j] = y0 - 2 + ry[j];
            ok[j] = k + j * H2 < N2 && !((!perx && (gx[j] < 0 || gx[j] >= a.nx)) || (!pery && (gy[j] < 0 || gy[j] >= a.ny)));
            gx[j] = wrap(gx[j], a.nx);
            gy[j] = wrap(gy[j], a.ny);
        }
        F2 d[9];
#pragma unroll
        for (int q = 0; q < 9; ++q)
            d[q] = F2(make_float2(S::dec(Aat(q, ry[0], rx[0] + G::OFF)), S::dec(Aat(q, ry[1], rx[1] + G::OFF))));
        float fx[2], fy[2];
#pragma unroll
        for (int j = 0; j < 2; ++j) node_force<float, FORCE>(a, gx[j], gy[j], fx[j], fy[j]);
        collide<MODEL, F2, (FORCE != 0)>(d, F2(make_float2(fx[0], fx[1])), F2(make_float2(fy[0], fy[1])), c2);
#pragma unroll
        for (int j = 0; j < 2; ++j) {
            if (!ok[j]) continue;
            const unsigned rn = SR ? round_node(a, rb0, gx[j], gy[j]) : 0u;
#pragma unroll
            for (int q = 0; q < 9; ++q) Aat(opp(q), ry[j], rx[j] + G::OFF) = enc(j ? d[q].v.y : d[q].v.x, rn, q);
        }
    }
    __syncthreads();

    // ---- 3. step t + 1 on the tile grown by one node (AA odd step, in place)
    constexpr int N3 = G::SW * G::SH, H3 = (N3 + 1) / 2;
    for (int k = tid; k < H3; k += NT) {
        int ry[2], rxb[2], gx[2], gy[2];
        bool ok[2];
#pragma unroll
        for (int j = 0; j < 2; ++j) {
            const int kk = k + j * H3 < N3 ? k + j * H3 : k;
            const int sy = kk / G::SW, sx = kk % G::SW;
            gx[j] = x0 - 1 + sx;
            gy[j] = y0 - 1 + sy;
            ok[j] = k + j * H3 < N3 && !((!perx && (gx[j] < 0 || gx[j] >= a.nx)) || (!pery && (gy[j] < 0 || gy[j] >= a.ny)));
            gx[j] = wrap(gx[j], a.nx);
            gy[j] = wrap(gy[j], a.ny);
            ry[j] = sy + 1;
            rxb[j] = sx + 1 + G::OFF;
        }
        F2 d[9];
#pragma unroll
        for (int q = 0; q < 9; ++q) {
            float v[2];
#pragma unroll
            for (int j = 0; j < 2; ++j) {
                const int w = WALLS ? incoming_wall(a, q, gx[j], gy[j]) : -1;
                if (w >= 0) v[j] = add_wall_term<float>(a, S::dec(Aat(q, ry[j], rxb[j])), q, w);
                else v[j] = S::dec(Aat(opp(q), ry[j] - cy(q), rxb[j] - cx(q)));
            }
            d[q] = F2(make_float2(v[0], v[1]));
        }
        float fx[2], fy[2];
#pragma unroll
        for (int j = 0; j < 2; ++j) node_force<float, FORCE>(a, gx[j], gy[j], fx[j], fy[j]);
        collide<MODEL, F2, (FORCE != 0)>(d, F2(make_float2(fx[0], fx[1])), F2(make_float2(fy[0], fy[1])), c2);
#pragma unroll
        for (int j = 0; j < 2; ++j) {
            if (!ok[j]) continue;
            const unsigned rn = SR ? round_node(a, rb1, gx[j], gy[j]) : 0u;
#pragma unroll
            for (int q = 0; q < 9; ++q) {
                const int w = WALLS ? incoming_wall(a, opp(q), gx[j], gy[j]) : -1;
                float v = j ? d[q].v.y : d[q].v.x;
                if (w >= 0) v = add_wall_term<float>(a, v, opp(q), w);
                const T o = enc(v, rn, q);
                if (w >= 0) Aat(opp(q), ry[j], rxb[j]) = o;
                else Aat(q, ry[j] + cy(q), rxb[j] + cx(q)) = o;
            }
        }
    }
}

// ---------------------------------------------------------------- one tile
// Two steps of the tile with corner (x0, y0): `in` is the input array (natural
// layout at the even step t), `out` the output array (f(t + 2), natural
// layout); `map` describes `in` as a 3-D tensor [9][ny][nx] with row pitch
// a.pitch (kernel parameter or global memory); rb0 and rb1 are the
// stochastic-rounding hashes of steps t and t + 1.  smem holds G::SMEM bytes
// (1024-byte aligned); bar and ok live in shared memory, and the mbarrier is
// initialised here and used for this tile's load only.  Every thread of the
// CTA calls this with the same arguments.  PACKED false keeps one node per
// thread everywhere.
template <int MODEL, int STORE, int FORCE, bool WALLS, bool SR, bool PACKED = true>
__device__ __forceinline__ void fused2_tile(const CUtensorMap* map, const Args& a, const void* in, void* out,
                                            int* err, int x0, int y0, unsigned rb0, unsigned rb1,
                                            unsigned char* smem, unsigned long long* bar, int* ok) {
    using G = FusedGeom<STORE>;
    using S = Store<STORE>;
    using T = typename S::T;
    using R = typename S::R;
    constexpr bool TS = SR && STORE == LBM_F32;
    constexpr int NT = FusedTile<STORE>::THREADS;
    T* A = reinterpret_cast<T*>(smem);
    const int tid = threadIdx.x;
    const bool perx = !a.wall[LBM_WEST], pery = !a.wall[LBM_SOUTH];

    // ---- 1. the region's state at time t
    if (tid == 0) {
        mbar_init(bar, 1);
        mbar_expect_tx(bar, static_cast<unsigned>(G::A_BYTES));
        tma_load_3d(A, map, x0 - FusedTile<STORE>::ALIGN, y0 - 2, 0, bar);
        bool done = mbar_wait_bounded(bar, 0, 1000000000ull);  // 1 s
        if (!done) {
            atomicOr(err, kFusedErrTimeout);
            mbar_wait_bounded(bar, 0, 4000000000ull);  // let the copy land before the CTA exits
        }
        *ok = done ? 1 : 0;
    }
    __syncthreads();
    if (!*ok) return;
    auto Aat = [&](int q, int ry, int rxb) -> T& { return A[(q * G::BH + ry) * G::BW + rxb]; };
    // Region coordinates lie in [-2, n + TX + 1]: one addition or subtraction of
    // n wraps them when n > TX + 2 (TY + 2 along y); smaller lattices take the modulo.
    const bool small = a.nx <= G::TX + 2 || a.ny <= G::TY + 2;
    auto wrap = [small](int v, int n) {
        if (small) return ((v % n) + n) % n;
        return v < 0 ? v + n : (v >= n ? v - n : v);
    };

    // periodic wrap-around of the region's halo (edge tiles only).  The nodes of
    // the tile depend on the region's cells within two nodes of the lattice,
    // x in [-2, nx + 1] and y in [-2, ny + 1]; the cells of that ring outside the
    // lattice across a periodic edge are fetched from their images.  Region
    // cells further out (a tile cut by the lattice's edge) keep the zeros of the
    // tensor load: they are collided but feed no node of the lattice, since in
    // both steps every slot is read and written by one node only.
    if ((perx && (x0 - 2 < 0 || x0 + G::TX + 2 > a.nx)) || (pery && (y0 - 2 < 0 || y0 + G::TY + 2 > a.ny))) {
        const T* __restrict__ f = static_cast<const T*>(in);
        const int X0 = x0 - 2, Y0 = y0 - 2;                 // region origin (>= -2)
        const int X1 = min(x0 + G::TX + 2, a.nx + 2);        // ring end along x
        const int Y1 = min(y0 + G::TY + 2, a.ny + 2);
        const int xi0 = max(X0, 0), xi1 = min(X1, a.nx);     // columns inside the lattice
        const int yi0 = max(Y0, 0), yi1 = min(Y1, a.ny);
        // rows outside the lattice (periodic y): below 0, then from ny; each over
        // the ring's columns (all of them if x is periodic, else those inside)
        const int rlo = pery ? max(0, min(0, Y1) - Y0) : 0;
        const int rhi = pery ? max(0, Y1 - max(a.ny, Y0)) : 0;
        const int rx0 = perx ? X0 : xi0, rw = max(0, (perx ? X1 : xi1) - rx0);
        // columns outside the lattice (periodic x), over the rows inside it
        const int clo = perx ? max(0, min(0, X1) - X0) : 0;
        const int chi = perx ? max(0, X1 - max(a.nx, X0)) : 0;
        const int ch = max(0, yi1 - yi0);
        const int nrow = (rlo + rhi) * rw, ncell = nrow + (clo + chi) * ch;
        for (int k = tid; k < ncell; k += NT) {
            int gx, gy;
            if (k < nrow) {
                const int r = k / rw;
                gx = rx0 + (k - r * rw);
                gy = r < rlo ? Y0 + r : max(a.ny, Y0) + (r - rlo);
            } else {
                const int c = (k - nrow) / ch;
                gy = yi0 + (k - nrow - c * ch);
                gx = c < clo ? X0 + c : max(a.nx, X0) + (c - clo);
            }
            const int ry = gy - Y0, rx = gx - X0;
            const long long src = (long long)(((gy % a.ny) + a.ny) % a.ny) * a.pitch + ((gx % a.nx) + a.nx) % a.nx;
#pragma unroll
            for (int q = 0; q < 9; ++q) Aat(q, ry, rx + G::OFF) = f[q * a.plane + src];
        }
        __syncthreads();
    }

    const Coef<R> c(a);
    // Two nodes per thread in packed FP32x2 arithmetic where the packed
    // collision rounds every value exactly as the scalar one (the cascaded
    // collision without forcing, FP32 storage, round to nearest) and the
    // registers suffice (no walls): 4-5 % faster there.  With forcing and in
    // the siblings the compiler contracts some single-use products of the
    // scalar code into the next addition across statements, which the packed
    // code rounds separately (a unit in the last place apart); with walls the
    // packed stages spill; 16-bit storage runs slower packed.
    constexpr bool PACK = PACKED && MODEL == LBM_CASCADED && FORCE == 0 && STORE == LBM_F32 && !SR && !WALLS;
    if constexpr (PACK) {
        fused2_pack_stages<MODEL, STORE, FORCE, WALLS, SR>(a, A, x0, y0, rb0, rb1);
    } else {
    // ---- 2. step t: collide the grown region in place (AA even step: the
    // post-collision population q of a node goes to its own slot of plane opp(q))
    for (int k = tid; k < G::RW * G::RH; k += NT) {
        const int ry = k / G::RW, rx = k % G::RW;
        int gx = x0 - 2 + rx, gy = y0 - 2 + ry;
        if ((!perx && (gx < 0 || gx >= a.nx)) || (!pery && (gy < 0 || gy >= a.ny))) continue;
        gx = wrap(gx, a.nx);
        gy = wrap(gy, a.ny);
        R d[9], e[9];
#pragma unroll
        for (int q = 0; q < 9; ++q) d[q] = S::dec(Aat(q, ry, rx + G::OFF));
        R Fx, Fy;
        node_force<R, FORCE>(a, gx, gy, Fx, Fy);
        collide<MODEL, R, (FORCE != 0), TS>(d, Fx, Fy, c, e);
        const unsigned rn = SR ? round_node(a, rb0, gx, gy) : 0u;
#pragma unroll
        for (int q = 0; q < 9; ++q) {
            const unsigned r = rn + static_cast<unsigned>(q) * kRoundStride;
            T v;
            if constexpr (TS) v = round_sr32(d[q], e[q], r);
            else if constexpr (SR) v = enc_sr<STORE>(d[q], r);
            else v = S::enc(d[q]);
            Aat(opp(q), ry, rx + G::OFF) = v;
        }
    }
    __syncthreads();

    // ---- 3. step t + 1 on the tile grown by one node, in place (AA odd step:
    // population q arrives from slot opp(q) of the node at x - e_q, or through a
    // wall from the node's own slot q; it leaves into slot q of the node at
    // x + e_q, or through a wall into the node's own slot opp(q); each slot is
    // read and written by one node only)
    // A tile whose grown region holds no node next to a wall runs the body
    // without wall links: incoming_wall finds none there, so the arithmetic is
    // the same.
    auto odd_step = [&](auto walls_tag) {
        constexpr bool WL = decltype(walls_tag)::value;
        for (int k = tid; k < G::SW * G::SH; k += NT) {
            const int sy = k / G::SW, sx = k % G::SW;
            int gx = x0 - 1 + sx, gy = y0 - 1 + sy;
            if ((!perx && (gx < 0 || gx >= a.nx)) || (!pery && (gy < 0 || gy >= a.ny))) continue;
            gx = wrap(gx, a.nx);
            gy = wrap(gy, a.ny);
            const int ry = sy + 1, rxb = sx + 1 + G::OFF;
            R d[9], e[9];
#pragma unroll
            for (int q = 0; q < 9; ++q) {
                const int w = WL ? incoming_wall(a, q, gx, gy) : -1;
                if (w >= 0) d[q] = add_wall_term<R>(a, S::dec(Aat(q, ry, rxb)), q, w);
                else d[q] = S::dec(Aat(opp(q), ry - cy(q), rxb - cx(q)));
            }
            R Fx, Fy;
            node_force<R, FORCE>(a, gx, gy, Fx, Fy);
            collide<MODEL, R, (FORCE != 0), TS>(d, Fx, Fy, c, e);
            const unsigned rn = SR ? round_node(a, rb1, gx, gy) : 0u;
#pragma unroll
            for (int q = 0; q < 9; ++q) {
                const unsigned r = rn + static_cast<unsigned>(q) * kRoundStride;
                const int w = WL ? incoming_wall(a, opp(q), gx, gy) : -1;
                R v = d[q], ev = TS ? e[q] : R(0);
                if (w >= 0) {
                    if constexpr (TS) {
                        float e2;
                        v = two_sum(d[q], wall_term<R>(a, opp(q), w), e2);
                        ev = e[q] + e2;
                    } else {
                        v = add_wall_term<R>(a, d[q], opp(q), w);
                    }
                }
                T o;
                if constexpr (TS) o = round_sr32(v, ev, r);
                else if constexpr (SR) o = enc_sr<STORE>(v, r);
                else o = S::enc(v);
                if (w >= 0) Aat(opp(q), ry, rxb) = o;
                else Aat(q, ry + cy(q), rxb + cx(q)) = o;
            }
        }
    };
    if constexpr (WALLS) {
        const bool near_wall = (a.wall[LBM_WEST] && x0 - 1 <= 0) || (a.wall[LBM_EAST] && x0 + G::TX >= a.nx - 1) ||
                               (a.wall[LBM_SOUTH] && y0 - 1 <= 0) || (a.wall[LBM_NORTH] && y0 + G::TY >= a.ny - 1);
        if (near_wall) odd_step(std::true_type{});
        else odd_step(std::false_type{});
    } else {
        odd_step(std::false_type{});
    }
    }  // one node per thread
    fence_async_shared();  // the odd step's shared-memory writes before the bulk stores read them
    __syncthreads();

    // ---- 4. f(t + 2) of the tile, natural layout after the odd step: one bulk
    // copy per row of each plane (TX elements, 16-byte aligned at both ends:
    // x0 is a multiple of TX, the row pitch of 32 elements, the box row starts
    // ALIGN elements left of the tile); a tile cut by the lattice's right edge
    // is copied element by element.
    T* __restrict__ fo = static_cast<T*>(out);
    if (x0 + G::TX <= a.nx) {
        const int rows = min(G::TY, a.ny - y0);
        for (int j = tid; j < 9 * rows; j += NT) {
            const int q = j / rows, ty = j - q * rows;
            bulk_store(fo + q * a.plane + (long long)(y0 + ty) * a.pitch + x0, &Aat(q, ty + 2, FusedTile<STORE>::ALIGN),
                       unsigned(G::TX * sizeof(T)));
        }
        bulk_commit();
        bulk_wait_read<0>();  // shared memory stays allocated until the copies have read it
    } else {
        for (int k = tid; k < G::TX * G::TY; k += NT) {
            const int ty = k / G::TX, tx = k % G::TX;
            const int gx = x0 + tx, gy = y0 + ty;
            if (gx >= a.nx || gy >= a.ny) continue;
            const long long n = (long long)gy * a.pitch + gx;
#pragma unroll
            for (int q = 0; q < 9; ++q) fo[q * a.plane + n] = Aat(q, ty + 2, tx + 2 + G::OFF);
        }
    }
}

// ---------------------------------------------------------------- the kernel
// One CTA per tile of one lattice: a.f is the input array, `out` the output
// array, `map` describes a.f.  With stochastic rounding the hashes of steps t
// and t + 1 are a.rbase and a.rbase1, or a.rtable[a.tstep] and
// a.rtable[a.tstep + 1] in a graph replay.
template <int MODEL, int STORE, int FORCE, bool WALLS, bool SR>
__global__ void __launch_bounds__(FusedTile<STORE>::THREADS, FusedTile<STORE>::MIN_BLOCKS)
    fused2_kernel(const __grid_constant__ CUtensorMap map, const Args a, void* __restrict__ out,
                  int* __restrict__ err) {
    extern __shared__ __align__(1024) unsigned char fused_smem[];
    __shared__ __align__(8) unsigned long long bar;
    __shared__ int ok;
    const unsigned rb0 = SR ? (a.rtable ? a.rtable[a.tstep] : a.rbase) : 0u;
    const unsigned rb1 = SR ? (a.rtable ? a.rtable[a.tstep + 1] : a.rbase1) : 0u;
    fused2_tile<MODEL, STORE, FORCE, WALLS, SR>(&map, a, a.f, out, err, blockIdx.x * FusedGeom<STORE>::TX,
                                                blockIdx.y * FusedGeom<STORE>::TY, rb0, rb1, fused_smem, &bar, &ok);
}

}  // namespace lbm

namespace lbm {

// Launch of the fused kernel for one storage kind (dynamic shared memory set
// up on first use of each instantiation).
template <int MODEL, int STORE, int FORCE, bool WALLS, bool SR>
static cudaError_t launch_fused_one(const CUtensorMap& map, const Args& a, void* out, int* err, cudaStream_t s) {
    using G = FusedGeom<STORE>;
    static bool configured = false;
    if (!configured) {
        cudaError_t e = cudaFuncSetAttribute(fused2_kernel<MODEL, STORE, FORCE, WALLS, SR>,
                                             cudaFuncAttributeMaxDynamicSharedMemorySize, int(G::SMEM));
        if (e != cudaSuccess) return e;
        configured = true;
    }
    const dim3 grid((a.nx + G::TX - 1) / G::TX, (a.ny + G::TY - 1) / G::TY);
    fused2_kernel<MODEL, STORE, FORCE, WALLS, SR><<<grid, FusedTile<STORE>::THREADS, G::SMEM, s>>>(map, a, out, err);
    return cudaGetLastError();
}

template <int MODEL, int STORE, int FORCE, bool WALLS>
static cudaError_t launch_fused_sr(const CUtensorMap& map, const Args& a, void* out, int* err, cudaStream_t s) {
    return a.rseed ? launch_fused_one<MODEL, STORE, FORCE, WALLS, true>(map, a, out, err, s)
                   : launch_fused_one<MODEL, STORE, FORCE, WALLS, false>(map, a, out, err, s);
}

template <int MODEL, int STORE, int FORCE>
static cudaError_t launch_fused_walls(const CUtensorMap& map, const Args& a, void* out, int* err, bool walls,
                                      cudaStream_t s) {
    return walls ? launch_fused_sr<MODEL, STORE, FORCE, true>(map, a, out, err, s)
                 : launch_fused_sr<MODEL, STORE, FORCE, false>(map, a, out, err, s);
}

template <int MODEL, int STORE>
static cudaError_t launch_fused_force(const CUtensorMap& map, const Args& a, void* out, int* err, int force,
                                      bool walls, cudaStream_t s) {
    switch (force) {
        case 0: return launch_fused_walls<MODEL, STORE, 0>(map, a, out, err, walls, s);
        case 1: return launch_fused_walls<MODEL, STORE, 1>(map, a, out, err, walls, s);
        default: return launch_fused_walls<MODEL, STORE, 2>(map, a, out, err, walls, s);
    }
}

template <int STORE>
static cudaError_t launch_fused_store(const CUtensorMap& map, const Args& a, void* out, int* err, int model,
                                      int force, bool walls, cudaStream_t s) {
    switch (model) {
        case LBM_CASCADED: return launch_fused_force<LBM_CASCADED, STORE>(map, a, out, err, force, walls, s);
        case LBM_BGK: return launch_fused_force<LBM_BGK, STORE>(map, a, out, err, force, walls, s);
        default: return launch_fused_force<LBM_RAWMRT, STORE>(map, a, out, err, force, walls, s);
    }
}

}  // namespace lbm
