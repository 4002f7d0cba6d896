// lbm3d_device.cuh -- per-node pieces of the D3Q27 central-moment update.
//
// The paper develops the cascaded (central-moment) method for D2Q9 (Sec. II)
// and names three-dimensional lattices as future work.  Carried to D3Q27 the
// method reads: take the 27 central moments kappa_ijk (i, j, k in {0,1,2}) of
// f_bar about u = (j + F/2)/rho, relax each towards the discrete Maxwellian
// rho m_i m_j m_k (m = 1, 0, 1/3) -- the trace of the second-order moments at
// omega_bulk, their deviators and off-diagonal parts at omega_shear, orders
// 3..6 at omega_3..omega_6, density and first order kept -- add the source
// whose central moments are (0; F; 0 ...), and transform back.
//
// GB300 formulation: the 27 x 27 transform factorises into three sweeps of
// the 1-D transform (e = -1, 0, 1 -> central moments of order 0, 1, 2 about
// u_x, then u_y, then u_z), 9 lines each, in registers.  Populations are held
// as deviations d = f - w rho0 and the sweeps act on d; the moments of the
// rest state w rho0 about u are rho0 prod mu(i, u) with mu = (1, -u, 1/3 + u^2),
// so the relaxation targets enter as Delta_ijk = (rho - rho0) m_i m_j m_k -
// rho0 (prod mu - prod m), expanded term by term (never an O(1) difference in
// FP32).  The inverse sweeps return the post-collision deviations.
//
// Direction a = (e_x+1) + 3 (e_y+1) + 9 (e_z+1) (tensor order; opposite 26 - a),
// moment index m = i + 3 j + 9 k, weights w = w1(e_x) w1(e_y) w1(e_z) with the
// D1Q3 weights w1(0) = 2/3, w1(+-1) = 1/6.
#pragma once

#include "lbm_device.cuh"

namespace lbm3 {

using lbm::recip;

__host__ __device__ constexpr int ex(int a) { return a % 3 - 1; }
__host__ __device__ constexpr int ey(int a) { return (a / 3) % 3 - 1; }
__host__ __device__ constexpr int ez(int a) { return a / 9 - 1; }
__host__ __device__ constexpr int opp(int a) { return 26 - a; }
template <typename R>
__host__ __device__ constexpr R w1(int e) { return e == 0 ? R(2) / R(3) : R(1) / R(6); }
template <typename R>
__host__ __device__ constexpr R wgt(int a) { return w1<R>(ex(a)) * w1<R>(ey(a)) * w1<R>(ez(a)); }

static_assert(opp(13) == 13 && ex(0) == -1 && ez(26) == 1, "tensor order");

// Launch arguments (plain old data).
struct Args3 {
    void* f;             // populations [27][nz][ny][pitch] of the stored type (deviations)
    long long plane;     // pitch * ny * nz
    int nx, ny, nz, pitch;
    double kd[10];       // omega_bulk, omega_shear, omega_3..omega_6, rho0, F_x, F_y, F_z (physical units)
    float kf[10];        // the same in FP32, rho0 and F times `scale` (the step works in stored units)
    double scale;        // storage scale of the deviations (Store<>::scale: 4096 for FP16, else 1)
};
enum : int { K3_OB = 0, K3_OS = 1, K3_O3 = 2, K3_RHO0 = 6, K3_FX = 7, K3_FY = 8, K3_FZ = 9 };

template <typename R> __device__ __forceinline__ const R* kconst3(const Args3& a);
template <> __device__ __forceinline__ const float* kconst3<float>(const Args3& a) { return a.kf; }
template <> __device__ __forceinline__ const double* kconst3<double>(const Args3& a) { return a.kd; }

// 1-D central-moment transform of the values at e = -1, 0, +1 about u, in
// place: (v-, v0, v+) -> (k0, k1, k2) with k_n = sum_e (e - u)^n v_e.
template <typename R>
__device__ __forceinline__ void sweep_fwd(R& a, R& b, R& c, R u) {
    const R k0 = a + b + c;
    const R s = c - a, p = c + a;
    const R k1 = s - u * k0;
    const R k2 = p - R(2) * u * s + u * u * k0;
    a = k0;
    b = k1;
    c = k2;
}
// Its inverse: raw moments r1 = k1 + u k0, r2 = k2 + 2 u k1 + u^2 k0, then
// v0 = k0 - r2, v+ = (r2 + r1)/2, v- = (r2 - r1)/2.
template <typename R>
__device__ __forceinline__ void sweep_inv(R& a, R& b, R& c, R u) {
    const R k0 = a, k1 = b, k2 = c;
    const R r1 = k1 + u * k0;
    const R r2 = k2 + R(2) * u * k1 + u * u * k0;
    a = R(0.5) * (r2 - r1);
    b = k0 - r2;
    c = R(0.5) * (r2 + r1);
}

// All 27 values: sweeps along x, y, z (forward) or z, y, x (inverse).
template <typename R>
__device__ __forceinline__ void transform_fwd(R c[27], R ux, R uy, R uz) {
#pragma unroll
    for (int l = 0; l < 9; ++l) sweep_fwd(c[3 * l], c[3 * l + 1], c[3 * l + 2], ux);
#pragma unroll
    for (int l = 0; l < 9; ++l) {
        const int b = (l % 3) + 9 * (l / 3);
        sweep_fwd(c[b], c[b + 3], c[b + 6], uy);
    }
#pragma unroll
    for (int l = 0; l < 9; ++l) sweep_fwd(c[l], c[l + 9], c[l + 18], uz);
}
template <typename R>
__device__ __forceinline__ void transform_inv(R c[27], R ux, R uy, R uz) {
#pragma unroll
    for (int l = 0; l < 9; ++l) sweep_inv(c[l], c[l + 9], c[l + 18], uz);
#pragma unroll
    for (int l = 0; l < 9; ++l) {
        const int b = (l % 3) + 9 * (l / 3);
        sweep_inv(c[b], c[b + 3], c[b + 6], uy);
    }
#pragma unroll
    for (int l = 0; l < 9; ++l) sweep_inv(c[3 * l], c[3 * l + 1], c[3 * l + 2], ux);
}

// prod_d mu(n_d, u_d) - prod_d m(n_d) for orders (i, j, k), written as the sum
// of the products that contain at least one eps = mu - m (eps = 0, -u, u^2);
// terms with a vanishing factor (m_1 = 0, eps_0 = 0) are left out at compile
// time, so nothing O(1) is ever subtracted.
template <typename R>
__device__ __forceinline__ R prod_excess(int i, int j, int k, const R epx[3], const R epy[3], const R epz[3]) {
    const R m[3] = {R(1), R(0), R(1.0 / 3.0)};
    const bool mi = i != 1, mj = j != 1, mk = k != 1;
    const bool ei = i != 0, ej = j != 0, ek = k != 0;
    R s = R(-0.0);
    if (ei && mj && mk) s += epx[i] * (m[j] * m[k]);
    if (mi && ej && mk) s += epy[j] * (m[i] * m[k]);
    if (mi && mj && ek) s += epz[k] * (m[i] * m[j]);
    if (ei && ej && mk) s += epx[i] * epy[j] * m[k];
    if (ei && mj && ek) s += epx[i] * epz[k] * m[j];
    if (mi && ej && ek) s += epy[j] * epz[k] * m[i];
    if (ei && ej && ek) s += epx[i] * epy[j] * epz[k];
    return s;
}

__host__ __device__ constexpr double meq(int n) { return n == 0 ? 1.0 : (n == 1 ? 0.0 : 1.0 / 3.0); }

// Collision of one node, on deviations d (in place).
template <typename R, bool FORCED>
__device__ __forceinline__ void collide3(R d[27], const Args3& a) {
    const R* k = kconst3<R>(a);
    const R rho0 = k[K3_RHO0];
    const R Fx = FORCED ? k[K3_FX] : R(0), Fy = FORCED ? k[K3_FY] : R(0), Fz = FORCED ? k[K3_FZ] : R(0);
    R drho = R(0), jx = R(0), jy = R(0), jz = R(0);
#pragma unroll
    for (int q = 0; q < 27; ++q) {
        drho += d[q];
        if (ex(q) != 0) jx += R(ex(q)) * d[q];
        if (ey(q) != 0) jy += R(ey(q)) * d[q];
        if (ez(q) != 0) jz += R(ez(q)) * d[q];
    }
    const R rho = rho0 + drho;
    const R inv = recip(rho);
    const R ux = (FORCED ? jx + R(0.5) * Fx : jx) * inv;
    const R uy = (FORCED ? jy + R(0.5) * Fy : jy) * inv;
    const R uz = (FORCED ? jz + R(0.5) * Fz : jz) * inv;
    transform_fwd(d, ux, uy, uz);  // d now holds the central moments of the deviations
    const R epx[3] = {R(0), -ux, ux * ux}, epy[3] = {R(0), -uy, uy * uy}, epz[3] = {R(0), -uz, uz * uz};
    // Delta_m = (rho - rho0) prod m - rho0 (prod mu - prod m): target minus rest-state moment
    auto delta = [&](int i, int j, int kk) -> R {
        const double pm = meq(i) * meq(j) * meq(kk);
        const R ex_ = prod_excess(i, j, kk, epx, epy, epz);
        return pm != 0.0 ? R(pm) * drho - rho0 * ex_ : -rho0 * ex_;
    };
    const R ob = k[K3_OB], os = k[K3_OS];
    // second order: trace at omega_bulk, deviators and off-diagonals at omega_shear
    constexpr int XX = 2, YY = 6, ZZ = 18, XY = 4, XZ = 10, YZ = 12;
    {
        const R dxx = delta(2, 0, 0), dyy = delta(0, 2, 0), dzz = delta(0, 0, 2);
        const R T = d[XX] + d[YY] + d[ZZ], D1 = d[XX] - d[YY], D2 = d[XX] - d[ZZ];
        const R Tn = T + ob * ((dxx + dyy + dzz) - T);
        const R D1n = D1 + os * ((dxx - dyy) - D1);
        const R D2n = D2 + os * ((dxx - dzz) - D2);
        const R third = R(1.0 / 3.0);
        d[XX] = third * (Tn + D1n + D2n);
        d[YY] = third * (Tn - R(2) * D1n + D2n);
        d[ZZ] = third * (Tn + D1n - R(2) * D2n);
        d[XY] += os * (delta(1, 1, 0) - d[XY]);
        d[XZ] += os * (delta(1, 0, 1) - d[XZ]);
        d[YZ] += os * (delta(0, 1, 1) - d[YZ]);
    }
    // orders 3 .. 6
#pragma unroll
    for (int m = 0; m < 27; ++m) {
        const int i = m % 3, j = (m / 3) % 3, kk = m / 9, n = i + j + kk;
        if (n < 3) continue;
        const R om = k[K3_O3 + (n - 3)];
        d[m] += om * (delta(i, j, kk) - d[m]);
    }
    // the source adds F to the first-order central moments
    if (FORCED) {
        d[1] += Fx;
        d[3] += Fy;
        d[9] += Fz;
    }
    transform_inv(d, ux, uy, uz);
}

// Deviations of the transformed start state f_bar = f_eq(rho, u) - S/2.
template <typename R>
__device__ __forceinline__ void equilibrium3(R d[27], R rho0, R drho, R ux, R uy, R uz, R Fx, R Fy, R Fz) {
    const R epx[3] = {R(0), -ux, ux * ux}, epy[3] = {R(0), -uy, uy * uy}, epz[3] = {R(0), -uz, uz * uz};
#pragma unroll
    for (int m = 0; m < 27; ++m) {
        const int i = m % 3, j = (m / 3) % 3, k = m / 9;
        const double pm = meq(i) * meq(j) * meq(k);
        const R ex_ = prod_excess(i, j, k, epx, epy, epz);
        d[m] = pm != 0.0 ? R(pm) * drho - rho0 * ex_ : -rho0 * ex_;
    }
    d[1] -= R(0.5) * Fx;
    d[3] -= R(0.5) * Fy;
    d[9] -= R(0.5) * Fz;
    transform_inv(d, ux, uy, uz);
}

// ---------------------------------------------------------------- AA-pattern access (periodic)
// even step: node x reads slot a of x and writes post-collision a into slot
// opp(a) of x; odd step: node x reads slot opp(a) of x - e_a and writes
// post-collision a into slot a of x + e_a.
template <typename T>
__device__ __forceinline__ long long node_off(const Args3& a, int x, int y, int z) {
    return ((long long)z * a.ny + y) * a.pitch + x;
}

template <int STORE, bool ODD>
__device__ __forceinline__ void load3(const Args3& a, int x, int y, int z, typename lbm::Store<STORE>::R d[27]) {
    using S = lbm::Store<STORE>;
    using T = typename S::T;
    const T* __restrict__ f = static_cast<const T*>(a.f);
    if (!ODD) {
        const long long n = node_off<T>(a, x, y, z);
#pragma unroll
        for (int q = 0; q < 27; ++q) d[q] = S::dec(f[q * a.plane + n]);
    } else {
        const int xs[3] = {x > 0 ? x - 1 : a.nx - 1, x, x < a.nx - 1 ? x + 1 : 0};
        const int ys[3] = {y > 0 ? y - 1 : a.ny - 1, y, y < a.ny - 1 ? y + 1 : 0};
        const int zs[3] = {z > 0 ? z - 1 : a.nz - 1, z, z < a.nz - 1 ? z + 1 : 0};
#pragma unroll
        for (int q = 0; q < 27; ++q)  // source x - e_q: index 1 - e
            d[q] = S::dec(f[opp(q) * a.plane + node_off<T>(a, xs[1 - ex(q)], ys[1 - ey(q)], zs[1 - ez(q)])]);
    }
}

template <int STORE, bool ODD>
__device__ __forceinline__ void store3(const Args3& a, int x, int y, int z, const typename lbm::Store<STORE>::R d[27]) {
    using S = lbm::Store<STORE>;
    using T = typename S::T;
    T* __restrict__ f = static_cast<T*>(a.f);
    if (!ODD) {
        const long long n = node_off<T>(a, x, y, z);
#pragma unroll
        for (int q = 0; q < 27; ++q) f[opp(q) * a.plane + n] = S::enc(d[q]);
    } else {
        const int xs[3] = {x > 0 ? x - 1 : a.nx - 1, x, x < a.nx - 1 ? x + 1 : 0};
        const int ys[3] = {y > 0 ? y - 1 : a.ny - 1, y, y < a.ny - 1 ? y + 1 : 0};
        const int zs[3] = {z > 0 ? z - 1 : a.nz - 1, z, z < a.nz - 1 ? z + 1 : 0};
#pragma unroll
        for (int q = 0; q < 27; ++q)  // target x + e_q: index 1 + e
            f[q * a.plane + node_off<T>(a, xs[1 + ex(q)], ys[1 + ey(q)], zs[1 + ez(q)])] = S::enc(d[q]);
    }
}

}  // namespace lbm3
