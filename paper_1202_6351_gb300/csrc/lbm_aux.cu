// lbm_aux.cu -- initialisation, state transfer and diagnostics kernels.
//
// These kernels read the populations at the current time through the same
// AA-pattern access as the step kernel (load_node), so they see exactly the
// state the next step would collide.  Their arithmetic is FP64 whatever the
// storage type: they run once per call, not once per step.
#include "lbm_internal.h"

namespace lbm {

namespace {

constexpr int kAuxThreads = 256;

__device__ __forceinline__ void node_force_any(const Args& a, int force, int x, int y, double& Fx, double& Fy,
                                               bool field_is_double) {
    Fx = 0.0; Fy = 0.0;
    if (force == 0) return;
    Fx = a.F[0]; Fy = a.F[1];
    if (force == 2) {
        const long long n = (long long)y * a.nx + x, p = (long long)a.nx * a.ny;
        if (field_is_double) {
            const double* ff = static_cast<const double*>(a.ffield);
            Fx += ff[n]; Fy += ff[p + n];
        } else {
            const float* ff = static_cast<const float*>(a.ffield);
            Fx += ff[n]; Fy += ff[p + n];
        }
    }
}

// Deviations of node (x, y) at the current time in physical units.
template <int STORE>
__device__ __forceinline__ void load_any(const Args& a, bool odd, int x, int y, double d[9]) {
    typename Store<STORE>::R r[9];
    if (odd) load_node<STORE, true, true>(a, x, y, r);
    else load_node<STORE, false, true>(a, x, y, r);
    constexpr double inv = 1.0 / Store<STORE>::scale;
#pragma unroll
    for (int q = 0; q < 9; ++q) d[q] = double(r[q]) * inv;
}

// Equilibria used to start a run, written directly as deviations f_eq - w rho0
// so that FP32 arithmetic keeps the full precision of small deviations.
// Cascaded: the populations whose central moments about u are (rho, 0, 0,
// rho/3, rho/3, 0, 0, 0, rho/9) (Eq. 10).  Their raw moments factor as
// rho M_m(ux) M_n(uy) with M_0 = 1, M_1 = u, M_2 = 1/3 + u^2, so
// f_eq(e) = rho phi(e_x; ux) phi(e_y; uy) with phi(0; u) = 2/3 - u^2 and
// phi(+-1; u) = (1/3 + u^2 +- u)/2.  With phi = w1 + dphi, w1(0) = 2/3,
// w1(+-1) = 1/6 (w = w1(e_x) w1(e_y)):
//   f_eq - w rho0 = (rho - rho0) w + rho (w1x dphi_y + dphi_x w1y + dphi_x dphi_y).
// Siblings: the 2nd-order polynomial, f_eq - w rho0 = w (rho - rho0) + w rho (3 eu + 9/2 eu^2 - 3/2 u^2).
template <typename R>
__device__ __forceinline__ R w1(int e) { return e == 0 ? R(2.0 / 3.0) : R(1.0 / 6.0); }
template <typename R>
__device__ __forceinline__ R dphi(int e, R u) { return e == 0 ? -u * u : R(0.5) * (u * u + R(e) * u); }

template <int STORE>
__global__ void init_kernel(const Args a, int model, int force, bool ffield_double, const double* rho,
                            const double* u) {
    using S = Store<STORE>;
    using T = typename S::T;
    using R = typename S::R;
    const int x = blockIdx.x * blockDim.x + threadIdx.x, y = blockIdx.y;
    if (x >= a.nx) return;
    const long long n = (long long)y * a.nx + x, p = (long long)a.nx * a.ny;
    const R dr = R(rho ? rho[n] - a.rho0 : 0.0);
    const R r = R(a.rho0) + dr;
    const R ux = R(u ? u[n] : 0.0), uy = R(u ? u[p + n] : 0.0);
    double Fxd, Fyd;
    node_force_any(a, force, x, y, Fxd, Fyd, ffield_double);
    R Sq[9];
    source<R>(ux, uy, R(Fxd), R(Fyd), Sq);
    T* f = static_cast<T*>(a.f);
    const long long off = (long long)y * a.pitch + x;
    const R usq = R(1.5) * (ux * ux + uy * uy);
#pragma unroll
    for (int q = 0; q < 9; ++q) {
        R dev;
        if (model == LBM_CASCADED) {
            const R ax = w1<R>(cx(q)), ay = w1<R>(cy(q));
            const R bx = dphi<R>(cx(q), ux), by = dphi<R>(cy(q), uy);
            dev = dr * (ax * ay) + r * (ax * by + bx * ay + bx * by);
        } else {
            const R eu = R(cx(q)) * ux + R(cy(q)) * uy;
            dev = wgt<R>(q) * (dr + r * (R(3) * eu + R(4.5) * eu * eu - usq));
        }
        dev -= R(0.5) * Sq[q];
        f[q * a.plane + off] = S::enc(dev * R(S::scale));
    }
}

template <int STORE>
__global__ void set_f_kernel(const Args a, const double* src) {
    using S = Store<STORE>;
    using T = typename S::T;
    using R = typename S::R;
    const int x = blockIdx.x * blockDim.x + threadIdx.x, y = blockIdx.y;
    if (x >= a.nx) return;
    const long long n = (long long)y * a.nx + x, p = (long long)a.nx * a.ny;
    T* f = static_cast<T*>(a.f);
#pragma unroll
    for (int q = 0; q < 9; ++q)
        f[q * a.plane + (long long)y * a.pitch + x] = S::enc(R((src[q * p + n] - wgt<double>(q) * a.rho0) * S::scale));
}

template <int STORE>
__global__ void get_f_kernel(const Args a, bool odd, double* dst) {
    const int x = blockIdx.x * blockDim.x + threadIdx.x, y = blockIdx.y;
    if (x >= a.nx) return;
    const long long n = (long long)y * a.nx + x, p = (long long)a.nx * a.ny;
    double d[9];
    load_any<STORE>(a, odd, x, y, d);
#pragma unroll
    for (int q = 0; q < 9; ++q) dst[q * p + n] = wgt<double>(q) * a.rho0 + d[q];
}

// rho, rho u (with F/2, Eq. 27) and the velocity of one node, FP64.
struct NodeMacros {
    double rho, mx, my, ux, uy, Fx, Fy;
    Moments<double> m;
};

// rho and u of one node in the storage's arithmetic type (FP32 for all but
// FP64 storage), returned in FP64: rho = rho0 + sum d keeps its precision.
template <int STORE>
__device__ __forceinline__ void node_rho_u(const Args& a, bool odd, int force, bool ffd, int x, int y, double& rho,
                                           double& ux, double& uy) {
    using R = typename Store<STORE>::R;
    R d[9];
    if (odd) load_node<STORE, true, true>(a, x, y, d);
    else load_node<STORE, false, true>(a, x, y, d);
    if (Store<STORE>::scale != 1.0) {
#pragma unroll
        for (int q = 0; q < 9; ++q) d[q] *= R(1.0 / Store<STORE>::scale);
    }
    const Moments<R> m = moments<R>(d, R(a.rho0));
    double Fx, Fy;
    node_force_any(a, force, x, y, Fx, Fy, ffd);
    const R px = m.jx + R(0.5 * Fx), py = m.jy + R(0.5 * Fy);
    const R rr = R(a.rho0) + m.drho;
    rho = a.rho0 + double(m.drho);
    ux = double(px / rr);
    uy = double(py / rr);
}

template <int STORE>
__device__ __forceinline__ NodeMacros node_macros(const Args& a, bool odd, int force, bool ffd, int x, int y) {
    NodeMacros r;
    double d[9];
    load_any<STORE>(a, odd, x, y, d);
    r.m = moments<double>(d, a.rho0);
    node_force_any(a, force, x, y, r.Fx, r.Fy, ffd);
    r.rho = r.m.rho;
    r.mx = r.m.jx + 0.5 * r.Fx;
    r.my = r.m.jy + 0.5 * r.Fy;
    r.ux = r.mx / r.rho;
    r.uy = r.my / r.rho;
    return r;
}

template <int STORE>
__global__ void macros_kernel(const Args a, bool odd, int force, bool ffd, double* rho, double* u) {
    const int x = blockIdx.x * blockDim.x + threadIdx.x, y = blockIdx.y;
    if (x >= a.nx) return;
    const long long n = (long long)y * a.nx + x, p = (long long)a.nx * a.ny;
    double r, ux, uy;
    node_rho_u<STORE>(a, odd, force, ffd, x, y, r, ux, uy);
    if (rho) rho[n] = r;
    if (u) { u[n] = ux; u[p + n] = uy; }
}

// Eq. (28)-(30) with the moments of f = f_bar + S/2: sum e_x^2 S = 2 F_x u_x,
// sum e_y^2 S = 2 F_y u_y, sum e_x e_y S = F_x u_y + F_y u_x (Eq. 13).
template <int STORE>
__global__ void strain_kernel(const Args a, bool odd, int force, bool ffd, double* out) {
    const int x = blockIdx.x * blockDim.x + threadIdx.x, y = blockIdx.y;
    if (x >= a.nx) return;
    const long long n = (long long)y * a.nx + x, p = (long long)a.nx * a.ny;
    const NodeMacros r = node_macros<STORE>(a, odd, force, ffd, x, y);
    const double ux = r.ux, uy = r.uy;
    const double kxx = r.m.kxx + r.Fx * ux, kyy = r.m.kyy + r.Fy * uy;
    const double kxy = r.m.kxy + 0.5 * (r.Fx * uy + r.Fy * ux);
    const double n3 = (kxx + kyy) - (2.0 / 3.0) * r.m.drho - r.rho * (ux * ux + uy * uy);
    const double n4 = (kxx - kyy) - r.rho * (ux * ux - uy * uy);
    const double n5 = kxy - r.rho * ux * uy;
    const double div = -1.5 * a.om[0] * n3, dif = -1.5 * a.om[1] * n4;
    out[n] = 0.5 * (div + dif);
    out[p + n] = 0.5 * (div - dif);
    out[2 * p + n] = -3.0 * a.om[2] * n5;
}

__device__ __forceinline__ double block_sum(double v, double* sh) {
    for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    __syncthreads();
    if (lane == 0) sh[warp] = v;
    __syncthreads();
    double t = 0.0;
    if (threadIdx.x == 0)
        for (int w = 0; w < (int)(blockDim.x >> 5); ++w) t += sh[w];
    return t;  // valid in thread 0
}

template <int STORE>
__global__ void stats_kernel(const Args a, bool odd, int force, bool ffd, double* partials) {
    __shared__ double sh[kAuxThreads / 32];
    double s0 = 0.0, s1 = 0.0, s2 = 0.0;
    const long long total = (long long)a.nx * a.ny;
    for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < total;
         i += (long long)gridDim.x * blockDim.x) {
        const int y = int(i / a.nx), x = int(i - (long long)y * a.nx);
        const NodeMacros r = node_macros<STORE>(a, odd, force, ffd, x, y);
        s0 += r.rho; s1 += r.mx; s2 += r.my;
    }
    s0 = block_sum(s0, sh);
    s1 = block_sum(s1, sh);
    s2 = block_sum(s2, sh);
    if (threadIdx.x == 0) {
        partials[blockIdx.x] = s0;
        partials[gridDim.x + blockIdx.x] = s1;
        partials[2 * gridDim.x + blockIdx.x] = s2;
    }
}

// Sums the per-block partials in a fixed order (deterministic).
__global__ void stats_finish_kernel(const double* partials, int nb, double* out) {
    __shared__ double sh[kAuxThreads / 32];
    for (int k = 0; k < 3; ++k) {
        double v = 0.0;
        for (int i = threadIdx.x; i < nb; i += blockDim.x) v += partials[k * nb + i];
        v = block_sum(v, sh);
        if (threadIdx.x == 0) out[k] = v;
    }
}

__global__ void narrow_kernel(const double* src, float* dst, size_t n) {
    for (size_t i = (size_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (size_t)gridDim.x * blockDim.x)
        dst[i] = float(src[i]);
}

dim3 node_grid(const Args& a) { return dim3((a.nx + kAuxThreads - 1) / kAuxThreads, a.ny); }

}  // namespace

#define LBM_STORE_SWITCH(store, CALL)                       \
    switch (store) {                                        \
        case LBM_F64: { constexpr int ST = LBM_F64; CALL; } break;        \
        case LBM_F32: { constexpr int ST = LBM_F32; CALL; } break;        \
        case LBM_BF16DEV: { constexpr int ST = LBM_BF16DEV; CALL; } break; \
        default: { constexpr int ST = LBM_F16DEV; CALL; } break;           \
    }

cudaError_t launch_init(const Args& a, int store, int model, int force, const double* rho, const double* u,
                        cudaStream_t s) {
    const bool ffd = store == LBM_F64;
    LBM_STORE_SWITCH(store, (init_kernel<ST><<<node_grid(a), kAuxThreads, 0, s>>>(a, model, force, ffd, rho, u)));
    return cudaGetLastError();
}

cudaError_t launch_set_f(const Args& a, int store, const double* f, cudaStream_t s) {
    LBM_STORE_SWITCH(store, (set_f_kernel<ST><<<node_grid(a), kAuxThreads, 0, s>>>(a, f)));
    return cudaGetLastError();
}

cudaError_t launch_get_f(const Args& a, int store, bool odd, bool /*walls*/, double* f, cudaStream_t s) {
    LBM_STORE_SWITCH(store, (get_f_kernel<ST><<<node_grid(a), kAuxThreads, 0, s>>>(a, odd, f)));
    return cudaGetLastError();
}

cudaError_t launch_macros(const Args& a, int store, bool odd, bool /*walls*/, int force, double* rho, double* u,
                          cudaStream_t s) {
    const bool ffd = store == LBM_F64;
    LBM_STORE_SWITCH(store, (macros_kernel<ST><<<node_grid(a), kAuxThreads, 0, s>>>(a, odd, force, ffd, rho, u)));
    return cudaGetLastError();
}

cudaError_t launch_strain(const Args& a, int store, bool odd, bool /*walls*/, int force, double* out,
                          cudaStream_t s) {
    const bool ffd = store == LBM_F64;
    LBM_STORE_SWITCH(store, (strain_kernel<ST><<<node_grid(a), kAuxThreads, 0, s>>>(a, odd, force, ffd, out)));
    return cudaGetLastError();
}

cudaError_t launch_narrow(const double* src, float* dst, size_t n, cudaStream_t s) {
    const size_t nb = (n + kAuxThreads - 1) / kAuxThreads;
    narrow_kernel<<<unsigned(nb < 4096 ? (nb ? nb : 1) : 4096), kAuxThreads, 0, s>>>(src, dst, n);
    return cudaGetLastError();
}

int stats_blocks(const Args& a) {
    const long long total = (long long)a.nx * a.ny;
    long long nb = (total + kAuxThreads - 1) / kAuxThreads;
    return int(nb < 1216 ? nb : 1216);  // 152 SMs x 8 resident blocks
}

cudaError_t launch_stats(const Args& a, int store, bool odd, bool /*walls*/, int force, double* partials,
                         double* out, cudaStream_t s) {
    const bool ffd = store == LBM_F64;
    const int nb = stats_blocks(a);
    LBM_STORE_SWITCH(store, (stats_kernel<ST><<<nb, kAuxThreads, 0, s>>>(a, odd, force, ffd, partials)));
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    stats_finish_kernel<<<1, kAuxThreads, 0, s>>>(partials, nb, out);
    return cudaGetLastError();
}

}  // namespace lbm
