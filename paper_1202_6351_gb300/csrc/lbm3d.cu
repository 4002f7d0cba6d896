// lbm3d.cu -- D3Q27 central-moment lattices: the kernels and the extern "C"
// entry points declared in include/lbm3d.h.
//
// One thread per node, AA-pattern streaming in place on one array
// f[27][nz][ny][pitch] (periodic in x, y and z), the collision of
// lbm3d_device.cuh in registers.  FP64 storage (parity build) and FP32
// deviations; FP32 arithmetic for FP32 storage.
#include <cmath>
#include <cstring>
#include <type_traits>

#include "lbm3d.h"
#include "lbm3d_device.cuh"
#include "lbm_internal.h"

using lbm3::Args3;

namespace {

constexpr int kBX = 128, kBY = 2;

template <int STORE, bool ODD, bool FORCED>
__global__ void __launch_bounds__(kBX * kBY) step3_kernel(const Args3 a) {
    const int x = blockIdx.x * blockDim.x + threadIdx.x;
    const int y = blockIdx.y * blockDim.y + threadIdx.y;
    const int z = blockIdx.z;
    if (x >= a.nx || y >= a.ny) return;
    typename lbm::Store<STORE>::R d[27];
    lbm3::load3<STORE, ODD>(a, x, y, z, d);
    lbm3::collide3<typename lbm::Store<STORE>::R, FORCED>(d, a);
    lbm3::store3<STORE, ODD>(a, x, y, z, d);
}

// rho [nz][ny][nx], u [3][nz][ny][nx] (FP64, device; either may be null: rho0 / rest)
template <int STORE>
__global__ void __launch_bounds__(kBX * kBY) init3_kernel(const Args3 a, const double* rho, const double* u) {
    using S = lbm::Store<STORE>;
    using R = typename S::R;
    using T = typename S::T;
    const int x = blockIdx.x * blockDim.x + threadIdx.x;
    const int y = blockIdx.y * blockDim.y + threadIdx.y;
    const int z = blockIdx.z;
    if (x >= a.nx || y >= a.ny) return;
    const long long p = ((long long)z * a.ny + y) * a.nx + x, n = (long long)a.nx * a.ny * a.nz;
    const R* k = lbm3::kconst3<R>(a);
    const R rho0 = k[lbm3::K3_RHO0];
    const R drho = rho ? R((rho[p] - a.kd[lbm3::K3_RHO0]) * a.scale) : R(0);  // stored units
    const R ux = u ? R(u[p]) : R(0), uy = u ? R(u[n + p]) : R(0), uz = u ? R(u[2 * n + p]) : R(0);
    R d[27];
    lbm3::equilibrium3<R>(d, rho0, drho, ux, uy, uz, k[lbm3::K3_FX], k[lbm3::K3_FY], k[lbm3::K3_FZ]);
    T* f = static_cast<T*>(a.f);
    const long long o = lbm3::node_off<T>(a, x, y, z);
#pragma unroll
    for (int q = 0; q < 27; ++q) f[q * a.plane + o] = S::enc(d[q]);
}

// The 27 populations of every node at the current time, as full FP64 values
// f = d + w rho0 in the natural layout [27][nz][ny][nx].
template <int STORE>
__global__ void __launch_bounds__(kBX * kBY) get3_kernel(const Args3 a, bool odd, double* out) {
    using S = lbm::Store<STORE>;
    using R = typename S::R;
    const int x = blockIdx.x * blockDim.x + threadIdx.x;
    const int y = blockIdx.y * blockDim.y + threadIdx.y;
    const int z = blockIdx.z;
    if (x >= a.nx || y >= a.ny) return;
    R d[27];
    if (odd) lbm3::load3<STORE, true>(a, x, y, z, d);
    else lbm3::load3<STORE, false>(a, x, y, z, d);
    const long long p = ((long long)z * a.ny + y) * a.nx + x, n = (long long)a.nx * a.ny * a.nz;
#pragma unroll
    for (int q = 0; q < 27; ++q) out[q * n + p] = double(d[q]) / a.scale + lbm3::wgt<double>(q) * a.kd[lbm3::K3_RHO0];
}

template <int STORE>
__global__ void __launch_bounds__(kBX * kBY) set3_kernel(const Args3 a, const double* in) {
    using S = lbm::Store<STORE>;
    using T = typename S::T;
    const int x = blockIdx.x * blockDim.x + threadIdx.x;
    const int y = blockIdx.y * blockDim.y + threadIdx.y;
    const int z = blockIdx.z;
    if (x >= a.nx || y >= a.ny) return;
    const long long p = ((long long)z * a.ny + y) * a.nx + x, n = (long long)a.nx * a.ny * a.nz;
    T* f = static_cast<T*>(a.f);
    const long long o = lbm3::node_off<T>(a, x, y, z);
#pragma unroll
    for (int q = 0; q < 27; ++q)
        f[q * a.plane + o] = S::enc(typename S::R((in[q * n + p] - lbm3::wgt<double>(q) * a.kd[lbm3::K3_RHO0]) * a.scale));
}

// rho, u (Eq. 26-27 in 3-D, with F/2) into FP64 device arrays (either may be null).
template <int STORE>
__global__ void __launch_bounds__(kBX * kBY) macros3_kernel(const Args3 a, bool odd, double* rho, double* u) {
    using S = lbm::Store<STORE>;
    using R = typename S::R;
    const int x = blockIdx.x * blockDim.x + threadIdx.x;
    const int y = blockIdx.y * blockDim.y + threadIdx.y;
    const int z = blockIdx.z;
    if (x >= a.nx || y >= a.ny) return;
    R d[27];
    if (odd) lbm3::load3<STORE, true>(a, x, y, z, d);
    else lbm3::load3<STORE, false>(a, x, y, z, d);
    double drho = 0.0, j[3] = {0.0, 0.0, 0.0};
#pragma unroll
    for (int q = 0; q < 27; ++q) {
        const double v = double(d[q]);
        drho += v;
        j[0] += lbm3::ex(q) * v;
        j[1] += lbm3::ey(q) * v;
        j[2] += lbm3::ez(q) * v;
    }
    drho /= a.scale;
    for (int k = 0; k < 3; ++k) j[k] /= a.scale;
    const double r = a.kd[lbm3::K3_RHO0] + drho;
    const long long p = ((long long)z * a.ny + y) * a.nx + x, n = (long long)a.nx * a.ny * a.nz;
    if (rho) rho[p] = r;
    if (u) {
        u[p] = (j[0] + 0.5 * a.kd[lbm3::K3_FX]) / r;
        u[n + p] = (j[1] + 0.5 * a.kd[lbm3::K3_FY]) / r;
        u[2 * n + p] = (j[2] + 0.5 * a.kd[lbm3::K3_FZ]) / r;
    }
}

dim3 grid_of(const Args3& a) { return dim3((a.nx + kBX - 1) / kBX, (a.ny + kBY - 1) / kBY, a.nz); }

template <int STORE>
cudaError_t launch_step3(const Args3& a, bool odd, bool forced, cudaStream_t s) {
    const dim3 g = grid_of(a), b(kBX, kBY);
    if (odd) {
        if (forced) step3_kernel<STORE, true, true><<<g, b, 0, s>>>(a);
        else step3_kernel<STORE, true, false><<<g, b, 0, s>>>(a);
    } else {
        if (forced) step3_kernel<STORE, false, true><<<g, b, 0, s>>>(a);
        else step3_kernel<STORE, false, false><<<g, b, 0, s>>>(a);
    }
    return cudaGetLastError();
}

int fail(int code, const char* msg) { return lbm::set_error(code, "%s", msg); }

int cuda_fail(cudaError_t e, const char* what) {
    return lbm::set_error(e == cudaErrorMemoryAllocation ? LBM_ENOMEM : LBM_ECUDA, "%s: %s", what,
                          cudaGetErrorString(e));
}

}  // namespace

struct lbm3_s {
    int device = 0;
    int store = LBM_F32;
    Args3 a{};
    long t = 0;
    cudaStream_t stream = nullptr;
    void* state = nullptr;
    size_t state_bytes = 0;
    bool forced = false;
};

namespace {

size_t es3(int store) { return store == LBM_F64 ? 8 : (store == LBM_F32 ? 4 : 2); }

// fn(std::integral_constant<int, STORE>) for the lattice's storage kind.
template <typename Fn>
void with_store(int store, Fn&& fn) {
    switch (store) {
        case LBM_F64: fn(std::integral_constant<int, LBM_F64>()); break;
        case LBM_F32: fn(std::integral_constant<int, LBM_F32>()); break;
        case LBM_BF16DEV: fn(std::integral_constant<int, LBM_BF16DEV>()); break;
        default: fn(std::integral_constant<int, LBM_F16DEV>()); break;
    }
}

cudaError_t run_init(lbm3_s* h, const double* rho, const double* u) {
    const dim3 g = grid_of(h->a), b(kBX, kBY);
    with_store(h->store, [&](auto st) { init3_kernel<decltype(st)::value><<<g, b, 0, h->stream>>>(h->a, rho, u); });
    return cudaGetLastError();
}

// Host buffer of `bytes` through a stream-ordered device copy.
struct Staging {
    void* p = nullptr;
    cudaStream_t s;
    explicit Staging(cudaStream_t st) : s(st) {}
    cudaError_t alloc(size_t bytes) { return cudaMallocAsync(&p, bytes, s); }
    ~Staging() { if (p) cudaFreeAsync(p, s); }
};

#define L3_CUDA(call, what)                                \
    do {                                                   \
        cudaError_t e_ = (call);                           \
        if (e_ != cudaSuccess) return cuda_fail(e_, what); \
    } while (0)

#define L3_HANDLE(h)                                                                 \
    if (!(h)) return fail(LBM_EINVAL, "null D3Q27 lattice handle");                  \
    int prev_dev_ = -1;                                                              \
    cudaGetDevice(&prev_dev_);                                                       \
    if (prev_dev_ != (h)->device && cudaSetDevice((h)->device) != cudaSuccess)       \
        return fail(LBM_ECUDA, "cannot select the lattice's device");                \
    struct Restore_ {                                                                \
        int d;                                                                       \
        ~Restore_() { if (d >= 0) cudaSetDevice(d); }                                \
    } restore_{prev_dev_ != (h)->device ? prev_dev_ : -1};

}  // namespace

extern "C" {

int lbm3_create(int nx, int ny, int nz, const double omegas[6], const double force[3], int store, double rho0,
                lbm3_t* out) {
    if (!out) return fail(LBM_EINVAL, "lbm3_create: out is NULL");
    if (nx < 1 || ny < 1 || nz < 1) return fail(LBM_EINVAL, "lbm3_create: nx, ny and nz must be >= 1");
    if (nz > 65535) return fail(LBM_EINVAL, "lbm3_create: nz exceeds 65535");
    const long long pitch = (nx + 31) / 32 * 32;
    if (pitch * ny * nz > 0x7fffffffLL) return fail(LBM_EINVAL, "lbm3_create: padded plane exceeds 2^31 - 1 elements");
    if (!omegas) return fail(LBM_EINVAL, "lbm3_create: omegas is NULL");
    for (int k = 0; k < 6; ++k)
        if (!(omegas[k] > 0.0 && omegas[k] < 2.0)) return fail(LBM_EINVAL, "lbm3_create: every omega must lie in (0, 2)");
    if (store != LBM_F64 && store != LBM_F32 && store != LBM_BF16DEV && store != LBM_F16DEV)
        return fail(LBM_EINVAL, "lbm3_create: storage must be LBM_F64, LBM_F32, LBM_BF16DEV or LBM_F16DEV");
    if (!(rho0 > 0.0 && std::isfinite(rho0))) return fail(LBM_EINVAL, "lbm3_create: rho0 must be positive and finite");
    if (force && !(std::isfinite(force[0]) && std::isfinite(force[1]) && std::isfinite(force[2])))
        return fail(LBM_EINVAL, "lbm3_create: force must be finite");
    lbm3_s* h = new lbm3_s;
    if (cudaGetDevice(&h->device) != cudaSuccess) {
        delete h;
        return fail(LBM_ECUDA, "lbm3_create: no CUDA device available");
    }
    h->store = store;
    Args3& a = h->a;
    a.nx = nx;
    a.ny = ny;
    a.nz = nz;
    a.pitch = int(pitch);
    a.plane = pitch * ny * nz;
    for (int k = 0; k < 6; ++k) a.kd[k] = omegas[k];
    a.kd[lbm3::K3_RHO0] = rho0;
    for (int k = 0; k < 3; ++k) a.kd[lbm3::K3_FX + k] = force ? force[k] : 0.0;
    a.scale = lbm::store_scale(store);
    for (int k = 0; k < 10; ++k) a.kf[k] = float(k >= lbm3::K3_RHO0 ? a.kd[k] * a.scale : a.kd[k]);
    h->forced = force && (force[0] != 0.0 || force[1] != 0.0 || force[2] != 0.0);
    h->state_bytes = 27 * size_t(a.plane) * es3(store);
    cudaError_t e = cudaMalloc(&h->state, h->state_bytes);
    if (e == cudaSuccess) e = cudaMemset(h->state, 0, h->state_bytes);  // deviation 0: the rest state w rho0
    if (e == cudaSuccess) e = cudaDeviceSynchronize();
    if (e != cudaSuccess) {
        if (h->state) cudaFree(h->state);
        delete h;
        return cuda_fail(e, "lbm3_create");
    }
    a.f = h->state;
    *out = h;
    return LBM_OK;
}

int lbm3_destroy(lbm3_t h) {
    if (!h) return LBM_OK;
    int prev = -1;
    cudaGetDevice(&prev);
    if (prev != h->device) cudaSetDevice(h->device);
    if (h->stream) cudaStreamSynchronize(h->stream);
    else cudaDeviceSynchronize();
    if (h->state) cudaFree(h->state);
    const cudaError_t e = cudaGetLastError();
    if (prev >= 0 && prev != h->device) cudaSetDevice(prev);
    delete h;
    return e == cudaSuccess ? LBM_OK : cuda_fail(e, "lbm3_destroy");
}

int lbm3_set_stream(lbm3_t h, void* stream) {
    L3_HANDLE(h);
    h->stream = static_cast<cudaStream_t>(stream);
    return LBM_OK;
}

int lbm3_init(lbm3_t h, const double* rho, const double* u) {
    L3_HANDLE(h);
    const size_t n = size_t(h->a.nx) * h->a.ny * h->a.nz;
    Staging buf(h->stream);
    double* drho = nullptr;
    double* du = nullptr;
    if (rho || u) {
        L3_CUDA(buf.alloc(4 * n * sizeof(double)), "lbm3_init staging");
        drho = static_cast<double*>(buf.p);
        du = drho + n;
        if (rho) L3_CUDA(cudaMemcpyAsync(drho, rho, n * sizeof(double), cudaMemcpyHostToDevice, h->stream), "rho copy");
        if (u) L3_CUDA(cudaMemcpyAsync(du, u, 3 * n * sizeof(double), cudaMemcpyHostToDevice, h->stream), "u copy");
    }
    L3_CUDA(run_init(h, rho ? drho : nullptr, u ? du : nullptr), "lbm3_init kernel");
    L3_CUDA(cudaStreamSynchronize(h->stream), "lbm3_init sync");
    h->t = 0;
    return LBM_OK;
}

int lbm3_step(lbm3_t h, long n) {
    L3_HANDLE(h);
    if (n < 0) return fail(LBM_EINVAL, "lbm3_step: n must be >= 0");
    for (long s = 0; s < n; ++s) {
        const bool odd = (h->t & 1) != 0;
        cudaError_t e = cudaSuccess;
        with_store(h->store, [&](auto st) { e = launch_step3<decltype(st)::value>(h->a, odd, h->forced, h->stream); });
        if (e != cudaSuccess) return cuda_fail(e, "lbm3_step launch");
        ++h->t;
    }
    return LBM_OK;
}

int lbm3_macros(lbm3_t h, double* rho, double* u) {
    L3_HANDLE(h);
    if (!rho && !u) return LBM_OK;
    const size_t n = size_t(h->a.nx) * h->a.ny * h->a.nz;
    Staging buf(h->stream);
    L3_CUDA(buf.alloc(4 * n * sizeof(double)), "lbm3_macros staging");
    double* drho = static_cast<double*>(buf.p);
    double* du = drho + n;
    const dim3 g = grid_of(h->a), b(kBX, kBY);
    const bool odd = (h->t & 1) != 0;
    with_store(h->store, [&](auto st) { macros3_kernel<decltype(st)::value><<<g, b, 0, h->stream>>>(h->a, odd, drho, du); });
    L3_CUDA(cudaGetLastError(), "lbm3_macros kernel");
    if (rho) L3_CUDA(cudaMemcpyAsync(rho, drho, n * sizeof(double), cudaMemcpyDeviceToHost, h->stream), "rho copy");
    if (u) L3_CUDA(cudaMemcpyAsync(u, du, 3 * n * sizeof(double), cudaMemcpyDeviceToHost, h->stream), "u copy");
    L3_CUDA(cudaStreamSynchronize(h->stream), "lbm3_macros sync");
    return LBM_OK;
}

int lbm3_get_f(lbm3_t h, double* f) {
    L3_HANDLE(h);
    if (!f) return fail(LBM_EINVAL, "lbm3_get_f: f is NULL");
    const size_t n = 27 * size_t(h->a.nx) * h->a.ny * h->a.nz;
    Staging buf(h->stream);
    L3_CUDA(buf.alloc(n * sizeof(double)), "lbm3_get_f staging");
    const dim3 g = grid_of(h->a), b(kBX, kBY);
    const bool odd = (h->t & 1) != 0;
    with_store(h->store, [&](auto st) {
        get3_kernel<decltype(st)::value><<<g, b, 0, h->stream>>>(h->a, odd, static_cast<double*>(buf.p));
    });
    L3_CUDA(cudaGetLastError(), "lbm3_get_f kernel");
    L3_CUDA(cudaMemcpyAsync(f, buf.p, n * sizeof(double), cudaMemcpyDeviceToHost, h->stream), "f copy");
    L3_CUDA(cudaStreamSynchronize(h->stream), "lbm3_get_f sync");
    return LBM_OK;
}

int lbm3_set_f(lbm3_t h, const double* f) {
    L3_HANDLE(h);
    if (!f) return fail(LBM_EINVAL, "lbm3_set_f: f is NULL");
    const size_t n = 27 * size_t(h->a.nx) * h->a.ny * h->a.nz;
    Staging buf(h->stream);
    L3_CUDA(buf.alloc(n * sizeof(double)), "lbm3_set_f staging");
    L3_CUDA(cudaMemcpyAsync(buf.p, f, n * sizeof(double), cudaMemcpyHostToDevice, h->stream), "f copy");
    const dim3 g = grid_of(h->a), b(kBX, kBY);
    with_store(h->store, [&](auto st) {
        set3_kernel<decltype(st)::value><<<g, b, 0, h->stream>>>(h->a, static_cast<const double*>(buf.p));
    });
    L3_CUDA(cudaGetLastError(), "lbm3_set_f kernel");
    L3_CUDA(cudaStreamSynchronize(h->stream), "lbm3_set_f sync");
    h->t = 0;
    return LBM_OK;
}

long lbm3_time(lbm3_t h) { return h ? h->t : -1; }

int lbm3_info(lbm3_t h, long dims[5], size_t* bytes, void** state) {
    if (!h) return fail(LBM_EINVAL, "null D3Q27 lattice handle");
    if (dims) {
        dims[0] = h->a.nx;
        dims[1] = h->a.ny;
        dims[2] = h->a.nz;
        dims[3] = h->a.pitch;
        dims[4] = h->store;
    }
    if (bytes) *bytes = h->state_bytes;
    if (state) *state = h->state;
    return LBM_OK;
}

size_t lbm3_bytes_per_update(int store) {
    return (store == LBM_F64 || store == LBM_F32 || store == LBM_BF16DEV || store == LBM_F16DEV) ? 54 * es3(store) : 0;
}

}  // extern "C"
