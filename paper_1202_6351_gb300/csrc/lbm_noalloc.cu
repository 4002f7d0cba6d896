// lbm_noalloc.cu -- lbm_stats_noalloc: the global FP64 sums of lbm_stats for
// callers that cannot allocate device memory.
//
// Some callers cannot call cudaMalloc: code that runs inside another
// framework's memory pool or under a strict memory budget where every device
// allocation must go through the host application, and drivers that forbid
// allocation after start-up.  This entry point allocates nothing: the caller
// passes the population array and the output, and the per-row partial sums
// live in a file-scope __device__ array of fixed size (kMaxRows rows), which
// every GPU that loads this library holds until the process exits.
#include <cuda.h>

#include <mutex>

#include "lbm.h"
#include "lbm_internal.h"

namespace lbm {
namespace {

constexpr int kThreads = 256;
constexpr int kMaxRows = LBM_NOALLOC_MAX_ROWS;
constexpr int kMaxDevices = 64;

// Per-row partial sums [3][kMaxRows]: sum rho, sum rho u_x, sum rho u_y of row y.
// Every call overwrites the rows it uses before reading them, so nothing needs
// to start at zero; the array keeps the last call's values.
static __device__ __align__(256) double g_row_partials[3 * kMaxRows];

std::mutex g_setup_mutex;

// The device address of g_row_partials belongs to the CUDA context that loaded
// this module: a device reset (cudaDeviceReset) destroys the primary context,
// and the next one may place the array elsewhere.  The address is therefore
// cached per device together with the id of the context it was looked up in,
// and looked up again (once) whenever that id changes.
struct PartialsCache {
    unsigned long long ctx_id = 0;
    double* addr = nullptr;
};
PartialsCache g_partials[kMaxDevices];

using CtxGetCurrentFn = CUresult(CUDAAPI*)(CUcontext*);
using CtxGetIdFn = CUresult(CUDAAPI*)(CUcontext, unsigned long long*);

// Id of the current context through the driver entry points (the library does
// not link the driver library itself).
cudaError_t current_context_id(unsigned long long* id) {
    static CtxGetCurrentFn get_current = nullptr;
    static CtxGetIdFn get_id = nullptr;
    if (!get_current || !get_id) {
        void* p = nullptr;
        cudaDriverEntryPointQueryResult q;
        cudaError_t e = cudaGetDriverEntryPointByVersion("cuCtxGetCurrent", &p, 12000, cudaEnableDefault, &q);
        if (e != cudaSuccess || q != cudaDriverEntryPointSuccess || !p) return e != cudaSuccess ? e : cudaErrorUnknown;
        get_current = reinterpret_cast<CtxGetCurrentFn>(p);
        e = cudaGetDriverEntryPointByVersion("cuCtxGetId", &p, 12000, cudaEnableDefault, &q);
        if (e != cudaSuccess || q != cudaDriverEntryPointSuccess || !p) return e != cudaSuccess ? e : cudaErrorUnknown;
        get_id = reinterpret_cast<CtxGetIdFn>(p);
    }
    CUcontext ctx = nullptr;
    if (get_current(&ctx) != CUDA_SUCCESS || !ctx) return cudaErrorDeviceUninitialized;
    if (get_id(ctx, id) != CUDA_SUCCESS) return cudaErrorUnknown;
    return cudaSuccess;
}

// Device address of g_row_partials on the current device (the symbol's
// host-side name is not a device address): looked up once per device, with
// that device current, and again only after its context has been replaced.
cudaError_t partials_address(int device, double** out) {
    std::lock_guard<std::mutex> lock(g_setup_mutex);
    PartialsCache& c = g_partials[device];
    unsigned long long id = 0;
    cudaError_t e = current_context_id(&id);
    if (e == cudaErrorDeviceUninitialized) {
        // No context is current yet: the runtime makes the device's primary
        // context current on its first call, here the lookup itself.
        void* p = nullptr;
        e = cudaGetSymbolAddress(&p, g_row_partials);
        if (e != cudaSuccess) return e;
        e = current_context_id(&id);
        if (e != cudaSuccess) return e;
        c.addr = static_cast<double*>(p);
        c.ctx_id = id;
    } else if (e != cudaSuccess) {
        return e;
    }
    if (c.ctx_id != id || !c.addr) {
        void* p = nullptr;
        e = cudaGetSymbolAddress(&p, g_row_partials);
        if (e != cudaSuccess) return e;
        c.addr = static_cast<double*>(p);
        c.ctx_id = id;
    }
    *out = c.addr;
    return cudaSuccess;
}

__device__ __forceinline__ double block_sum(double v, double* sh) {
    for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
    __syncthreads();
    if ((threadIdx.x & 31) == 0) sh[threadIdx.x >> 5] = v;
    __syncthreads();
    double t = 0.0;
    if (threadIdx.x == 0)
        for (int w = 0; w < kThreads / 32; ++w) t += sh[w];
    return t;
}

// One block per row y: sums of rho and rho u (Eq. 26-27, with F/2) over the row.
template <int STORE>
__global__ void __launch_bounds__(kThreads) row_sums_kernel(const Args a, bool odd, double* partials) {
    __shared__ double sh[kThreads / 32];
    const int y = blockIdx.x;
    double s0 = 0.0, s1 = 0.0, s2 = 0.0;
    for (int x = threadIdx.x; x < a.nx; x += kThreads) {
        typename Store<STORE>::R r[9];
        if (odd) load_node<STORE, true, true>(a, x, y, r);
        else load_node<STORE, false, true>(a, x, y, r);
        double d[9];
        constexpr double inv = 1.0 / Store<STORE>::scale;
#pragma unroll
        for (int q = 0; q < 9; ++q) d[q] = double(r[q]) * inv;
        const Moments<double> m = moments<double>(d, a.rho0);
        s0 += m.rho;
        s1 += m.jx + 0.5 * a.F[0];
        s2 += m.jy + 0.5 * a.F[1];
    }
    s0 = block_sum(s0, sh);
    s1 = block_sum(s1, sh);
    s2 = block_sum(s2, sh);
    if (threadIdx.x == 0) {
        partials[y] = s0;
        partials[kMaxRows + y] = s1;
        partials[2 * kMaxRows + y] = s2;
    }
}

// Sums the row partials in a fixed order (deterministic) into out[3].
__global__ void __launch_bounds__(kThreads) rows_finish_kernel(const double* partials, int ny, double* out) {
    __shared__ double sh[kThreads / 32];
    for (int k = 0; k < 3; ++k) {
        double v = 0.0;
        for (int y = threadIdx.x; y < ny; y += kThreads) v += partials[k * kMaxRows + y];
        v = block_sum(v, sh);
        if (threadIdx.x == 0) out[k] = v;
    }
}

}  // namespace
}  // namespace lbm

extern "C" int lbm_stats_noalloc(const void* f, const lbm_layout_t* layout, double* out, void* stream) {
    using namespace lbm;
    auto fail = [](int code, const char* msg) { return set_error(code, "lbm_stats_noalloc: %s", msg); };
    if (!f || !layout || !out) return fail(LBM_EINVAL, "f, layout and out must not be NULL");
    const lbm_layout_t& L = *layout;
    if (L.nx < 1 || L.ny < 1) return fail(LBM_EINVAL, "nx and ny must be >= 1");
    if (L.ny > kMaxRows) return fail(LBM_EINVAL, "ny exceeds LBM_NOALLOC_MAX_ROWS (16384), the rows the static scratch holds");
    if (L.pitch < L.nx || (long long)L.pitch * L.ny > 0x7fffffffLL) return fail(LBM_EINVAL, "pitch must be >= nx and pitch * ny < 2^31");
    if (L.store < LBM_F64 || L.store > LBM_F16DEV) return fail(LBM_EINVAL, "unknown storage kind");
    if (!(L.rho0 > 0.0)) return fail(LBM_EINVAL, "rho0 must be positive");
    for (int k = 0; k < 4; ++k)
        if (L.bc.edge[k] < LBM_PERIODIC || L.bc.edge[k] > LBM_MOVING_WALL) return fail(LBM_EINVAL, "unknown edge kind");
    // the pairing lbm_create enforces: opposite edges both periodic or both walls
    if ((L.bc.edge[LBM_WEST] == LBM_PERIODIC) != (L.bc.edge[LBM_EAST] == LBM_PERIODIC))
        return fail(LBM_EINVAL, "west and east edges must both be periodic or both be walls");
    if ((L.bc.edge[LBM_SOUTH] == LBM_PERIODIC) != (L.bc.edge[LBM_NORTH] == LBM_PERIODIC))
        return fail(LBM_EINVAL, "south and north edges must both be periodic or both be walls");

    int device = 0;
    if (cudaGetDevice(&device) != cudaSuccess || device < 0 || device >= kMaxDevices)
        return fail(LBM_ECUDA, "no usable current CUDA device");
    double* partials = nullptr;
    if (partials_address(device, &partials) != cudaSuccess)
        return fail(LBM_ECUDA, "cannot look up the device address of the static scratch");

    Args a{};
    a.f = const_cast<void*>(f);
    a.nx = L.nx;
    a.ny = L.ny;
    a.pitch = L.pitch;
    a.plane = (long long)L.pitch * L.ny;
    a.rho0 = L.rho0;
    a.F[0] = L.force[0];
    a.F[1] = L.force[1];
    a.scale = store_scale(L.store);
    for (int k = 0; k < 6; ++k) a.om[k] = 1.0;  // unused by the sums
    for (int k = 0; k < 4; ++k) {
        a.wall[k] = L.bc.edge[k] != LBM_PERIODIC;
        const double U = L.bc.edge[k] == LBM_MOVING_WALL ? L.bc.wall_u[k] : 0.0;
        a.wallx[k] = k >= LBM_SOUTH ? 6.0 * L.rho0 * U : 0.0;
        a.wally[k] = k >= LBM_SOUTH ? 0.0 : 6.0 * L.rho0 * U;
    }
    prepare_constants(a);
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    const bool odd = L.odd != 0;
    switch (L.store) {
        case LBM_F64: row_sums_kernel<LBM_F64><<<L.ny, kThreads, 0, s>>>(a, odd, partials); break;
        case LBM_F32: row_sums_kernel<LBM_F32><<<L.ny, kThreads, 0, s>>>(a, odd, partials); break;
        case LBM_BF16DEV: row_sums_kernel<LBM_BF16DEV><<<L.ny, kThreads, 0, s>>>(a, odd, partials); break;
        default: row_sums_kernel<LBM_F16DEV><<<L.ny, kThreads, 0, s>>>(a, odd, partials); break;
    }
    if (cudaGetLastError() != cudaSuccess) return fail(LBM_ECUDA, "row-sum kernel launch failed");
    rows_finish_kernel<<<1, kThreads, 0, s>>>(partials, L.ny, out);
    if (cudaGetLastError() != cudaSuccess) return fail(LBM_ECUDA, "finish kernel launch failed");
    return LBM_OK;
}
