// lbm_capi.cu -- the extern "C" boundary declared in include/lbm.h.
//
// Validates arguments, owns the device memory of a lattice, tracks the step
// counter (whose parity selects the AA-pattern kernel) and turns CUDA failures
// into status codes with a per-thread message.
#include <algorithm>
#include <cmath>
#include <cstdarg>
#include <cstdio>
#include <cstring>
#include <string>

#include "lbm.h"
#include "lbm_fused.cuh"
#include "lbm_internal.h"
#include "lbm_handle.h"

using lbm::Args;

namespace {

thread_local std::string g_error;

int fail(int code, const char* fmt, ...) {
    char buf[512];
    va_list ap;
    va_start(ap, fmt);
    vsnprintf(buf, sizeof buf, fmt, ap);
    va_end(ap);
    g_error = buf;
    return code;
}

int cuda_fail(cudaError_t e, const char* what) {
    return fail(e == cudaErrorMemoryAllocation ? LBM_ENOMEM : LBM_ECUDA, "%s: %s", what, cudaGetErrorString(e));
}

}  // namespace

int lbm::force_mode(const lbm_s* h) {
    if (h->has_field) return 2;
    return (h->a.F[0] != 0.0 || h->a.F[1] != 0.0) ? 1 : 0;
}

cudaError_t lbm::launch_step_any(const Args& a, int store, int model, bool odd, int force, bool walls,
                                 cudaStream_t s) {
    switch (store) {
        case LBM_F64: return launch_step_f64(a, model, odd, force, walls, s);
        case LBM_F32: return launch_step_f32(a, model, odd, force, walls, s);
        case LBM_BF16DEV: return launch_step_bf16(a, model, odd, force, walls, s);
        default: return launch_step_f16(a, model, odd, force, walls, s);
    }
}

int lbm::set_error(int code, const char* fmt, ...) {
    char buf[512];
    va_list ap;
    va_start(ap, fmt);
    vsnprintf(buf, sizeof buf, fmt, ap);
    va_end(ap);
    g_error = buf;
    return code;
}

namespace {

#define LBM_CUDA(call, what)                              \
    do {                                                  \
        cudaError_t e_ = (call);                          \
        if (e_ != cudaSuccess) return cuda_fail(e_, what); \
    } while (0)

// Makes the handle's device current for the duration of a call.
struct DeviceGuard {
    int prev = -1;
    bool ok = true;
    explicit DeviceGuard(int dev) {
        if (cudaGetDevice(&prev) != cudaSuccess) { ok = false; return; }
        if (prev != dev && cudaSetDevice(dev) != cudaSuccess) ok = false;
    }
    ~DeviceGuard() {
        int cur;
        if (prev >= 0 && cudaGetDevice(&cur) == cudaSuccess && cur != prev) cudaSetDevice(prev);
    }
};

size_t elem_size(int store) {
    switch (store) {
        case LBM_F64: return 8;
        case LBM_F32: return 4;
        case LBM_BF16DEV:
        case LBM_F16DEV: return 2;
        default: return 0;
    }
}

using lbm::force_mode;

// The single-step variant that stands in for variant 3 (two fused steps) where
// one step is taken alone: four nodes per thread for 16-bit stores, else one.
int single_variant(const lbm_s* h) {
    if (h->a.variant != 3) return h->a.variant;
    return (h->store == LBM_F16DEV || h->store == LBM_BF16DEV) ? 2 : 0;
}

cudaError_t launch_step_at(lbm_s* h, bool odd, long t) {
    if (h->a.rseed) {  // stochastic rounding: the hash of (seed, step) of this launch
        h->a.rbase = lbm::round_hash(h->a.rseed, static_cast<unsigned long long>(t));
        h->a.rtable = nullptr;
        h->a.tstep = 0;
    }
    lbm::Args a = h->a;
    a.variant = single_variant(h);
    return lbm::launch_step_any(a, h->store, h->model, odd, force_mode(h), h->walls, h->stream);
}

cudaError_t launch_step(lbm_s* h, bool odd) { return launch_step_at(h, odd, h->t); }

// ---------------------------------------------------------------- two fused steps (variant 3)

using EncodeTiledFn = CUresult(CUDAAPI*)(CUtensorMap*, CUtensorMapDataType, cuuint32_t, void*, const cuuint64_t*,
                                         const cuuint64_t*, const cuuint32_t*, const cuuint32_t*,
                                         CUtensorMapInterleave, CUtensorMapSwizzle, CUtensorMapL2promotion,
                                         CUtensorMapFloatOOBfill);

// cuTensorMapEncodeTiled through the runtime's driver entry point (the library
// does not link the driver library itself).
EncodeTiledFn encode_tiled() {
    static EncodeTiledFn fn = [] {
        void* p = nullptr;
        cudaDriverEntryPointQueryResult q;
        if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &p, 12000, cudaEnableDefault, &q) != cudaSuccess ||
            q != cudaDriverEntryPointSuccess)
            p = nullptr;
        return reinterpret_cast<EncodeTiledFn>(p);
    }();
    return fn;
}

template <int ST>
void fused_box(cuuint32_t box[3]) {
    box[0] = lbm::FusedGeom<ST>::BW;
    box[1] = lbm::FusedGeom<ST>::BH;
    box[2] = 9;
}

// TMA descriptor of a population array of the lattice: a 3-D tensor
// [9][ny][nx] (x fastest, row pitch `pitch`, plane pitch * ny), box = the
// fused kernel's region; coordinates beyond nx or ny read zeros.
cudaError_t encode_map(const lbm_s* h, void* base, CUtensorMap* map) {
    EncodeTiledFn fn = encode_tiled();
    if (!fn) return cudaErrorNotSupported;
    const size_t es = elem_size(h->store);
    const cuuint64_t dims[3] = {cuuint64_t(h->a.nx), cuuint64_t(h->a.ny), 9};
    const cuuint64_t strides[2] = {cuuint64_t(h->a.pitch) * es, cuuint64_t(h->a.plane) * es};
    cuuint32_t box[3];
    CUtensorMapDataType type;
    if (h->store == LBM_F32) {
        fused_box<LBM_F32>(box);
        type = CU_TENSOR_MAP_DATA_TYPE_FLOAT32;
    } else {
        fused_box<LBM_F16DEV>(box);
        type = CU_TENSOR_MAP_DATA_TYPE_UINT16;
    }
    const cuuint32_t estr[3] = {1, 1, 1};
    const CUresult r = fn(map, type, 3, base, dims, strides, box, estr, CU_TENSOR_MAP_INTERLEAVE_NONE,
                          CU_TENSOR_MAP_SWIZZLE_NONE, CU_TENSOR_MAP_L2_PROMOTION_L2_128B,
                          CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
    return r == CUDA_SUCCESS ? cudaSuccess : cudaErrorInvalidValue;
}

// The fused kernel runs on FP32 and 16-bit storage, lattices of at least 4 x 4
// nodes and without the divergence check (which needs the state every step).
bool fused_active(const lbm_s* h) {
    return h->a.variant == 3 && h->store != LBM_F64 && h->a.nx >= 4 && h->a.ny >= 4 && h->check_every == 0;
}

// Second population array, descriptors and error word (first use of variant 3).
cudaError_t ensure_fused(lbm_s* h) {
    cudaError_t e = cudaSuccess;
    if (!h->state_alt) e = cudaMalloc(&h->state_alt, h->state_bytes);
    if (e == cudaSuccess && !h->d_err) {
        e = cudaMalloc((void**)&h->d_err, sizeof(int));
        if (e == cudaSuccess) e = cudaMemset(h->d_err, 0, sizeof(int));
    }
    // The two arrays only ever swap roles, so one descriptor each, made once.
    if (e == cudaSuccess && !h->tmap_ptr[0]) {
        e = encode_map(h, h->state, &h->tmap[0]);
        if (e == cudaSuccess) e = encode_map(h, h->state_alt, &h->tmap[1]);
        if (e == cudaSuccess) {
            h->tmap_ptr[0] = h->state;
            h->tmap_ptr[1] = h->state_alt;
        }
    }
    return e;
}

const CUtensorMap& map_of(const lbm_s* h, const void* base) { return h->tmap[h->tmap_ptr[0] == base ? 0 : 1]; }

// Two steps from a.f (natural layout, t even) into `out`, the other array.
cudaError_t launch_fused(lbm_s* h, const lbm::Args& a, void* out, cudaStream_t s) {
    const CUtensorMap& map = map_of(h, a.f);
    switch (h->store) {
        case LBM_F32: return lbm::launch_fused_f32(map, a, out, h->d_err, h->model, force_mode(h), h->walls, s);
        case LBM_BF16DEV: return lbm::launch_fused_bf16(map, a, out, h->d_err, h->model, force_mode(h), h->walls, s);
        default: return lbm::launch_fused_f16(map, a, out, h->d_err, h->model, force_mode(h), h->walls, s);
    }
}

void swap_arrays(lbm_s* h) {
    std::swap(h->state, h->state_alt);
    h->a.f = h->state;
}

// Two fused steps t, t + 1 (t even) outside a graph.
cudaError_t launch_pair_at(lbm_s* h, long t) {
    lbm::Args a = h->a;
    if (a.rseed) {
        a.rbase = lbm::round_hash(a.rseed, static_cast<unsigned long long>(t));
        a.rbase1 = lbm::round_hash(a.rseed, static_cast<unsigned long long>(t + 1));
        a.rtable = nullptr;
        a.tstep = 0;
    }
    cudaError_t e = launch_fused(h, a, h->state_alt, h->stream);
    if (e == cudaSuccess) swap_arrays(h);
    return e;
}

// Error word of the fused kernel (a tile load that timed out), read after a
// synchronisation; cleared once reported.
int fused_error(lbm_s* h) {
    if (!h->d_err) return LBM_OK;
    int v = 0;
    if (cudaMemcpy(&v, h->d_err, sizeof(int), cudaMemcpyDeviceToHost) != cudaSuccess) return LBM_ECUDA;
    if (v == 0) return LBM_OK;
    cudaMemset(h->d_err, 0, sizeof(int));
    return lbm::set_error(LBM_ECUDA, "a fused two-step launch timed out waiting for its tile load; the state is invalid");
}

// Steps per graph replay: a multiple of 4 with fused steps (an even number of
// fused launches ends on the array the graph started from).
int graph_len(const lbm_s* h) { return fused_active(h) ? (h->graph_steps / 4) * 4 : h->graph_steps; }

// rtable[k] = the hash of (seed, t0 + k) for the k-th launch of a graph replay.
__global__ void fill_round_table(unsigned* rtable, unsigned long long seed, unsigned long long t0, int n) {
    const int k = blockIdx.x * blockDim.x + threadIdx.x;
    if (k < n) rtable[k] = lbm::round_hash(seed, t0 + static_cast<unsigned long long>(k));
}

long long nodes(const lbm_s* h) { return (long long)h->a.nx * h->a.ny; }

// Stream-ordered temporary device buffer for host-pointer calls.
struct DevBuf {
    void* p = nullptr;
    cudaStream_t s;
    explicit DevBuf(cudaStream_t st) : s(st) {}
    cudaError_t alloc(size_t bytes) { return cudaMallocAsync(&p, bytes, s); }
    ~DevBuf() { if (p) cudaFreeAsync(p, s); }
};

// True if two argument blocks launch the same step kernels on the same data.
bool same_launch(const Args& x, const Args& y) {
    if (x.f != y.f || x.fo != y.fo || x.plane != y.plane || x.nx != y.nx || x.ny != y.ny || x.pitch != y.pitch)
        return false;
    if (x.ffield != y.ffield || x.variant != y.variant || x.block_x != y.block_x || x.scale != y.scale) return false;
    if (x.rseed != y.rseed) return false;
    for (int k = 0; k < 4; ++k)
        if (x.wall[k] != y.wall[k] || x.wallx[k] != y.wallx[k] || x.wally[k] != y.wally[k] ||
            x.wallxf[k] != y.wallxf[k] || x.wallyf[k] != y.wallyf[k])
            return false;
    for (int k = 0; k < lbm::K_COUNT; ++k)
        if (x.kd[k] != y.kd[k] || x.kf[k] != y.kf[k]) return false;
    return true;
}

void drop_graph(lbm_s* h) {
    if (h->graph) cudaGraphExecDestroy(h->graph);
    h->graph = nullptr;
}

// Captures graph_steps launches (even parity first) on the internal stream.
cudaError_t capture_graph(lbm_s* h, int fm) {
    drop_graph(h);
    cudaError_t e = cudaSuccess;
    if (!h->gstream) e = cudaStreamCreateWithFlags(&h->gstream, cudaStreamNonBlocking);
    if (e == cudaSuccess && !h->ev_in) e = cudaEventCreateWithFlags(&h->ev_in, cudaEventDisableTiming);
    if (e == cudaSuccess && !h->ev_out) e = cudaEventCreateWithFlags(&h->ev_out, cudaEventDisableTiming);
    if (e != cudaSuccess) return e;
    if (h->a.rseed && h->rtable_cap < h->graph_steps) {  // one hash per step of a replay
        if (h->d_rtable) cudaFree(h->d_rtable);             // (synchronous: no replay still reads it)
        h->d_rtable = nullptr;
        h->rtable_cap = 0;
        e = cudaMalloc((void**)&h->d_rtable, h->graph_steps * sizeof(unsigned));
        if (e != cudaSuccess) return e;
        h->rtable_cap = h->graph_steps;
    }
    cudaGraph_t g = nullptr;
    const bool fused = fused_active(h);
    if (fused) e = ensure_fused(h);
    if (e != cudaSuccess) return e;
    e = cudaStreamBeginCapture(h->gstream, cudaStreamCaptureModeThreadLocal);
    if (e != cudaSuccess) return e;
    const int len = graph_len(h);
    if (fused) {  // len / 2 fused launches, alternating between the two arrays
        for (int k = 0; k < len / 2 && e == cudaSuccess; ++k) {
            lbm::Args ak = h->a;
            ak.f = (k & 1) ? h->state_alt : h->state;
            if (ak.rseed) {
                ak.rtable = h->d_rtable;
                ak.tstep = 2 * k;
            }
            e = launch_fused(h, ak, (k & 1) ? h->state : h->state_alt, h->gstream);
        }
    }
    for (int k = 0; !fused && k < len && e == cudaSuccess; ++k) {
        lbm::Args ak = h->a;
        ak.variant = single_variant(h);
        if (ak.rseed) {
            ak.rtable = h->d_rtable;
            ak.tstep = k;
        }
        e = lbm::launch_step_any(ak, h->store, h->model, (k & 1) != 0, fm, h->walls, h->gstream);
    }
    cudaError_t e2 = cudaStreamEndCapture(h->gstream, &g);
    if (e == cudaSuccess) e = e2;
    if (e == cudaSuccess) e = cudaGraphInstantiate(&h->graph, g, 0);
    if (g) cudaGraphDestroy(g);
    if (e == cudaSuccess) {
        h->graph_args = h->a;
        h->graph_force = fm;
    }
    return e;
}

// graph_steps steps from an even step: ordered after prior work on h->stream,
// and later work on h->stream waits for them.
cudaError_t replay_graph(lbm_s* h) {
    const int fm = force_mode(h);
    cudaError_t e = cudaSuccess;
    if (!h->graph || fm != h->graph_force || !same_launch(h->a, h->graph_args)) e = capture_graph(h, fm);
    if (e == cudaSuccess) e = cudaEventRecord(h->ev_in, h->stream);
    if (e == cudaSuccess) e = cudaStreamWaitEvent(h->gstream, h->ev_in, 0);
    if (e == cudaSuccess && h->a.rseed) {
        fill_round_table<<<(graph_len(h) + 255) / 256, 256, 0, h->gstream>>>(
            h->d_rtable, h->a.rseed, static_cast<unsigned long long>(h->t), graph_len(h));
        e = cudaGetLastError();
    }
    if (e == cudaSuccess) e = cudaGraphLaunch(h->graph, h->gstream);
    if (e == cudaSuccess) e = cudaEventRecord(h->ev_out, h->gstream);
    if (e == cudaSuccess) e = cudaStreamWaitEvent(h->stream, h->ev_out, 0);
    return e;
}

int stats_into(lbm_s* h, double out[3]) {
    LBM_CUDA(lbm::launch_stats(h->a, h->store, h->t & 1, h->walls, force_mode(h), h->partials, h->sums, h->stream),
             "stats kernel");
    LBM_CUDA(cudaMemcpyAsync(out, h->sums, 3 * sizeof(double), cudaMemcpyDeviceToHost, h->stream), "stats copy");
    LBM_CUDA(cudaStreamSynchronize(h->stream), "stats sync");
    return fused_error(h);
}

int after_reset(lbm_s* h) {
    h->t = 0;
    if (h->check_every > 0) {
        double s[3];
        int rc = stats_into(h, s);
        if (rc) return rc;
        h->mass0 = s[0];
    }
    return LBM_OK;
}

#define CHECK_HANDLE(h)                                              \
    if (!(h)) return fail(LBM_EINVAL, "null lattice handle");        \
    DeviceGuard guard_((h)->device);                                 \
    if (!guard_.ok) return fail(LBM_ECUDA, "cannot select the lattice's device");

}  // namespace

cudaError_t lbm_prepare_two_step(lbm_s* h) { return ensure_fused(h); }
const CUtensorMap& lbm_tensor_map(const lbm_s* h, const void* base) { return map_of(h, base); }

extern "C" {

const char* lbm_last_error(void) { return g_error.c_str(); }

size_t lbm_bytes_per_update(int store) { return 18 * elem_size(store); }

int lbm_create(int nx, int ny, const double omegas[6], const double force[2], const lbm_bc_t* bc, int model,
               int store, double rho0, lbm_t* out) {
    g_error.clear();
    if (!out) return fail(LBM_EINVAL, "out is NULL");
    if (nx < 1 || ny < 1) return fail(LBM_EINVAL, "nx and ny must be >= 1 (got %d x %d)", nx, ny);
    if ((long long)nx * ny > 0x7fffffffLL) return fail(LBM_EINVAL, "nx * ny exceeds 2^31 - 1");
    if (ny > 65535) return fail(LBM_EINVAL, "ny = %d exceeds 65535", ny);
    if ((long long)((nx + 31) / 32 * 32) * ny > 0x7fffffffLL)
        return fail(LBM_EINVAL, "padded plane (nx rounded up to 32) x ny exceeds 2^31 - 1");
    if (!omegas) return fail(LBM_EINVAL, "omegas is NULL");
    for (int k = 0; k < 6; ++k)
        if (!(omegas[k] > 0.0 && omegas[k] < 2.0))
            return fail(LBM_EINVAL, "omega_%d = %g is outside (0, 2)", k + 3, omegas[k]);
    if (model < LBM_CASCADED || model > LBM_RAWMRT) return fail(LBM_EINVAL, "unknown model %d", model);
    if (elem_size(store) == 0) return fail(LBM_EINVAL, "unknown storage kind %d", store);
    if (!(rho0 > 0.0 && std::isfinite(rho0))) return fail(LBM_EINVAL, "rho0 must be positive and finite");
    if (force && !(std::isfinite(force[0]) && std::isfinite(force[1])))
        return fail(LBM_EINVAL, "force must be finite");
    int edge[4] = {LBM_PERIODIC, LBM_PERIODIC, LBM_PERIODIC, LBM_PERIODIC};
    double wall_u[4] = {0, 0, 0, 0};
    if (bc) {
        for (int k = 0; k < 4; ++k) {
            if (bc->edge[k] < LBM_PERIODIC || bc->edge[k] > LBM_MOVING_WALL)
                return fail(LBM_EINVAL, "unknown edge kind %d on edge %d", bc->edge[k], k);
            if (!std::isfinite(bc->wall_u[k])) return fail(LBM_EINVAL, "wall speed on edge %d is not finite", k);
            edge[k] = bc->edge[k];
            wall_u[k] = bc->wall_u[k];
        }
        if ((edge[LBM_WEST] == LBM_PERIODIC) != (edge[LBM_EAST] == LBM_PERIODIC))
            return fail(LBM_EINVAL, "west and east edges must both be periodic or both be walls");
        if ((edge[LBM_SOUTH] == LBM_PERIODIC) != (edge[LBM_NORTH] == LBM_PERIODIC))
            return fail(LBM_EINVAL, "south and north edges must both be periodic or both be walls");
    }

    lbm_s* h = new lbm_s;
    if (cudaGetDevice(&h->device) != cudaSuccess) {
        delete h;
        return fail(LBM_ECUDA, "no CUDA device available");
    }
    h->model = model;
    h->store = store;
    Args& a = h->a;
    a.nx = nx;
    a.ny = ny;
    a.pitch = (nx + 31) / 32 * 32;
    a.plane = (long long)a.pitch * ny;
    a.scale = lbm::store_scale(store);
    for (int k = 0; k < 6; ++k) a.om[k] = omegas[k];
    a.F[0] = force ? force[0] : 0.0;
    a.F[1] = force ? force[1] : 0.0;
    a.rho0 = rho0;
    a.ffield = nullptr;
    for (int k = 0; k < 4; ++k) {
        h->edge[k] = edge[k];
        h->wall_u[k] = wall_u[k];
        a.wall[k] = edge[k] != LBM_PERIODIC;
        const double U = edge[k] == LBM_MOVING_WALL ? wall_u[k] : 0.0;
        a.wallx[k] = k >= LBM_SOUTH ? 6.0 * rho0 * U : 0.0;
        a.wally[k] = k >= LBM_SOUTH ? 0.0 : 6.0 * rho0 * U;
        h->walls = h->walls || a.wall[k];
    }
    // Four nodes per thread for large 16-bit lattices (measured fastest there);
    // below ~1M nodes a launch is latency-bound and one node per thread is faster.
    a.variant = ((store == LBM_F16DEV || store == LBM_BF16DEV) && (long long)nx * ny >= (1LL << 20)) ? 2 : 0;
    lbm::prepare_constants(a);
    h->state_bytes = 9 * (size_t)a.plane * elem_size(store);
    cudaError_t e = cudaMalloc(&h->state, h->state_bytes);
    if (e == cudaSuccess) e = cudaMemset(h->state, 0, h->state_bytes);  // deviation 0: the rest state w rho0
    if (e == cudaSuccess) e = cudaMalloc((void**)&h->partials, (3 * (size_t)lbm::stats_blocks(a) + 3) * sizeof(double));
    if (e == cudaSuccess) {
        h->sums = h->partials + 3 * (size_t)lbm::stats_blocks(a);
        e = cudaDeviceSynchronize();
    }
    if (e != cudaSuccess) {
        int rc = cuda_fail(e, "lbm_create");
        if (h->state) cudaFree(h->state);
        if (h->partials) cudaFree(h->partials);
        delete h;
        return rc;
    }
    a.f = h->state;
    *out = h;
    return LBM_OK;
}

int lbm_destroy(lbm_t h) {
    if (!h) return LBM_OK;
    int rc = LBM_OK;
    {
        DeviceGuard g(h->device);
        if (h->stream) cudaStreamSynchronize(h->stream);
        else cudaDeviceSynchronize();
        if (h->gstream) cudaStreamSynchronize(h->gstream);
        drop_graph(h);
        if (h->ev_in) cudaEventDestroy(h->ev_in);
        if (h->ev_out) cudaEventDestroy(h->ev_out);
        if (h->gstream) cudaStreamDestroy(h->gstream);
        if (h->state) cudaFree(h->state);
        if (h->ffield) cudaFree(h->ffield);
        if (h->partials) cudaFree(h->partials);
        if (h->d_rtable) cudaFree(h->d_rtable);
        if (h->state_alt) cudaFree(h->state_alt);
        if (h->d_err) cudaFree(h->d_err);
        cudaError_t e = cudaGetLastError();
        if (e != cudaSuccess) rc = cuda_fail(e, "lbm_destroy");
    }
    delete h;
    return rc;
}

int lbm_set_stream(lbm_t h, void* stream) {
    CHECK_HANDLE(h);
    h->stream = static_cast<cudaStream_t>(stream);
    return LBM_OK;
}

int lbm_set_force(lbm_t h, const double force[2]) {
    CHECK_HANDLE(h);
    if (!force || !std::isfinite(force[0]) || !std::isfinite(force[1]))
        return fail(LBM_EINVAL, "force must be two finite numbers");
    h->a.F[0] = force[0];
    h->a.F[1] = force[1];
    lbm::prepare_constants(h->a);
    return LBM_OK;
}

int lbm_set_omegas(lbm_t h, const double omegas[6]) {
    CHECK_HANDLE(h);
    if (!omegas) return fail(LBM_EINVAL, "omegas is NULL");
    for (int k = 0; k < 6; ++k)
        if (!(omegas[k] > 0.0 && omegas[k] < 2.0))
            return fail(LBM_EINVAL, "omega_%d = %g is outside (0, 2)", k + 3, omegas[k]);
    for (int k = 0; k < 6; ++k) h->a.om[k] = omegas[k];
    lbm::prepare_constants(h->a);
    return LBM_OK;
}

int lbm_set_graph_steps(lbm_t h, int steps) {
    CHECK_HANDLE(h);
    if (steps < 0 || (steps & 1)) return fail(LBM_EINVAL, "graph steps must be even and >= 0");
    if (h->gstream) LBM_CUDA(cudaStreamSynchronize(h->gstream), "graph stream sync");
    drop_graph(h);
    h->graph_steps = steps;
    return LBM_OK;
}

int lbm_set_rounding(lbm_t h, int mode, unsigned long long seed) {
    CHECK_HANDLE(h);
    if (mode != LBM_ROUND_NEAREST && mode != LBM_ROUND_STOCHASTIC)
        return fail(LBM_EINVAL, "rounding mode must be LBM_ROUND_NEAREST or LBM_ROUND_STOCHASTIC");
    if (mode == LBM_ROUND_STOCHASTIC && h->store == LBM_F64)
        return fail(LBM_EINVAL, "stochastic rounding applies to LBM_F32, LBM_BF16DEV and LBM_F16DEV storage");
    // rseed != 0 selects stochastic rounding; mix the caller's seed into a nonzero word
    h->a.rseed = mode == LBM_ROUND_STOCHASTIC ? ((seed ^ 0x2545f4914f6cdd1dULL) | 1ULL) : 0ULL;
    h->a.rtable = nullptr;
    h->a.rbase = 0;
    h->a.tstep = 0;
    return LBM_OK;
}

// Variants the storage kind admits: 0 for FP64; 0, 1 and 3 for FP32; 0-3 for 16-bit.
static bool variant_allowed(int store, int v) {
    if (store == LBM_F64) return v == 0;
    if (store == LBM_F32) return v == 0 || v == 1 || v == 3;
    return v >= 0 && v <= 3;
}

int lbm_set_variant(lbm_t h, int variant) {
    CHECK_HANDLE(h);
    if (variant < 0 || variant >= LBM_NUM_VARIANTS) return fail(LBM_EINVAL, "variant must be 0, 1, 2 or 3");
    const int v = variant_allowed(h->store, variant) ? variant : 0;
    if (v == 3) LBM_CUDA(ensure_fused(h), "second population array for fused steps");
    h->a.variant = v;
    return LBM_OK;
}

int lbm_tune(lbm_t h, int trial_steps, float ms[LBM_NUM_VARIANTS]) {
    CHECK_HANDLE(h);
    if (trial_steps < 1) return fail(LBM_EINVAL, "trial_steps must be >= 1");
    const int steps = trial_steps + (trial_steps & 1);  // even: the state returns to its layout
    if (ms)
        for (int v = 0; v < LBM_NUM_VARIANTS; ++v) ms[v] = 0.f;
    static const int widths[4] = {128, 256, 64, 32};  // CTA shapes 128x2, 256x1, 64x4, 32x8
    const int v_prev = h->a.variant;
    // `steps` steps from step h->t as lbm_step takes them without graphs
    auto run = [&](int k0, int count) -> cudaError_t {
        cudaError_t e = cudaSuccess;
        for (long t = h->t + k0, end = h->t + k0 + count; t < end && e == cudaSuccess;) {
            if (fused_active(h) && (t & 1) == 0 && end - t >= 2) {
                e = launch_pair_at(h, t);
                t += 2;
            } else {
                e = launch_step_at(h, (t & 1) != 0, t);
                t += 1;
            }
        }
        return e;
    };
    void* backup = nullptr;
    LBM_CUDA(cudaMallocAsync(&backup, h->state_bytes, h->stream), "tune snapshot allocation");
    cudaEvent_t t0 = nullptr, t1 = nullptr;
    cudaError_t e = cudaMemcpyAsync(backup, h->state, h->state_bytes, cudaMemcpyDeviceToDevice, h->stream);
    if (e == cudaSuccess) e = cudaEventCreate(&t0);
    if (e == cudaSuccess) e = cudaEventCreate(&t1);
    float best = 1e30f;
    int best_v = 0, best_w = 128;
    for (int v = 0; v < LBM_NUM_VARIANTS && e == cudaSuccess; ++v) {
        if (!variant_allowed(h->store, v)) continue;
        if (v == 3 && (ensure_fused(h) != cudaSuccess || h->check_every != 0)) {
            cudaGetLastError();  // no room for the second array: variant 3 is not a candidate
            continue;
        }
        float best_of_v = 1e30f;
        for (int wi = 0; wi < (v == 3 ? 1 : 4) && e == cudaSuccess; ++wi) {  // variant 3 has a fixed tile
            h->a.variant = v;
            h->a.block_x = widths[wi];
            e = run(0, 2);
            if (e == cudaSuccess) e = cudaEventRecord(t0, h->stream);
            if (e == cudaSuccess) e = run(2, steps);
            if (e == cudaSuccess) e = cudaEventRecord(t1, h->stream);
            if (e == cudaSuccess) e = cudaEventSynchronize(t1);
            float t = 0.f;
            if (e == cudaSuccess) e = cudaEventElapsedTime(&t, t0, t1);
            if (e == cudaSuccess) {
                best_of_v = std::min(best_of_v, t / steps);
                if (t < best) { best = t; best_v = v; best_w = widths[wi]; }
                e = cudaMemcpyAsync(h->state, backup, h->state_bytes, cudaMemcpyDeviceToDevice, h->stream);
            }
        }
        if (ms && e == cudaSuccess) ms[v] = best_of_v;
    }
    h->a.variant = e == cudaSuccess ? best_v : v_prev;
    h->a.block_x = best_w;
    cudaFreeAsync(backup, h->stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(h->stream);
    if (t0) cudaEventDestroy(t0);
    if (t1) cudaEventDestroy(t1);
    if (e != cudaSuccess) return cuda_fail(e, "lbm_tune");
    return LBM_OK;
}

int lbm_set_force_field(lbm_t h, const double* fxy, int on_device) {
    CHECK_HANDLE(h);
    if (!fxy) {
        h->has_field = false;
        h->a.ffield = nullptr;
        return LBM_OK;
    }
    const size_t n = 2 * (size_t)nodes(h);
    const bool dbl = h->store == LBM_F64;
    if (!h->ffield) LBM_CUDA(cudaMalloc(&h->ffield, n * (dbl ? 8 : 4)), "force field allocation");
    DevBuf tmp(h->stream);
    const double* src = fxy;
    if (!on_device) {
        LBM_CUDA(tmp.alloc(n * sizeof(double)), "force field staging");
        LBM_CUDA(cudaMemcpyAsync(tmp.p, fxy, n * sizeof(double), cudaMemcpyHostToDevice, h->stream), "force copy");
        src = static_cast<const double*>(tmp.p);
    }
    if (dbl) {
        LBM_CUDA(cudaMemcpyAsync(h->ffield, src, n * sizeof(double), cudaMemcpyDeviceToDevice, h->stream),
                 "force copy");
    } else {
        // FP32 arithmetic kernels read the field in FP32
        LBM_CUDA(lbm::launch_narrow(src, static_cast<float*>(h->ffield), n, h->stream), "force narrowing");
    }
    LBM_CUDA(cudaStreamSynchronize(h->stream), "force field sync");
    h->has_field = true;
    h->a.ffield = h->ffield;
    return LBM_OK;
}

static int init_common(lbm_t h, const double* rho, const double* u) {
    LBM_CUDA(lbm::launch_init(h->a, h->store, h->model, force_mode(h), rho, u, h->stream), "init kernel");
    return LBM_OK;
}

int lbm_init_device(lbm_t h, const double* rho, const double* u) {
    CHECK_HANDLE(h);
    int rc = init_common(h, rho, u);
    if (rc) return rc;
    return after_reset(h);
}

// Address under which the kernels may access a host buffer directly: page-locked
// memory mapped into the device address space (cudaHostAlloc / cudaMallocHost /
// cudaHostRegister memory), else nullptr (pageable memory goes through a copy).
static double* mapped_host(const double* p) {
    if (!p) return nullptr;
    cudaPointerAttributes at;
    if (cudaPointerGetAttributes(&at, p) != cudaSuccess) {
        cudaGetLastError();
        return nullptr;
    }
    return at.type == cudaMemoryTypeHost ? static_cast<double*>(at.devicePointer) : nullptr;
}

int lbm_init(lbm_t h, const double* rho, const double* u) {
    CHECK_HANDLE(h);
    const size_t n = (size_t)nodes(h);
    const double* mrho = mapped_host(rho);
    const double* mu = mapped_host(u);
    if ((rho || u) && (!rho || mrho) && (!u || mu)) {  // the init kernel reads the caller's buffers in place
        int rc = init_common(h, mrho, mu);
        if (rc) return rc;
        LBM_CUDA(cudaStreamSynchronize(h->stream), "init sync");
        return after_reset(h);
    }
    DevBuf buf(h->stream);
    double* drho = nullptr;
    double* du = nullptr;
    if (rho || u) {
        LBM_CUDA(buf.alloc(3 * n * sizeof(double)), "init staging");
        drho = static_cast<double*>(buf.p);
        du = drho + n;
        if (rho) LBM_CUDA(cudaMemcpyAsync(drho, rho, n * sizeof(double), cudaMemcpyHostToDevice, h->stream), "rho copy");
        if (u) LBM_CUDA(cudaMemcpyAsync(du, u, 2 * n * sizeof(double), cudaMemcpyHostToDevice, h->stream), "u copy");
    }
    int rc = init_common(h, rho ? drho : nullptr, u ? du : nullptr);
    if (rc) return rc;
    LBM_CUDA(cudaStreamSynchronize(h->stream), "init sync");
    return after_reset(h);
}

int lbm_step(lbm_t h, long n) {
    CHECK_HANDLE(h);
    if (n < 0) return fail(LBM_EINVAL, "step count must be >= 0");
    const bool fused = fused_active(h);
    if (fused) LBM_CUDA(ensure_fused(h), "second population array for fused steps");
    for (long s = 0; s < n;) {
        const int len = graph_len(h);
        if (len > 0 && h->check_every == 0 && (h->t & 1) == 0 && n - s >= len) {
            LBM_CUDA(replay_graph(h), "step graph");
            h->t += len;
            s += len;
            continue;
        }
        if (fused && (h->t & 1) == 0 && n - s >= 2) {
            LBM_CUDA(launch_pair_at(h, h->t), "fused step launch");
            h->t += 2;
            s += 2;
            continue;
        }
        LBM_CUDA(launch_step(h, (h->t & 1) != 0), "step kernel launch");
        ++h->t;
        ++s;
        if (h->check_every > 0 && h->t % h->check_every == 0) {
            double st[3];
            int rc = stats_into(h, st);
            if (rc) return rc;
            const bool finite = std::isfinite(st[0]) && std::isfinite(st[1]) && std::isfinite(st[2]);
            if (!finite || std::fabs(st[0] - h->mass0) > h->check_rtol * std::fabs(h->mass0))
                return fail(LBM_EDIVERGED, "diverged at step %ld: mass %.17g (start %.17g), momentum (%g, %g)", h->t,
                            st[0], h->mass0, st[1], st[2]);
        }
    }
    return LBM_OK;
}

int lbm_macros_device(lbm_t h, double* rho, double* u) {
    CHECK_HANDLE(h);
    LBM_CUDA(lbm::launch_macros(h->a, h->store, h->t & 1, h->walls, force_mode(h), rho, u, h->stream),
             "macros kernel");
    return LBM_OK;
}

int lbm_macros(lbm_t h, double* rho, double* u) {
    CHECK_HANDLE(h);
    if (!rho && !u) return LBM_OK;
    const size_t n = (size_t)nodes(h);
    double* mrho = mapped_host(rho);
    double* mu = mapped_host(u);
    if ((!rho || mrho) && (!u || mu)) {  // the macros kernel writes the caller's buffers in place
        LBM_CUDA(lbm::launch_macros(h->a, h->store, h->t & 1, h->walls, force_mode(h), mrho, mu, h->stream),
                 "macros kernel");
        LBM_CUDA(cudaStreamSynchronize(h->stream), "macros sync");
        return fused_error(h);
    }
    DevBuf buf(h->stream);
    LBM_CUDA(buf.alloc(3 * n * sizeof(double)), "macros staging");
    double* drho = static_cast<double*>(buf.p);
    double* du = drho + n;
    LBM_CUDA(lbm::launch_macros(h->a, h->store, h->t & 1, h->walls, force_mode(h), rho ? drho : nullptr,
                                u ? du : nullptr, h->stream),
             "macros kernel");
    if (rho) LBM_CUDA(cudaMemcpyAsync(rho, drho, n * sizeof(double), cudaMemcpyDeviceToHost, h->stream), "rho copy");
    if (u) LBM_CUDA(cudaMemcpyAsync(u, du, 2 * n * sizeof(double), cudaMemcpyDeviceToHost, h->stream), "u copy");
    LBM_CUDA(cudaStreamSynchronize(h->stream), "macros sync");
    return fused_error(h);
}

// Eq. (28)-(30) divide by the rates at which the second-order moments relax:
// omega_3, omega_4, omega_5 for the cascaded and raw-MRT collisions, the single
// rate omega_4 for BGK.
static lbm::Args strain_args(const lbm_s* h) {
    lbm::Args a = h->a;
    if (h->model == LBM_BGK) a.om[0] = a.om[2] = a.om[1];
    return a;
}

int lbm_strain_device(lbm_t h, double* out) {
    CHECK_HANDLE(h);
    if (!out) return fail(LBM_EINVAL, "out is NULL");
    LBM_CUDA(lbm::launch_strain(strain_args(h), h->store, h->t & 1, h->walls, force_mode(h), out, h->stream), "strain kernel");
    return LBM_OK;
}

int lbm_strain(lbm_t h, double* out) {
    CHECK_HANDLE(h);
    if (!out) return fail(LBM_EINVAL, "out is NULL");
    const size_t n = 3 * (size_t)nodes(h);
    DevBuf buf(h->stream);
    LBM_CUDA(buf.alloc(n * sizeof(double)), "strain staging");
    LBM_CUDA(lbm::launch_strain(strain_args(h), h->store, h->t & 1, h->walls, force_mode(h), static_cast<double*>(buf.p),
                                h->stream),
             "strain kernel");
    LBM_CUDA(cudaMemcpyAsync(out, buf.p, n * sizeof(double), cudaMemcpyDeviceToHost, h->stream), "strain copy");
    LBM_CUDA(cudaStreamSynchronize(h->stream), "strain sync");
    return LBM_OK;
}

int lbm_get_f_device(lbm_t h, double* f) {
    CHECK_HANDLE(h);
    if (!f) return fail(LBM_EINVAL, "f is NULL");
    LBM_CUDA(lbm::launch_get_f(h->a, h->store, h->t & 1, h->walls, f, h->stream), "get_f kernel");
    return LBM_OK;
}

int lbm_get_f(lbm_t h, double* f) {
    CHECK_HANDLE(h);
    if (!f) return fail(LBM_EINVAL, "f is NULL");
    const size_t n = 9 * (size_t)nodes(h);
    DevBuf buf(h->stream);
    LBM_CUDA(buf.alloc(n * sizeof(double)), "get_f staging");
    LBM_CUDA(lbm::launch_get_f(h->a, h->store, h->t & 1, h->walls, static_cast<double*>(buf.p), h->stream),
             "get_f kernel");
    LBM_CUDA(cudaMemcpyAsync(f, buf.p, n * sizeof(double), cudaMemcpyDeviceToHost, h->stream), "f copy");
    LBM_CUDA(cudaStreamSynchronize(h->stream), "get_f sync");
    return fused_error(h);
}

int lbm_set_f_device(lbm_t h, const double* f) {
    CHECK_HANDLE(h);
    if (!f) return fail(LBM_EINVAL, "f is NULL");
    LBM_CUDA(lbm::launch_set_f(h->a, h->store, f, h->stream), "set_f kernel");
    return after_reset(h);
}

int lbm_set_f(lbm_t h, const double* f) {
    CHECK_HANDLE(h);
    if (!f) return fail(LBM_EINVAL, "f is NULL");
    const size_t n = 9 * (size_t)nodes(h);
    DevBuf buf(h->stream);
    LBM_CUDA(buf.alloc(n * sizeof(double)), "set_f staging");
    LBM_CUDA(cudaMemcpyAsync(buf.p, f, n * sizeof(double), cudaMemcpyHostToDevice, h->stream), "f copy");
    LBM_CUDA(lbm::launch_set_f(h->a, h->store, static_cast<const double*>(buf.p), h->stream), "set_f kernel");
    LBM_CUDA(cudaStreamSynchronize(h->stream), "set_f sync");
    return after_reset(h);
}

int lbm_stats(lbm_t h, double out[3]) {
    CHECK_HANDLE(h);
    if (!out) return fail(LBM_EINVAL, "out is NULL");
    return stats_into(h, out);
}

int lbm_set_check(lbm_t h, long every, double mass_rtol) {
    CHECK_HANDLE(h);
    if (every < 0 || !(mass_rtol >= 0.0)) return fail(LBM_EINVAL, "every must be >= 0 and mass_rtol >= 0");
    h->check_every = every;
    h->check_rtol = mass_rtol;
    if (every > 0) {
        double s[3];
        int rc = stats_into(h, s);
        if (rc) return rc;
        h->mass0 = s[0];
    }
    return LBM_OK;
}

long lbm_time(lbm_t h) { return h ? h->t : -1; }

int lbm_info(lbm_t h, long dims[7], size_t* bytes, void** state) {
    if (!h) return fail(LBM_EINVAL, "null lattice handle");
    if (dims) {
        dims[0] = h->a.nx; dims[1] = h->a.ny; dims[2] = h->a.pitch; dims[3] = h->model; dims[4] = h->store;
        dims[5] = h->a.variant; dims[6] = h->a.block_x > 0 ? h->a.block_x : lbm::kStepBX;
    }
    if (bytes) *bytes = h->state_bytes;
    if (state) *state = h->state;
    return LBM_OK;
}

}  // extern "C"
