// lbm_adjoint.cu -- discrete adjoint of a periodic cascaded run (gradients of a
// final-state velocity loss with respect to the initial velocity, the per-node
// body force and the relaxation rates).
//
// Forward: f^0 = f_eq(rho, u0) - S/2 (Eq. 6, 12), f^{n+1} = P C(f^n; F, omega)
// (collide Eq. 23, stream Eq. 24), L = 1/2 sum_x |u(x, T) - u_target(x)|^2 with
// u from Eq. (26)-(27).  Reverse: lambda^T = dL/df^T; for n = T-1 .. 0
//   mu_a(x) = lambda^{n+1}_a(x + e_a)             (transpose of the pull: a push)
//   lambda^n(x) = (dC/df)^T mu(x)                  (collide_cascaded_vjp, in registers)
//   dL/dF(x) += (dC/dF)^T mu(x),                   dL/dc += (dC/dc)^T mu(x)  (FP64 sums)
// with dL/dF summed in the arithmetic type over the steps of one checkpoint
// segment and in FP64 across segments (and over the whole run for FP64 storage)
// and finally dL/du0 = (df^0/du0)^T lambda^0.  The states f^n are recomputed one
// segment at a time from checkpoints taken every `every` steps.
#include <algorithm>
#include <vector>

#include "lbm.h"
#include "lbm_adjoint.cuh"
#include "lbm_internal.h"
#include "lbm_handle.h"

namespace lbm {
namespace {

constexpr int kThreads = 256;

template <typename R>
__device__ __forceinline__ void force_rt(const Args& a, int force, int x, int y, R& Fx, R& Fy) {
    if (force == 0) { Fx = R(0); Fy = R(0); return; }
    if (force == 1) { node_force<R, 1>(a, x, y, Fx, Fy); return; }
    node_force<R, 2>(a, x, y, Fx, Fy);
}

template <int ST>
__device__ __forceinline__ void load_rt(const Args& a, bool odd, int x, int y, typename Store<ST>::R d[9]) {
    if (odd) load_node<ST, true, false>(a, x, y, d);
    else load_node<ST, false, false>(a, x, y, d);
}

// Sums v[0..N) over the block and adds the totals to the FP64 accumulators
// acc[0..N).  The sum inside a warp runs in the values' own type (FP32 for
// the FP32 adjoint: a warp adds 32 terms); the warp totals are added in FP64,
// and so is the accumulation over blocks and time steps.
template <int N, typename V>
__device__ __forceinline__ void block_atomic_add(V (&v)[N], double* acc) {
    __shared__ double sh[N][kThreads / 32];
#pragma unroll
    for (int k = 0; k < N; ++k)
        for (int o = 16; o > 0; o >>= 1) v[k] += __shfl_down_sync(0xffffffffu, v[k], o);
    if ((threadIdx.x & 31) == 0)
#pragma unroll
        for (int k = 0; k < N; ++k) sh[k][threadIdx.x >> 5] = double(v[k]);
    __syncthreads();
    if (threadIdx.x < N) {
        double t = 0.0;
        for (int w = 0; w < kThreads / 32; ++w) t += sh[threadIdx.x][w];
        atomicAdd(acc + threadIdx.x, t);
    }
}

// Loss at the final state and its adjoint lambda^T (natural layout), plus the
// direct part of dL/dF through u(T) = (j + F/2)/rho, which initialises gF.
template <int ST>
__global__ void __launch_bounds__(kThreads) adj_final_kernel(const Args a, bool odd, int force,
                                                             const double* target, typename Store<ST>::R* lam,
                                                             double* gF, double* loss) {
    using R = typename Store<ST>::R;
    const int x = blockIdx.x * kThreads + threadIdx.x, y = blockIdx.y;
    double l[1] = {0.0};
    if (x < a.nx) {
        R d[9];
        load_rt<ST>(a, odd, x, y, d);
        R Fx, Fy;
        force_rt<R>(a, force, x, y, Fx, Fy);
        const Moments<R> m = moments(d, R(a.rho0));
        const double rho = double(m.rho);
        const double ux = (double(m.jx) + 0.5 * double(Fx)) / rho, uy = (double(m.jy) + 0.5 * double(Fy)) / rho;
        const int n = y * a.nx + x, p = a.nx * a.ny;
        const double rx = ux - target[n], ry = uy - target[p + n];
        l[0] = 0.5 * (rx * rx + ry * ry);
        const double jxa = rx / rho, jya = ry / rho, rhoa = -(rx * ux + ry * uy) / rho;
        const int o = y * a.pitch + x;
#pragma unroll
        for (int q = 0; q < 9; ++q) lam[q * a.plane + o] = R(rhoa + cx(q) * jxa + cy(q) * jya);
        gF[n] = 0.5 * jxa;
        gF[p + n] = 0.5 * jya;
    }
    block_atomic_add<1>(l, loss);
}

// One reverse step: lambda^n from lambda^{n+1} at the state f^n held in a.f.
// The force gradient of the step goes into gs, in the arithmetic type: written
// on the first reverse step of a checkpoint segment (`first`), added after
// that; adj_fold_kernel adds each segment's sum into the FP64 gradient (for
// FP64 storage gs is the FP64 gradient itself and `first` is false).
// Each thread takes kAdjRows node rows (y0, y0 + 1, ...) of its column and
// sums their rate adjoints in registers, so the block reduction of the six
// sums runs once per kAdjRows nodes.
constexpr int kAdjRows = 4;

template <int ST>
__global__ void __launch_bounds__(kThreads, ST == LBM_F32 ? 4 : 1) adj_step_kernel(const Args a, bool odd, int force,
                                                            const typename Store<ST>::R* __restrict__ lin,
                                                            typename Store<ST>::R* __restrict__ lout,
                                                            typename Store<ST>::R* __restrict__ gs, bool first,
                                                            double* gc) {
    using R = typename Store<ST>::R;
    const int x = blockIdx.x * kThreads + threadIdx.x, y0 = blockIdx.y * kAdjRows;
    R c[6] = {0, 0, 0, 0, 0, 0};
    if (x < a.nx) {
        const int xm = x > 0 ? x - 1 : a.nx - 1, xp = x < a.nx - 1 ? x + 1 : 0;
        const int yend = min(y0 + kAdjRows, a.ny);
#pragma unroll 1
        for (int y = y0; y < yend; ++y) {
            const Coef<R> co(a);
            R d[9];
            load_rt<ST>(a, odd, x, y, d);
            R Fx, Fy;
            force_rt<R>(a, force, x, y, Fx, Fy);
            const int rm = (y > 0 ? y - 1 : a.ny - 1) * a.pitch, rp = (y < a.ny - 1 ? y + 1 : 0) * a.pitch;
            const int r0 = y * a.pitch;
            R mu[9];
#pragma unroll
            for (int q = 0; q < 9; ++q) {  // mu_q(x) = lambda_q(x + e_q)
                const int tx = cx(q) == 1 ? xp : (cx(q) == -1 ? xm : x);
                const int tr = cy(q) == 1 ? rp : (cy(q) == -1 ? rm : r0);
                mu[q] = lin[q * a.plane + tr + tx];
            }
            CollideAdjoint<R> g;
            collide_cascaded_vjp<R>(d, Fx, Fy, co, mu, g);
#pragma unroll
            for (int q = 0; q < 9; ++q) lout[q * a.plane + r0 + x] = g.d[q];
            const int n = y * a.nx + x, p = a.nx * a.ny;
            if (first) {
                gs[n] = g.Fx;
                gs[p + n] = g.Fy;
            } else {
                gs[n] += g.Fx;
                gs[p + n] += g.Fy;
            }
#pragma unroll
            for (int k = 0; k < 6; ++k) c[k] += g.c[k];
        }
    }
    block_atomic_add<6>(c, gc);
}

__device__ __forceinline__ double phi(int e, double u) {
    return e == 0 ? (2.0 / 3.0 - u * u) : 0.5 * (1.0 / 3.0 + u * u + e * u);
}
__device__ __forceinline__ double dphi(int e, double u) { return e == 0 ? -2.0 * u : u + 0.5 * e; }

// dL/du0 = (d f^0 / d u0)^T lambda^0 with f^0 = rho phi(e_x; ux) phi(e_y; uy) - S(u0, F)/2
// (the cascaded equilibrium in product form), and the -S/2 part of dL/dF.
template <int ST>
__global__ void __launch_bounds__(kThreads) adj_init_kernel(const Args a, int force, const double* rho,
                                                            const double* u0, const typename Store<ST>::R* lam,
                                                            double* gu0, double* gF) {
    using R = typename Store<ST>::R;
    const int x = blockIdx.x * kThreads + threadIdx.x, y = blockIdx.y;
    if (x >= a.nx) return;
    const int n = y * a.nx + x, p = a.nx * a.ny, o = y * a.pitch + x;
    const double r = rho ? rho[n] : a.rho0;
    const double ux = u0[n], uy = u0[p + n];
    R Fr, Gr;
    force_rt<R>(a, force, x, y, Fr, Gr);
    const double Fx = double(Fr) / a.scale, Fy = double(Gr) / a.scale;
    double mu[9];
#pragma unroll
    for (int q = 0; q < 9; ++q) mu[q] = double(lam[q * a.plane + o]);
    double gux = 0.0, guy = 0.0;
#pragma unroll
    for (int q = 0; q < 9; ++q) {
        gux += mu[q] * r * dphi(cx(q), ux) * phi(cy(q), uy);
        guy += mu[q] * r * phi(cx(q), ux) * dphi(cy(q), uy);
    }
    double half[9];
#pragma unroll
    for (int q = 0; q < 9; ++q) half[q] = -0.5 * mu[q];
    double gFx = 0.0, gFy = 0.0;
    source_vjp<double>(ux, uy, Fx, Fy, half, gux, guy, gFx, gFy);
    if (gu0) { gu0[n] = gux; gu0[p + n] = guy; }
    gF[n] += gFx;
    gF[p + n] += gFy;
}

// gF[i] += gs[i] for the 2 nx ny force-gradient entries of one segment (GB300's
// FP64 pipe is far narrower than its FP32 one: FP64 work once per segment, not
// once per step).
__global__ void __launch_bounds__(kThreads) adj_fold_kernel(long long count, const float* __restrict__ gs,
                                                            double* __restrict__ gF) {
    const long long i = (long long)blockIdx.x * kThreads + threadIdx.x;
    if (i < count) gF[i] += double(gs[i]);
}

// The launch arguments of forward step t: with stochastic rounding of the
// stores, the hash of (seed, t), so that the recomputed states are bit for bit
// the forward ones (the reverse pass treats the rounding as the identity).
Args at_step(const Args& a, long t) {
    Args ak = a;
    if (ak.rseed) {
        ak.rbase = round_hash(ak.rseed, static_cast<unsigned long long>(t));
        ak.rtable = nullptr;
        ak.tstep = 0;
    }
    return ak;
}

template <int ST>
cudaError_t run_reverse(lbm_s* h, long nsteps, long every, const double* rho, const double* u0, const double* target,
                        char* ckpt, char* seg, void* lam0, void* lam1, double* gF, float* gseg, double* acc,
                        double* gu0) {
    using R = typename Store<ST>::R;
    const Args& a = h->a;
    cudaStream_t s = h->stream;
    const int fm = force_mode(h);
    const size_t SB = h->state_bytes;
    const dim3 grid((a.nx + kThreads - 1) / kThreads, a.ny);
    const long nck = (nsteps + every - 1) / every;
    cudaError_t e;

    // Forward pass.  f^t lives in ckpt[c] at the checkpoint times t = c every and
    // in the lattice's own array otherwise (and at t = nsteps); a step whose
    // input and output live in different arrays runs out of place (Args::fo),
    // the others in place, so no state is ever copied.
    auto where = [&](long t) -> char* {
        return (t % every == 0 && t < nsteps) ? ckpt + (t / every) * SB : static_cast<char*>(h->state);
    };
    {
        Args a0 = a;
        a0.f = ckpt;
        if ((e = launch_init(a0, h->store, h->model, fm, rho, u0, s)) != cudaSuccess) return e;
    }
    h->t = 0;
    for (long t = 0; t < nsteps; ++t) {
        Args ak = at_step(a, t);
        ak.f = where(t);
        char* out = where(t + 1);
        ak.fo = out != ak.f ? out : nullptr;
        if ((e = launch_step_any(ak, h->store, h->model, t & 1, fm, false, s)) != cudaSuccess) return e;
        ++h->t;
    }
    R* cur = static_cast<R*>(lam0);
    R* nxt = static_cast<R*>(lam1);
    adj_final_kernel<ST><<<grid, kThreads, 0, s>>>(a, nsteps & 1, fm, target, cur, gF, acc);
    if ((e = cudaGetLastError()) != cudaSuccess) return e;

    // Reverse sweep, one segment at a time: f^{n0} is read from its checkpoint
    // and f^{n0 + k}, k = 1 .. len - 1, recomputed out of place into seg slot k - 1.
    for (long c = nck - 1; c >= 0; --c) {
        const long n0 = c * every, len = std::min(every, nsteps - n0);
        auto state = [&](long k) -> char* { return k == 0 ? ckpt + c * SB : seg + (k - 1) * SB; };
        for (long k = 1; k < len; ++k) {
            Args ak = at_step(a, n0 + k - 1);
            ak.f = state(k - 1);
            ak.fo = state(k);
            if ((e = launch_step_any(ak, h->store, h->model, (n0 + k - 1) & 1, fm, false, s)) != cudaSuccess) return e;
        }
        R* gs = ST == LBM_F64 ? reinterpret_cast<R*>(gF) : reinterpret_cast<R*>(gseg);
        const dim3 agrid(grid.x, (a.ny + kAdjRows - 1) / kAdjRows);
        for (long k = len - 1; k >= 0; --k) {
            Args ak = a;
            ak.f = state(k);
            const bool first = ST != LBM_F64 && k == len - 1;
            adj_step_kernel<ST><<<agrid, kThreads, 0, s>>>(ak, (n0 + k) & 1, fm, cur, nxt, gs, first, acc + 1);
            if ((e = cudaGetLastError()) != cudaSuccess) return e;
            std::swap(cur, nxt);
        }
        if (ST != LBM_F64) {
            const long long count = 2LL * a.nx * a.ny;
            adj_fold_kernel<<<unsigned((count + kThreads - 1) / kThreads), kThreads, 0, s>>>(count, gseg, gF);
            if ((e = cudaGetLastError()) != cudaSuccess) return e;
        }
    }
    adj_init_kernel<ST><<<grid, kThreads, 0, s>>>(a, fm, rho, u0, cur, gu0, gF);
    return cudaGetLastError();
}

}  // namespace
}  // namespace lbm

extern "C" int lbm_adjoint_run(lbm_t h, long nsteps, long every, const double* rho, const double* u0,
                               const double* u_target, double* loss, double* grad_u0, double* grad_force,
                               double grad_omega[6]) {
    using namespace lbm;
    if (!h) return set_error(LBM_EINVAL, "null lattice handle");
    if (h->model != LBM_CASCADED) return set_error(LBM_EINVAL, "lbm_adjoint_run: the adjoint is for the cascaded model");
    if (h->store != LBM_F64 && h->store != LBM_F32)
        return set_error(LBM_EINVAL, "lbm_adjoint_run: FP64 or FP32 storage required");
    if (h->walls) return set_error(LBM_EINVAL, "lbm_adjoint_run: all four edges must be periodic");
    if (nsteps < 1 || every < 1) return set_error(LBM_EINVAL, "lbm_adjoint_run: nsteps and every must be >= 1");
    if (!u0 || !u_target || !loss) return set_error(LBM_EINVAL, "lbm_adjoint_run: u0, u_target and loss are required");
    int prev = -1;
    cudaGetDevice(&prev);
    if (prev != h->device) cudaSetDevice(h->device);
    cudaStream_t s = h->stream;
    const size_t SB = h->state_bytes;
    const long nck = (nsteps + every - 1) / every;
    const long seglen = std::min(every, nsteps);
    const size_t lam_bytes = 9 * (size_t)h->a.plane * (h->store == LBM_F64 ? 8 : 4);
    const size_t n = (size_t)h->a.nx * h->a.ny;
    std::vector<void*> bufs;
    auto alloc = [&](size_t bytes) -> void* {
        void* p = nullptr;
        if (cudaMallocAsync(&p, bytes, s) != cudaSuccess) return nullptr;
        bufs.push_back(p);
        return p;
    };
    auto release = [&]() {
        for (void* p : bufs) cudaFreeAsync(p, s);
        bufs.clear();
    };
    char* ckpt = static_cast<char*>(alloc(nck * SB));
    char* seg = static_cast<char*>(alloc(std::max(1L, seglen - 1) * SB));
    void* lam0 = alloc(lam_bytes);
    void* lam1 = alloc(lam_bytes);
    double* acc = static_cast<double*>(alloc(7 * sizeof(double)));
    double* gF = grad_force ? grad_force : static_cast<double*>(alloc(2 * n * sizeof(double)));
    float* gseg = h->store == LBM_F64 ? nullptr : static_cast<float*>(alloc(2 * n * sizeof(float)));
    if (!ckpt || !seg || !lam0 || !lam1 || !acc || !gF || (h->store != LBM_F64 && !gseg)) {
        release();
        cudaGetLastError();
        if (prev >= 0 && prev != h->device) cudaSetDevice(prev);
        return set_error(LBM_ENOMEM, "lbm_adjoint_run: cannot allocate %.1f MB of checkpoints and buffers",
                         ((nck + std::max(1L, seglen - 1)) * SB + 2 * lam_bytes) / 1e6);
    }
    cudaError_t e = cudaMemsetAsync(acc, 0, 7 * sizeof(double), s);
    if (e == cudaSuccess) {
        e = h->store == LBM_F64
                ? run_reverse<LBM_F64>(h, nsteps, every, rho, u0, u_target, ckpt, seg, lam0, lam1, gF, gseg, acc,
                                       grad_u0)
                : run_reverse<LBM_F32>(h, nsteps, every, rho, u0, u_target, ckpt, seg, lam0, lam1, gF, gseg, acc,
                                       grad_u0);
    }
    double host[7] = {0, 0, 0, 0, 0, 0, 0};
    if (e == cudaSuccess) e = cudaMemcpyAsync(host, acc, sizeof host, cudaMemcpyDeviceToHost, s);
    release();
    if (e == cudaSuccess) e = cudaStreamSynchronize(s);
    if (prev >= 0 && prev != h->device) cudaSetDevice(prev);
    if (e != cudaSuccess)
        return set_error(e == cudaErrorMemoryAllocation ? LBM_ENOMEM : LBM_ECUDA, "lbm_adjoint_run: %s",
                         cudaGetErrorString(e));
    *loss = host[0];
    if (grad_omega) {
        grad_omega[0] = host[1] / 12.0;
        for (int k = 1; k < 6; ++k) grad_omega[k] = host[1 + k] / 4.0;
    }
    return LBM_OK;
}
