// lbm_batch.cu -- many independent lattices advanced together: one kernel
// launch per time step for all of them (a persistent grid walking a tile list,
// or one CTA per tile), or one launch per two steps for each class of lattice
// (lbm_batch_fused.cuh), CUDA graphs of `graph_steps` steps, and an autotuner
// that picks the tile shape, the order of the work list and the scheduling
// policy by timing them on the batch itself.
#include <algorithm>
#include <numeric>
#include <vector>

#include "lbm.h"
#include "lbm_batch_fused.cuh"
#include "lbm_batch_impl.cuh"
#include "lbm_handle.h"

namespace lbm {
cudaError_t launch_batch_cascaded(int, const BatchDomain*, const int*, int, int, int, int, int, int*, const unsigned*, int,
                                  int, cudaStream_t);
cudaError_t launch_batch_bgk(int, const BatchDomain*, const int*, int, int, int, int, int, int*, const unsigned*, int, int,
                             cudaStream_t);
cudaError_t launch_batch_rawmrt(int, const BatchDomain*, const int*, int, int, int, int, int, int*, const unsigned*, int,
                                int, cudaStream_t);
cudaError_t launch_batch_fused_cascaded(int, int, const BatchDomain*, const BatchPair*, const int*, int, const unsigned*,
                                        int, int, int*, cudaStream_t);
cudaError_t launch_batch_fused_bgk(int, int, const BatchDomain*, const BatchPair*, const int*, int, const unsigned*, int,
                                   int, int*, cudaStream_t);
cudaError_t launch_batch_fused_rawmrt(int, int, const BatchDomain*, const BatchPair*, const int*, int, const unsigned*,
                                      int, int, int*, cudaStream_t);

// rtab[d * rstride + k] = the hash of (seed, t + base + k) of domain d, for the
// k-th launch of a sequence that starts `base` steps after the domains' counts t.
__global__ void __launch_bounds__(kBatchThreads) fill_batch_round_table(const BatchDomain* __restrict__ doms,
                                                                        int ndoms, unsigned* rtab, int rstride,
                                                                        long long base) {
    const int i = blockIdx.x * kBatchThreads + threadIdx.x;
    if (i >= ndoms * rstride) return;
    const int d = i / rstride, k = i % rstride;
    const BatchDomain& D = doms[d];
    rtab[i] = D.a.rseed ? round_hash(D.a.rseed, static_cast<unsigned long long>(D.t + base + k)) : 0u;
}


int batch_blocks_per_sm_cascaded();
int batch_blocks_per_sm_bgk();
int batch_blocks_per_sm_rawmrt();
}  // namespace lbm

using lbm::BatchDomain;

struct lbm_batch_s {
    int device = 0;
    int model = 0;
    std::vector<lbm_s*> doms;
    cudaStream_t stream = nullptr;  // internal, non-blocking (graphs are captured on it)
    cudaEvent_t done = nullptr;
    BatchDomain* h_doms = nullptr;  // pinned staging of the domain table
    BatchDomain* d_doms = nullptr;
    int* d_tiles = nullptr;
    size_t tiles_cap = 0;  // ints
    int ntiles = 0;
    int* d_counters = nullptr;
    int ncounters = 0;
    int lbx = 7, rows = 1, policy = lbm::kPolicyRoundRobin, order = 0, grid = 0;
    int resident = 0;  // grid of the persistent policies: SMs x resident CTAs per SM
    bool flat = false; // one CTA per tile (grid = tiles) instead of a persistent grid
    int sms = 0;
    int graph_steps = 100;
    cudaGraphExec_t graph = nullptr;
    float tuned_ms = 0.f;
    // Stochastic rounding: per-domain hashes of (seed, step) for the launches of
    // a graph replay or a single launch, [doms][ncounters], filled before each.
    unsigned* d_rtab = nullptr;
    bool any_sr = false;
    // Two steps per launch (lbm_batch_set_two_step, or chosen by the tuner):
    // every lattice's two arrays and their tensor maps (pinned staging and
    // device copy), the list of 64 x 16 tiles, the kernels' error word and a
    // graph of two-step launches.  The tile list is ordered by lattice class
    // (class_first[c] .. class_first[c + 1] - 1 are the tiles of class c) for
    // the classes in cls2; the kernels of the second and later classes of a
    // launch run on branch streams forked from the batch stream.
    bool two_step = false;
    lbm::BatchPair* h_pairs = nullptr;
    lbm::BatchPair* d_pairs = nullptr;
    int* d_tiles2 = nullptr;
    int ntiles2 = 0;
    int* d_err = nullptr;
    cudaGraphExec_t graph2 = nullptr;
    std::vector<int> cls2;
    int class_first[lbm::kBatchClasses + 1] = {};
    struct Branch {
        cudaStream_t s;
        cudaEvent_t joined;  // recorded on s after its kernel; the batch stream waits on it
    };
    std::vector<Branch> branch;
    cudaEvent_t fork = nullptr;  // recorded on the batch stream before a launch's branches
};

namespace {

constexpr int kShapes[4] = {7, 8, 6, 5};  // log2 of the tile width: 128x2, 256x1, 64x4, 32x8

int fail(int code, const char* msg) { return lbm::set_error(code, "%s", msg); }

constexpr int kRows[2] = {1, 4};  // node rows per thread

long long tiles_of(const lbm_s* h, int lbx, int rows) {
    const int bx = 1 << lbx, by = (lbm::kBatchThreads >> lbx) * rows;
    return (long long)((h->a.nx + bx - 1) / bx) * ((h->a.ny + by - 1) / by);
}

// Work list for tile shape lbx with `rows` node rows per thread (a tile is
// bx x (256 / bx) * rows nodes).  order 0: domain after domain, largest domain
// first; order 1: one tile of each domain in turn (largest first).
std::vector<int> build_tiles(const lbm_batch_s* b, int lbx, int rows, int order) {
    const int bx = 1 << lbx, by = (lbm::kBatchThreads >> lbx) * rows;
    std::vector<int> idx(b->doms.size());
    std::iota(idx.begin(), idx.end(), 0);
    std::stable_sort(idx.begin(), idx.end(), [&](int p, int q) {
        return (long long)b->doms[p]->a.nx * b->doms[p]->a.ny > (long long)b->doms[q]->a.nx * b->doms[q]->a.ny;
    });
    std::vector<int> t;
    if (order == 0) {
        for (int d : idx) {
            const int tx = (b->doms[d]->a.nx + bx - 1) / bx, ty = (b->doms[d]->a.ny + by - 1) / by;
            for (int j = 0; j < ty; ++j)
                for (int i = 0; i < tx; ++i) t.insert(t.end(), {d, i, j});
        }
    } else {
        std::vector<long long> next(idx.size(), 0);
        bool any = true;
        while (any) {
            any = false;
            for (size_t k = 0; k < idx.size(); ++k) {
                const int d = idx[k];
                const int tx = (b->doms[d]->a.nx + bx - 1) / bx, ty = (b->doms[d]->a.ny + by - 1) / by;
                if (next[k] < (long long)tx * ty) {
                    const long long n = next[k]++;
                    t.insert(t.end(), {d, int(n % tx), int(n / tx)});
                    any = true;
                }
            }
        }
    }
    return t;
}

cudaError_t upload_tiles(lbm_batch_s* b, int lbx, int rows, int order) {
    const std::vector<int> t = build_tiles(b, lbx, rows, order);
    b->ntiles = int(t.size() / 3);
    return cudaMemcpyAsync(b->d_tiles, t.data(), t.size() * sizeof(int), cudaMemcpyHostToDevice, b->stream);
}

// Waits for the batch stream and every branch stream.  After a complete
// two-step launch the batch stream already waits for its branches; a launch
// that failed half way may have left a branch kernel without that wait.
cudaError_t sync_all(lbm_batch_s* b) {
    cudaError_t e = cudaStreamSynchronize(b->stream);
    for (const lbm_batch_s::Branch& br : b->branch) {
        const cudaError_t e2 = cudaStreamSynchronize(br.s);
        if (e == cudaSuccess) e = e2;
    }
    return e;
}

// Copies each domain's current arguments and parity into the device table
// (and, once two-step launches are prepared, each lattice's arrays and maps).
cudaError_t order_tiles2(lbm_batch_s* b, int* dt);
std::vector<int> domain_classes(const lbm_batch_s* b);

cudaError_t refresh_domains(lbm_batch_s* b) {
    cudaError_t e = cudaEventSynchronize(b->done);  // the previous upload has finished reading h_doms
    if (e != cudaSuccess) return e;
    if (b->h_pairs && domain_classes(b) != b->cls2) {  // a lattice changed its force or rounding
        e = sync_all(b);  // no launch still reads the tile list
        if (e == cudaSuccess) e = order_tiles2(b, b->d_tiles2);
        if (e != cudaSuccess) return e;
        if (b->graph2) cudaGraphExecDestroy(b->graph2);
        b->graph2 = nullptr;
    }
    if (b->h_pairs) {
        for (size_t i = 0; i < b->doms.size(); ++i) {
            const lbm_s* h = b->doms[i];
            lbm::BatchPair& P = b->h_pairs[i];
            P.arr[0] = h->state;
            P.arr[1] = h->state_alt;
            P.map[0] = lbm_tensor_map(h, h->state);
            P.map[1] = lbm_tensor_map(h, h->state_alt);
        }
        e = cudaMemcpyAsync(b->d_pairs, b->h_pairs, b->doms.size() * sizeof(lbm::BatchPair), cudaMemcpyHostToDevice,
                            b->stream);
        if (e != cudaSuccess) return e;
    }
    bool any_sr = false;
    for (size_t i = 0; i < b->doms.size(); ++i) {
        const lbm_s* h = b->doms[i];
        BatchDomain& D = b->h_doms[i];
        D.a = h->a;
        D.store = h->store;
        D.walls = h->walls ? 1 : 0;
        D.force = lbm::force_mode(h);
        D.parity = int(h->t & 1);
        D.t = h->t;
        any_sr = any_sr || h->a.rseed != 0;
    }
    b->any_sr = any_sr;
    return cudaMemcpyAsync(b->d_doms, b->h_doms, b->doms.size() * sizeof(BatchDomain), cudaMemcpyHostToDevice,
                           b->stream);
}

// Hashes for `count` launches that start `base` steps after the domains' counts.
cudaError_t fill_round_table(lbm_batch_s* b, int count, long long base) {
    if (!b->any_sr) return cudaSuccess;
    const int n = int(b->doms.size()) * count;
    lbm::fill_batch_round_table<<<(n + lbm::kBatchThreads - 1) / lbm::kBatchThreads, lbm::kBatchThreads, 0, b->stream>>>(
        b->d_doms, int(b->doms.size()), b->d_rtab, count, base);
    return cudaGetLastError();
}

// kstep: the launch's index in a sequence whose round table has rstride entries per domain.
cudaError_t launch(lbm_batch_s* b, int flip, int* counter, int rstride, int kstep) {
    // one CTA per tile: the hardware scheduler hands out the tiles and a CTA
    // that finishes makes room for the next, so loads of many tiles are in
    // flight at once; the persistent grid walks the list with resident CTAs
    b->grid = b->flat ? std::max(1, b->ntiles) : b->resident;
    switch (b->model) {
        case LBM_CASCADED:
            return lbm::launch_batch_cascaded(b->grid, b->d_doms, b->d_tiles, b->ntiles, b->lbx, b->rows, flip, b->policy,
                                              counter, b->d_rtab, rstride, kstep, b->stream);
        case LBM_BGK:
            return lbm::launch_batch_bgk(b->grid, b->d_doms, b->d_tiles, b->ntiles, b->lbx, b->rows, flip, b->policy, counter,
                                         b->d_rtab, rstride, kstep, b->stream);
        default:
            return lbm::launch_batch_rawmrt(b->grid, b->d_doms, b->d_tiles, b->ntiles, b->lbx, b->rows, flip, b->policy,
                                            counter, b->d_rtab, rstride, kstep, b->stream);
    }
}

// One step outside a graph, `base` steps after the domains' counts (the counter
// of the dynamic policy is reset first).
cudaError_t launch_single(lbm_batch_s* b, int flip, long long base) {
    cudaError_t e = fill_round_table(b, 1, base);
    if (e == cudaSuccess && b->policy == lbm::kPolicyDynamic) e = cudaMemsetAsync(b->d_counters, 0, sizeof(int), b->stream);
    if (e != cudaSuccess) return e;
    return launch(b, flip, b->d_counters, 1, 0);
}

void drop_graph(lbm_batch_s* b) {
    if (b->graph) cudaGraphExecDestroy(b->graph);
    b->graph = nullptr;
    if (b->graph2) cudaGraphExecDestroy(b->graph2);
    b->graph2 = nullptr;
}

// ---------------------------------------------------------------- two steps per launch
// Every lattice admits two-step launches if it has at least 4 x 4 nodes (the
// storage kinds of a batch all do); a sequence of them needs every lattice at
// an even step, so a call whose lattices differ in parity takes single steps.
bool two_step_admitted(const lbm_batch_s* b) {
    for (const lbm_s* h : b->doms)
        if (h->a.nx < 4 || h->a.ny < 4) return false;
    return true;
}

bool same_parity(const lbm_batch_s* b) {
    for (const lbm_s* h : b->doms)
        if ((h->t & 1) != (b->doms[0]->t & 1)) return false;
    return true;
}

std::vector<int> domain_classes(const lbm_batch_s* b) {
    std::vector<int> c;
    for (const lbm_s* h : b->doms) c.push_back(lbm::batch_class(h->store, h->walls, lbm::force_mode(h), h->a.rseed != 0));
    return c;
}

// The 64 x 16 tiles of every lattice into dt, ordered by class and within a
// class largest lattice first; records the class ranges and the classes, and
// makes a branch stream for every class present after the first.
cudaError_t order_tiles2(lbm_batch_s* b, int* dt) {
    const std::vector<int> cls = domain_classes(b);
    std::vector<int> idx(b->doms.size());
    std::iota(idx.begin(), idx.end(), 0);
    auto nodes = [&](int d) { return (long long)b->doms[d]->a.nx * b->doms[d]->a.ny; };
    std::stable_sort(idx.begin(), idx.end(), [&](int p, int q) {
        return cls[p] != cls[q] ? cls[p] < cls[q] : nodes(p) > nodes(q);
    });
    std::vector<int> t;
    int first[lbm::kBatchClasses + 1] = {};
    for (int d : idx) {
        const int tx = (b->doms[d]->a.nx + lbm::kBatchFusedTX - 1) / lbm::kBatchFusedTX;
        const int ty = (b->doms[d]->a.ny + lbm::kBatchFusedTY - 1) / lbm::kBatchFusedTY;
        for (int j = 0; j < ty; ++j)
            for (int i = 0; i < tx; ++i) t.insert(t.end(), {d, i, j});
        first[cls[d] + 1] += tx * ty;
    }
    int present = 0;
    for (int c = 0; c < lbm::kBatchClasses; ++c) {
        present += first[c + 1] > 0;
        first[c + 1] += first[c];
    }
    cudaError_t e = cudaSuccess;
    if (!b->fork) e = cudaEventCreateWithFlags(&b->fork, cudaEventDisableTiming);
    while (e == cudaSuccess && int(b->branch.size()) < present - 1) {
        lbm_batch_s::Branch br{nullptr, nullptr};
        e = cudaStreamCreateWithFlags(&br.s, cudaStreamNonBlocking);
        if (e == cudaSuccess) e = cudaEventCreateWithFlags(&br.joined, cudaEventDisableTiming);
        if (e == cudaSuccess) {
            b->branch.push_back(br);
        } else {
            if (br.s) cudaStreamDestroy(br.s);
            if (br.joined) cudaEventDestroy(br.joined);
        }
    }
    if (e == cudaSuccess) e = cudaMemcpyAsync(dt, t.data(), t.size() * sizeof(int), cudaMemcpyHostToDevice, b->stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(b->stream);  // t is a local vector
    if (e != cudaSuccess) return e;
    std::copy(first, first + lbm::kBatchClasses + 1, b->class_first);
    b->cls2 = cls;
    return cudaSuccess;
}

// Second arrays and tensor maps of every lattice, the 64 x 16 tile list and
// the error word; made once.
cudaError_t prepare_two_step(lbm_batch_s* b) {
    if (b->h_pairs) return cudaSuccess;
    cudaError_t e = cudaSuccess;
    for (lbm_s* h : b->doms)
        if (e == cudaSuccess) e = lbm_prepare_two_step(h);
    size_t ntiles = 0;  // fewer than the one-step list's, whose size lbm_batch_create bounds
    for (const lbm_s* h : b->doms)
        ntiles += size_t((h->a.nx + lbm::kBatchFusedTX - 1) / lbm::kBatchFusedTX) *
                  ((h->a.ny + lbm::kBatchFusedTY - 1) / lbm::kBatchFusedTY);
    lbm::BatchPair* hp = nullptr;
    lbm::BatchPair* dp = nullptr;
    int* dt = nullptr;
    int* de = nullptr;
    if (e == cudaSuccess) e = cudaMallocHost((void**)&hp, b->doms.size() * sizeof(lbm::BatchPair));
    if (e == cudaSuccess) e = cudaMalloc((void**)&dp, b->doms.size() * sizeof(lbm::BatchPair));
    if (e == cudaSuccess) e = cudaMalloc((void**)&dt, 3 * ntiles * sizeof(int));
    if (e == cudaSuccess) e = cudaMalloc((void**)&de, sizeof(int));
    if (e == cudaSuccess) e = cudaMemsetAsync(de, 0, sizeof(int), b->stream);
    if (e == cudaSuccess) e = order_tiles2(b, dt);
    if (e != cudaSuccess) {  // nothing kept: a later call starts over
        if (hp) cudaFreeHost(hp);
        if (dp) cudaFree(dp);
        if (dt) cudaFree(dt);
        if (de) cudaFree(de);
        return e;
    }
    b->ntiles2 = int(ntiles);
    b->h_pairs = hp;
    b->d_pairs = dp;
    b->d_tiles2 = dt;
    b->d_err = de;
    return cudaSuccess;
}

cudaError_t launch_class(lbm_batch_s* b, int c, int k, int rstride, int kstep, cudaStream_t s) {
    const int n = b->class_first[c + 1] - b->class_first[c];
    const int* tiles = b->d_tiles2 + 3 * b->class_first[c];
    switch (b->model) {
        case LBM_CASCADED:
            return lbm::launch_batch_fused_cascaded(c, n, b->d_doms, b->d_pairs, tiles, k, b->d_rtab, rstride, kstep,
                                                    b->d_err, s);
        case LBM_BGK:
            return lbm::launch_batch_fused_bgk(c, n, b->d_doms, b->d_pairs, tiles, k, b->d_rtab, rstride, kstep,
                                               b->d_err, s);
        default:
            return lbm::launch_batch_fused_rawmrt(c, n, b->d_doms, b->d_pairs, tiles, k, b->d_rtab, rstride, kstep,
                                                  b->d_err, s);
    }
}

// Two-step launch k of a sequence (reads each lattice's arr[k & 1]); the round
// table holds rstride hashes per lattice, two per launch from 2 kstep.  One
// kernel per class present: the first on the batch stream, each other one on a
// branch stream that waits for the batch stream and that the batch stream then
// waits for, so the kernels run side by side (also inside a captured graph).
cudaError_t launch_pair(lbm_batch_s* b, int k, int rstride, int kstep) {
    int used[lbm::kBatchClasses];
    int n = 0;
    for (int c = 0; c < lbm::kBatchClasses; ++c)
        if (b->class_first[c + 1] > b->class_first[c]) used[n++] = c;
    if (n > int(b->branch.size()) + 1) return cudaErrorInvalidValue;
    cudaError_t e = n > 1 ? cudaEventRecord(b->fork, b->stream) : cudaSuccess;
    for (int i = 0; i < n && e == cudaSuccess; ++i) {
        if (i == 0) {
            e = launch_class(b, used[0], k, rstride, kstep, b->stream);
            continue;
        }
        const lbm_batch_s::Branch& br = b->branch[i - 1];
        e = cudaStreamWaitEvent(br.s, b->fork, 0);
        if (e == cudaSuccess) e = launch_class(b, used[i], k, rstride, kstep, br.s);
        if (e == cudaSuccess) e = cudaEventRecord(br.joined, br.s);
        if (e == cudaSuccess) e = cudaStreamWaitEvent(b->stream, br.joined, 0);
    }
    return e;
}

// Launches per replay of the two-step graph: graph_steps / 2, rounded down to an
// even number (the arrays are back in place after each replay).
int pair_graph_len(const lbm_batch_s* b) { return (b->graph_steps / 4) * 2; }

cudaError_t build_graph2(lbm_batch_s* b) {
    if (b->graph2) cudaGraphExecDestroy(b->graph2);
    b->graph2 = nullptr;
    const int len = pair_graph_len(b);
    cudaGraph_t g = nullptr;
    cudaError_t e = cudaStreamBeginCapture(b->stream, cudaStreamCaptureModeThreadLocal);
    if (e != cudaSuccess) return e;
    for (int k = 0; k < len && e == cudaSuccess; ++k) e = launch_pair(b, k & 1, 2 * len, k);
    cudaError_t e2 = cudaStreamEndCapture(b->stream, &g);
    if (e == cudaSuccess) e = e2;
    if (e == cudaSuccess) e = cudaGraphInstantiate(&b->graph2, g, 0);
    if (g) cudaGraphDestroy(g);
    return e;
}

// `pairs` two-step launches from the domains' current steps plus `base` (all
// even); the lattices' arrays trade roles if pairs is odd.
cudaError_t run_pairs(lbm_batch_s* b, long pairs, long long base) {
    cudaError_t e = cudaSuccess;
    long p = 0;
    const int len = pair_graph_len(b);
    if (len > 0 && pairs >= len) {
        if (!b->graph2) e = build_graph2(b);
        for (; e == cudaSuccess && pairs - p >= len; p += len) {
            e = fill_round_table(b, 2 * len, base + 2 * p);
            if (e == cudaSuccess) e = cudaGraphLaunch(b->graph2, b->stream);
        }
    }
    for (; e == cudaSuccess && p < pairs; ++p) {
        e = fill_round_table(b, 2, base + 2 * p);
        if (e == cudaSuccess) e = launch_pair(b, int(p & 1), 2, 0);
    }
    if (e == cudaSuccess && (pairs & 1)) {
        for (lbm_s* h : b->doms) {
            std::swap(h->state, h->state_alt);
            h->a.f = h->state;
        }
    }
    return e;
}

cudaError_t build_graph(lbm_batch_s* b) {
    drop_graph(b);
    cudaGraph_t g = nullptr;
    cudaError_t e = cudaStreamBeginCapture(b->stream, cudaStreamCaptureModeThreadLocal);
    if (e != cudaSuccess) return e;
    if (b->policy == lbm::kPolicyDynamic) e = cudaMemsetAsync(b->d_counters, 0, b->graph_steps * sizeof(int), b->stream);
    for (int k = 0; k < b->graph_steps && e == cudaSuccess; ++k)
        e = launch(b, k & 1, b->d_counters + k, b->graph_steps, k);
    cudaError_t e2 = cudaStreamEndCapture(b->stream, &g);
    if (e == cudaSuccess) e = e2;
    if (e == cudaSuccess) e = cudaGraphInstantiate(&b->graph, g, 0);
    if (g) cudaGraphDestroy(g);
    return e;
}

int blocks_per_sm(int model) {
    switch (model) {
        case LBM_CASCADED: return lbm::batch_blocks_per_sm_cascaded();
        case LBM_BGK: return lbm::batch_blocks_per_sm_bgk();
        default: return lbm::batch_blocks_per_sm_rawmrt();
    }
}

// Work on the domains' own streams that precedes the batch must finish first.
cudaError_t wait_for_domains(lbm_batch_s* b) {
    std::vector<cudaStream_t> seen;
    for (lbm_s* h : b->doms) {
        if (std::find(seen.begin(), seen.end(), h->stream) != seen.end()) continue;
        seen.push_back(h->stream);
        cudaError_t e = cudaStreamSynchronize(h->stream);
        if (e != cudaSuccess) return e;
    }
    return cudaSuccess;
}

// Later work on the domains' streams waits for the batch.
cudaError_t release_domains(lbm_batch_s* b) {
    cudaError_t e = cudaEventRecord(b->done, b->stream);
    std::vector<cudaStream_t> seen;
    for (lbm_s* h : b->doms) {
        if (e != cudaSuccess) break;
        if (std::find(seen.begin(), seen.end(), h->stream) != seen.end()) continue;
        seen.push_back(h->stream);
        e = cudaStreamWaitEvent(h->stream, b->done, 0);
    }
    return e;
}

#define BATCH_CUDA(call, what)                                                              \
    do {                                                                                    \
        cudaError_t e_ = (call);                                                            \
        if (e_ != cudaSuccess)                                                              \
            return lbm::set_error(e_ == cudaErrorMemoryAllocation ? LBM_ENOMEM : LBM_ECUDA, \
                                  "%s: %s", what, cudaGetErrorString(e_));                  \
    } while (0)

struct Guard {
    int prev = -1;
    explicit Guard(int dev) {
        cudaGetDevice(&prev);
        if (prev != dev) cudaSetDevice(dev);
    }
    ~Guard() {
        int cur;
        if (prev >= 0 && cudaGetDevice(&cur) == cudaSuccess && cur != prev) cudaSetDevice(prev);
    }
};

}  // namespace

extern "C" {

int lbm_batch_create(const lbm_t* lattices, int count, lbm_batch_t* out) {
    if (!lattices || count < 1 || !out) return fail(LBM_EINVAL, "lbm_batch_create: need count >= 1 lattices and out");
    const lbm_s* first = lattices[0];
    if (!first) return fail(LBM_EINVAL, "lbm_batch_create: null lattice");
    for (int i = 0; i < count; ++i) {
        const lbm_s* h = lattices[i];
        if (!h) return fail(LBM_EINVAL, "lbm_batch_create: null lattice");
        if (h->device != first->device) return fail(LBM_EINVAL, "lbm_batch_create: lattices on different devices");
        if (h->model != first->model) return fail(LBM_EINVAL, "lbm_batch_create: lattices of different models");
        if (h->store != LBM_F32 && h->store != LBM_F16DEV && h->store != LBM_BF16DEV)
            return fail(LBM_EINVAL, "lbm_batch_create: storage must be LBM_F32, LBM_BF16DEV or LBM_F16DEV");
        if (h->has_field) return fail(LBM_EINVAL, "lbm_batch_create: per-node force fields are not batched");
        for (int j = 0; j < i; ++j)
            if (lattices[j] == h) return fail(LBM_EINVAL, "lbm_batch_create: a lattice appears twice");
    }
    Guard g(first->device);
    lbm_batch_s* b = new lbm_batch_s;
    b->device = first->device;
    b->model = first->model;
    for (int i = 0; i < count; ++i) b->doms.push_back(lattices[i]);
    long long maxtiles = 0;
    for (int lbx : kShapes) {
        long long n = 0;
        for (lbm_s* h : b->doms) n += tiles_of(h, lbx, 1);  // one row per thread gives the most tiles
        maxtiles = std::max(maxtiles, n);
    }
    if (maxtiles > 0x7fffffffLL / 3) {
        delete b;
        return fail(LBM_EINVAL, "lbm_batch_create: too many tiles");
    }
    b->tiles_cap = size_t(3 * maxtiles);
    b->ncounters = 1 << 12;
    cudaError_t e = cudaStreamCreateWithFlags(&b->stream, cudaStreamNonBlocking);
    if (e == cudaSuccess) e = cudaEventCreateWithFlags(&b->done, cudaEventDisableTiming);
    if (e == cudaSuccess) e = cudaEventRecord(b->done, b->stream);
    if (e == cudaSuccess) e = cudaMallocHost((void**)&b->h_doms, count * sizeof(BatchDomain));
    if (e == cudaSuccess) e = cudaMalloc((void**)&b->d_doms, count * sizeof(BatchDomain));
    if (e == cudaSuccess) e = cudaMalloc((void**)&b->d_tiles, b->tiles_cap * sizeof(int));
    if (e == cudaSuccess) e = cudaMalloc((void**)&b->d_counters, b->ncounters * sizeof(int));
    if (e == cudaSuccess) e = cudaMalloc((void**)&b->d_rtab, size_t(count) * b->ncounters * sizeof(unsigned));
    if (e == cudaSuccess) e = cudaDeviceGetAttribute(&b->sms, cudaDevAttrMultiProcessorCount, b->device);
    if (e == cudaSuccess) {
        b->resident = b->sms * blocks_per_sm(b->model);
        b->grid = b->resident;
        e = upload_tiles(b, b->lbx, b->rows, b->order);
    }
    if (e == cudaSuccess) e = cudaStreamSynchronize(b->stream);
    if (e != cudaSuccess) {
        lbm_batch_destroy(b);
        return lbm::set_error(e == cudaErrorMemoryAllocation ? LBM_ENOMEM : LBM_ECUDA, "lbm_batch_create: %s",
                              cudaGetErrorString(e));
    }
    *out = b;
    return LBM_OK;
}

int lbm_batch_destroy(lbm_batch_t b) {
    if (!b) return LBM_OK;
    Guard g(b->device);
    if (b->stream) sync_all(b);
    drop_graph(b);
    if (b->d_counters) cudaFree(b->d_counters);
    if (b->h_pairs) cudaFreeHost(b->h_pairs);
    if (b->d_pairs) cudaFree(b->d_pairs);
    if (b->d_tiles2) cudaFree(b->d_tiles2);
    if (b->d_err) cudaFree(b->d_err);
    if (b->d_rtab) cudaFree(b->d_rtab);
    if (b->d_tiles) cudaFree(b->d_tiles);
    if (b->d_doms) cudaFree(b->d_doms);
    if (b->h_doms) cudaFreeHost(b->h_doms);
    for (const lbm_batch_s::Branch& br : b->branch) {
        cudaEventDestroy(br.joined);
        cudaStreamDestroy(br.s);
    }
    if (b->fork) cudaEventDestroy(b->fork);
    if (b->done) cudaEventDestroy(b->done);
    if (b->stream) cudaStreamDestroy(b->stream);
    delete b;
    return LBM_OK;
}

int lbm_batch_set_graph_steps(lbm_batch_t b, int steps) {
    if (!b) return fail(LBM_EINVAL, "null batch");
    if (steps < 0 || (steps & 1) || steps > b->ncounters)
        return fail(LBM_EINVAL, "lbm_batch_set_graph_steps: steps must be even, >= 0 and <= 4096");
    Guard g(b->device);
    BATCH_CUDA(cudaStreamSynchronize(b->stream), "lbm_batch_set_graph_steps");
    drop_graph(b);
    b->graph_steps = steps;
    return LBM_OK;
}

int lbm_batch_step(lbm_batch_t b, long n) {
    if (!b) return fail(LBM_EINVAL, "null batch");
    if (n < 0) return fail(LBM_EINVAL, "lbm_batch_step: n must be >= 0");
    if (n == 0) return LBM_OK;
    Guard g(b->device);
    for (lbm_s* h : b->doms)
        if (h->has_field) return fail(LBM_EINVAL, "lbm_batch_step: a lattice now has a per-node force field");
    BATCH_CUDA(wait_for_domains(b), "lbm_batch_step: waiting for the lattices' streams");
    BATCH_CUDA(refresh_domains(b), "lbm_batch_step: domain table");
    if (b->two_step && same_parity(b)) {  // [one step to an even step,] pairs of steps[, one step]
        long done = 0;
        if (b->doms[0]->t & 1) {
            BATCH_CUDA(launch_single(b, 0, 0), "lbm_batch_step: launch");
            done = 1;
        }
        const long pairs = (n - done) / 2;
        BATCH_CUDA(run_pairs(b, pairs, done), "lbm_batch_step: two-step launches");
        for (lbm_s* h : b->doms) h->t += done + 2 * pairs;
        if (done + 2 * pairs < n) {  // the arrays may have traded roles: a fresh table for the last step
            BATCH_CUDA(cudaStreamSynchronize(b->stream), "lbm_batch_step: sync");
            BATCH_CUDA(cudaEventRecord(b->done, b->stream), "lbm_batch_step: event");
            BATCH_CUDA(refresh_domains(b), "lbm_batch_step: domain table");
            BATCH_CUDA(launch_single(b, 0, 0), "lbm_batch_step: launch");
            for (lbm_s* h : b->doms) h->t += 1;
        }
        BATCH_CUDA(release_domains(b), "lbm_batch_step: event");
        return LBM_OK;
    }
    long done = 0;
    if (b->graph_steps > 0 && n >= b->graph_steps) {
        if (!b->graph) BATCH_CUDA(build_graph(b), "lbm_batch_step: graph capture");
        for (; n - done >= b->graph_steps; done += b->graph_steps) {
            BATCH_CUDA(fill_round_table(b, b->graph_steps, done), "lbm_batch_step: round table");
            BATCH_CUDA(cudaGraphLaunch(b->graph, b->stream), "lbm_batch_step: graph launch");
        }
    }
    for (long k = done; k < n; ++k) BATCH_CUDA(launch_single(b, int((k - done) & 1), k), "lbm_batch_step: launch");
    for (lbm_s* h : b->doms) h->t += n;
    BATCH_CUDA(release_domains(b), "lbm_batch_step: event");
    return LBM_OK;
}

int lbm_batch_sync(lbm_batch_t b) {
    if (!b) return fail(LBM_EINVAL, "null batch");
    Guard g(b->device);
    BATCH_CUDA(sync_all(b), "lbm_batch_sync");
    if (b->d_err) {  // a two-step launch whose tile load timed out (cleared once reported)
        int v = 0;
        BATCH_CUDA(cudaMemcpy(&v, b->d_err, sizeof(int), cudaMemcpyDeviceToHost), "lbm_batch_sync: error word");
        if (v) {
            cudaMemset(b->d_err, 0, sizeof(int));
            return fail(LBM_ECUDA, "lbm_batch_sync: a two-step launch timed out waiting for its tile load");
        }
    }
    return LBM_OK;
}

int lbm_batch_set_two_step(lbm_batch_t b, int on) {
    if (!b) return fail(LBM_EINVAL, "null batch");
    Guard g(b->device);
    if (on && !two_step_admitted(b))
        return fail(LBM_EINVAL, "lbm_batch_set_two_step: every lattice needs at least 4 x 4 nodes");
    BATCH_CUDA(cudaStreamSynchronize(b->stream), "lbm_batch_set_two_step");
    if (on) BATCH_CUDA(prepare_two_step(b), "lbm_batch_set_two_step: second arrays");
    b->two_step = on != 0;
    return LBM_OK;
}

int lbm_batch_tune(lbm_batch_t b, int trial_steps, float* best_ms) {
    if (!b) return fail(LBM_EINVAL, "null batch");
    if (trial_steps < 1) return fail(LBM_EINVAL, "lbm_batch_tune: trial_steps must be >= 1");
    Guard g(b->device);
    BATCH_CUDA(wait_for_domains(b), "lbm_batch_tune: waiting for the lattices' streams");
    BATCH_CUDA(cudaStreamSynchronize(b->stream), "lbm_batch_tune");
    // snapshot every domain (the trial steps must leave the states unchanged)
    size_t total = 0;
    for (lbm_s* h : b->doms) total += h->state_bytes;
    char* backup = nullptr;
    BATCH_CUDA(cudaMallocAsync((void**)&backup, total, b->stream), "lbm_batch_tune: snapshot allocation");
    auto copy_all = [&](bool save) {
        size_t off = 0;
        cudaError_t e = cudaSuccess;
        for (lbm_s* h : b->doms) {
            if (e == cudaSuccess)
                e = save ? cudaMemcpyAsync(backup + off, h->state, h->state_bytes, cudaMemcpyDeviceToDevice, b->stream)
                         : cudaMemcpyAsync(h->state, backup + off, h->state_bytes, cudaMemcpyDeviceToDevice, b->stream);
            off += h->state_bytes;
        }
        return e;
    };
    cudaEvent_t t0 = nullptr, t1 = nullptr;
    cudaError_t e = copy_all(true);
    if (e == cudaSuccess) e = cudaEventCreate(&t0);
    if (e == cudaSuccess) e = cudaEventCreate(&t1);
    if (e == cudaSuccess) e = refresh_domains(b);
    float best = 1e30f;
    int best_lbx = b->lbx, best_rows = b->rows, best_policy = b->policy, best_order = b->order;
    bool best_flat = b->flat;
    for (int rows : kRows) {
      for (int lbx : kShapes) {
        for (int order = 0; order < 2 && e == cudaSuccess; ++order) {
            e = upload_tiles(b, lbx, rows, order);
            for (int policy = 0; policy < 4 && e == cudaSuccess; ++policy) {  // 3: one CTA per tile
                b->lbx = lbx;
                b->rows = rows;
                b->order = order;
                b->flat = policy == 3;
                b->policy = b->flat ? lbm::kPolicyRoundRobin : policy;
                for (int k = 0; k < 2 && e == cudaSuccess; ++k) e = launch_single(b, k & 1, k);
                if (e == cudaSuccess) e = cudaEventRecord(t0, b->stream);
                for (int k = 0; k < trial_steps && e == cudaSuccess; ++k) e = launch_single(b, k & 1, k);
                if (e == cudaSuccess) e = cudaEventRecord(t1, b->stream);
                if (e == cudaSuccess) e = cudaEventSynchronize(t1);
                float ms = 0.f;
                if (e == cudaSuccess) e = cudaEventElapsedTime(&ms, t0, t1);
                if (e == cudaSuccess && ms < best) {
                    best = ms;
                    best_lbx = lbx;
                    best_rows = rows;
                    best_policy = b->policy;
                    best_order = order;
                    best_flat = b->flat;
                }
                if (e == cudaSuccess) e = copy_all(false);  // back to the snapshot for the next candidate
            }
        }
      }
    }
    // two steps per launch: an even number of launches, so the states end in
    // the arrays they started from
    bool best_two = false;
    float best_step = best / trial_steps;
    if (e == cudaSuccess && two_step_admitted(b) && same_parity(b) && (b->doms[0]->t & 1) == 0) {
        if (prepare_two_step(b) != cudaSuccess) {
            cudaGetLastError();  // no room for the second arrays: not a candidate
        } else {
            const int launches = std::max(2, ((trial_steps + 1) / 2 + 1) & ~1);
            e = cudaStreamSynchronize(b->stream);
            if (e == cudaSuccess) e = cudaEventRecord(b->done, b->stream);
            if (e == cudaSuccess) e = refresh_domains(b);
            if (e == cudaSuccess) e = fill_round_table(b, 2, 0);
            for (int k = 0; k < 2 && e == cudaSuccess; ++k) e = launch_pair(b, k & 1, 2, 0);
            if (e == cudaSuccess) e = cudaEventRecord(t0, b->stream);
            for (int k = 0; k < launches && e == cudaSuccess; ++k) e = launch_pair(b, k & 1, 2, 0);
            if (e == cudaSuccess) e = cudaEventRecord(t1, b->stream);
            if (e == cudaSuccess) e = cudaEventSynchronize(t1);
            float ms = 0.f;
            if (e == cudaSuccess) e = cudaEventElapsedTime(&ms, t0, t1);
            if (e == cudaSuccess && ms / (2 * launches) < best_step) {
                best_step = ms / (2 * launches);
                best_two = true;
            }
            if (e == cudaSuccess) e = copy_all(false);
        }
    }
    b->two_step = best_two;
    b->lbx = best_lbx;
    b->rows = best_rows;
    b->policy = best_policy;
    b->order = best_order;
    b->flat = best_flat;
    b->tuned_ms = best_step;
    if (e == cudaSuccess) e = upload_tiles(b, b->lbx, b->rows, b->order);
    if (e == cudaSuccess) e = copy_all(false);
    cudaFreeAsync(backup, b->stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(b->stream);
    if (t0) cudaEventDestroy(t0);
    if (t1) cudaEventDestroy(t1);
    drop_graph(b);
    if (e != cudaSuccess)
        return lbm::set_error(e == cudaErrorMemoryAllocation ? LBM_ENOMEM : LBM_ECUDA, "lbm_batch_tune: %s",
                              cudaGetErrorString(e));
    if (best_ms) *best_ms = b->tuned_ms;
    return LBM_OK;
}

int lbm_batch_info(lbm_batch_t b, int cfg[6], void** stream) {
    if (!b) return fail(LBM_EINVAL, "null batch");
    if (cfg && b->two_step) {
        cfg[0] = lbm::kBatchFusedTX;
        cfg[1] = lbm::kBatchFusedTY;
        cfg[2] = 4;
        cfg[3] = 0;
        cfg[4] = b->ntiles2;
        cfg[5] = b->ntiles2;
    } else if (cfg) {
        cfg[0] = 1 << b->lbx;
        cfg[1] = (lbm::kBatchThreads >> b->lbx) * b->rows;
        cfg[2] = b->flat ? 3 : b->policy;
        cfg[3] = b->order;
        cfg[4] = b->flat ? std::max(1, b->ntiles) : b->resident;
        cfg[5] = b->ntiles;
    }
    if (stream) *stream = b->stream;
    return LBM_OK;
}

}  // extern "C"
