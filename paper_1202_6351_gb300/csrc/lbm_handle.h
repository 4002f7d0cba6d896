// lbm_handle.h -- the state behind an lbm_t handle (include/lbm.h), shared by
// the host-side translation units of the library.
#pragma once

#include "lbm_internal.h"

// The state behind an lbm_t handle (include/lbm.h).
struct lbm_s {
    int device = 0;
    lbm::Args a{};
    int model = 0, store = 0;
    int edge[4] = {0, 0, 0, 0};
    double wall_u[4] = {0, 0, 0, 0};
    bool walls = false;
    bool has_field = false;
    long t = 0;                  // steps since create / init / set_f (parity selects the AA kernel)
    cudaStream_t stream = nullptr;
    void* state = nullptr;       // populations [9][ny][pitch] of the stored type
    size_t state_bytes = 0;
    void* ffield = nullptr;      // per-node force [2][ny][nx], FP64 for LBM_F64 storage, FP32 otherwise
    double* partials = nullptr;  // [3 * stats_blocks] FP64 scratch of lbm_stats
    double* sums = nullptr;      // [3] device result of lbm_stats
    long check_every = 0;
    double check_rtol = 0.0, mass0 = 0.0;
    // CUDA-graph replay of lbm_step: `graph_steps` launches captured from an even
    // step on an internal stream, ordered against `stream` by two events; the
    // launch arguments it was captured with are kept to detect any change.
    int graph_steps = 64;
    cudaGraphExec_t graph = nullptr;
    cudaStream_t gstream = nullptr;
    cudaEvent_t ev_in = nullptr, ev_out = nullptr;
    lbm::Args graph_args{};
    int graph_force = -1;
    // Stochastic rounding of 16-bit stores (lbm_set_rounding): per-step hashes
    // C0 of a graph replay, filled on the graph stream before each replay.
    unsigned* d_rtable = nullptr;
    int rtable_cap = 0;
    // Two fused steps per launch (variant 3): the second population array of
    // the ping-pong, a TMA descriptor of each array (tmap[k] describes
    // tmap_ptr[k]) and the kernels' error word.  Allocated on first use.
    void* state_alt = nullptr;
    CUtensorMap tmap[2];
    void* tmap_ptr[2] = {nullptr, nullptr};
    int* d_err = nullptr;
};

// The second population array and the tensor maps of both arrays (variant 3),
// made on first use; lbm_batch_* uses them for its two-step launches.
cudaError_t lbm_prepare_two_step(lbm_s* h);
// The tensor map of population array `base` (h->state or h->state_alt) after
// lbm_prepare_two_step.
const CUtensorMap& lbm_tensor_map(const lbm_s* h, const void* base);
