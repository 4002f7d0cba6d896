/*
 * lbm.h -- C ABI of the GB300 (sm_103a) cascaded lattice Boltzmann library.
 *
 * The library advances a two-dimensional D2Q9 lattice with the cascaded
 * (central-moment MRT) collision of Ning & Premnath, Sec. II, Eq. (13)-(27),
 * or with one of the two sibling collisions the paper compares it with
 * (SRT-BGK and raw-moment MRT, Sec. IV-V).  One call to lbm_step performs
 * collide-and-stream (Eq. 23-24) at every node in one fused CUDA kernel.
 *
 * Conventions shared by every entry point
 *   - Every function returns an int status: LBM_OK (0) or one of the LBM_E*
 *     codes below; lbm_last_error() then gives a one-line message (per host
 *     thread).  No function aborts or prints.
 *   - Fields passed in or out are row-major with x fastest: a scalar field is
 *     [ny][nx], a vector field [2][ny][nx] (x component first), populations
 *     [9][ny][nx] in the paper's direction order (Eq. 1):
 *     e = (0,0) (1,0) (0,1) (-1,0) (0,-1) (1,1) (-1,1) (-1,-1) (1,-1).
 *   - Lattice units: node spacing 1, time step 1, c_s^2 = 1/3.  Node (i, j)
 *     sits at x = i, y = j; half-way bounce-back walls sit half a link outside
 *     the first and last nodes.
 *   - "host" pointers are ordinary (pageable or pinned) CPU memory; the call
 *     copies through a stream-ordered device buffer (lbm_init and lbm_macros
 *     access mapped page-locked buffers in place instead) and returns after
 *     the transfer has completed.  "device" pointers are CUDA device memory of
 *     the device that was current at lbm_create; those calls are asynchronous
 *     on the handle's stream.
 *   - A handle is used by one host thread at a time.  The library owns the
 *     device memory it allocates; lbm_destroy releases it.
 */
#ifndef LBM_GB300_H
#define LBM_GB300_H

#include <stddef.h>

#ifdef __cplusplus
extern "C" {
#endif

/* status codes */
#define LBM_OK 0
#define LBM_EINVAL 1    /* an argument is out of range or inconsistent */
#define LBM_ENOMEM 2    /* a device allocation failed */
#define LBM_ECUDA 3     /* a CUDA runtime call or kernel launch failed */
#define LBM_EDIVERGED 4 /* the divergence check found a non-finite or drifting state */

/* edge kinds, one per edge in the order west, east, south, north */
#define LBM_PERIODIC 0
#define LBM_BOUNCEBACK 1   /* half-way bounce-back, wall at rest (Sec. III-A) */
#define LBM_MOVING_WALL 2  /* half-way bounce-back with the moving-wall correction (Sec. III-C);
                              a diagonal link through a corner where two walls meet is bounced
                              back without it */
#define LBM_WEST 0
#define LBM_EAST 1
#define LBM_SOUTH 2
#define LBM_NORTH 3

/* collision models */
#define LBM_CASCADED 0 /* central-moment cascaded collision, Sec. II Eq. (13)-(25) */
#define LBM_BGK 1      /* single relaxation time, rate omega_4 (named in Sec. I, V) */
#define LBM_RAWMRT 2   /* raw-moment MRT in the basis K of Eq. (3) (named in Sec. IV-V) */

/* population storage; arithmetic is FP64 for LBM_F64 and FP32 otherwise.
 * The stored quantity is the deviation f_a - w_a rho0 (w = 4/9, 1/9, 1/36). */
#define LBM_F64 0
#define LBM_F32 1
#define LBM_BF16DEV 2 /* bfloat16 deviation, round to nearest even (or stochastically: lbm_set_rounding) */
#define LBM_F16DEV 3  /* IEEE half of 4096 x deviation, rounded as LBM_BF16DEV */

/* boundary specification: edge[k] is the kind of edge k (W, E, S, N);
 * wall_u[k] the tangential speed of a moving wall (along x on the south and
 * north edges, along y on the west and east edges; ignored otherwise).
 * Opposite edges must both be periodic or both be walls. */
typedef struct {
    int edge[4];
    double wall_u[4];
} lbm_bc_t;

typedef struct lbm_s* lbm_t;

/* Create a lattice of nx x ny nodes on the current CUDA device.
 *   omegas  : relaxation rates omega_3..omega_8, each in (0, 2) (Sec. II,
 *             after Eq. 22); omega_4 = omega_5 set the shear viscosity
 *             nu = (1/omega_4 - 1/2)/3.  BGK uses omega_4 only.
 *   force   : uniform body force (F_x, F_y) of Eq. (5); NULL means zero.
 *   bc      : edges; NULL means periodic on all four edges.
 *   model   : LBM_CASCADED, LBM_BGK or LBM_RAWMRT.
 *   store   : LBM_F64, LBM_F32, LBM_BF16DEV or LBM_F16DEV.
 *   rho0    : reference density (> 0): the deviation origin and the density
 *             used in the moving-wall correction.
 * The populations start at rest, f = w rho0.  Allocates 9*pitch*ny*sizeof(store)
 * bytes of device memory (pitch = nx rounded up to 32).
 * Errors: LBM_EINVAL (nx, ny < 1, ny > 65535 or nx*ny > 2^31 - 1; an omega outside (0,2);
 * unknown model, store or edge kind; mismatched periodic edges; rho0 <= 0;
 * out == NULL), LBM_ENOMEM, LBM_ECUDA.  *out is set only on success. */
int lbm_create(int nx, int ny, const double omegas[6], const double force[2], const lbm_bc_t* bc,
               int model, int store, double rho0, lbm_t* out);

/* Release the handle and its device memory (after the handle's stream has
 * drained).  lbm_destroy(NULL) is a no-op returning LBM_OK. */
int lbm_destroy(lbm_t h);

/* Launch all later work on this CUDA stream (a cudaStream_t; NULL is the
 * legacy default stream). */
int lbm_set_stream(lbm_t h, void* stream);

/* Replace the uniform body force (Eq. 5). */
int lbm_set_force(lbm_t h, const double force[2]);

/* Replace the relaxation rates omega_3..omega_8 (each in (0, 2)). */
int lbm_set_omegas(lbm_t h, const double omegas[6]);

/* Kernel variant of lbm_step for FP32-arithmetic storage (ignored for LBM_F64):
 * 0 = one node per thread; 1 = two rows per thread with packed FP32x2
 * arithmetic; 2 (LBM_BF16DEV and LBM_F16DEV only; LBM_F32 runs variant 0) =
 * four consecutive nodes of a row per thread, each population plane moved
 * with 64-bit accesses, elements at vector edges exchanged between
 * neighbouring lanes, and the per-node path where a neighbour wraps or a wall
 * is near; 3 (LBM_F32, LBM_BF16DEV, LBM_F16DEV) = two time steps per launch
 * (temporal blocking): a CTA loads a 64 x 16 tile with a two-node halo by one
 * TMA copy into shared memory, takes both steps there and writes the tile
 * once, so the populations cross HBM once per two steps.  Variant 3 keeps a
 * second population array (ping-pong, allocated by this call; LBM_ENOMEM if
 * it does not fit), runs pairs of steps from even steps and single steps
 * (variant 2 for 16-bit stores, else 0) otherwise, needs a lattice of at
 * least 4 x 4 nodes and is not used while the divergence check is on.
 * The default is 2 for 16-bit stores of at least 2^20 nodes and 0
 * otherwise (a smaller launch is latency-bound and one node per thread is
 * faster).
 * Variants 0, 2 and 3 produce bit-identical states; variant 1 may round
 * differently in the last bit because it fuses multiply-adds explicitly.
 * With a per-node force field variant 2 runs variant 0.  LBM_EINVAL for a
 * variant outside 0..3; a variant the storage kind does not admit selects 0. */
int lbm_set_variant(lbm_t h, int variant);

/* Rounding of the stored deviations (LBM_F32, LBM_BF16DEV, LBM_F16DEV).
 * LBM_ROUND_NEAREST (the default) rounds to nearest even.  LBM_ROUND_STOCHASTIC
 * rounds each stored value up with probability equal to its distance above the
 * representable value below, in units of their spacing, so that the stored
 * state is an unbiased estimate of the computed one.  Round to nearest loses
 * every per-step change smaller than half a spacing; over long runs this stalls
 * the slow viscous decay (a Taylor-Green vortex on 256^2 in FP16 ends one decay
 * time 22 % too strong), which stochastic rounding removes.  For FP32 storage
 * the computed value is known exactly: the last addition of the collision
 * (Eq. 25) is an error-free sum (TwoSum), and its remainder is rounded in.
 * The random bits come from a counter-based hash of (seed, step, node,
 * population): a run is reproducible for a given seed, independent of kernel
 * variant, CTA shape and CUDA-graph replay (variant 1 runs variant 0 in this
 * mode).  Costs extra integer and FP32 instructions per stored value.
 * LBM_EINVAL for another mode or for stochastic rounding with FP64 storage.
 * Batches (lbm_batch_*) round each lattice as it is set here, with the same
 * results as lbm_step; lbm_adjoint_run recomputes the rounded forward states
 * and differentiates the rounding as the identity. */
#define LBM_ROUND_NEAREST 0
#define LBM_ROUND_STOCHASTIC 1
int lbm_set_rounding(lbm_t h, int mode, unsigned long long seed);

/* Autotuner for one lattice: times `trial_steps` steps of each kernel variant
 * the storage admits with each CTA shape (128x2, 256x1, 64x4, 32x8 threads;
 * variant 3 has one fixed tile) on the lattice itself (the state is snapshot
 * and restored, so it is left unchanged) and keeps the fastest pair; ms (may
 * be NULL) receives the best time per step of variants 0..3 (0 where not run).
 * Synchronous. */
#define LBM_NUM_VARIANTS 4
int lbm_tune(lbm_t h, int trial_steps, float ms[LBM_NUM_VARIANTS]);

/* Per-node body force [2][ny][nx] added to the uniform force; NULL removes it.
 * on_device selects a device or a host pointer.  The library keeps its own
 * copy (FP64 for LBM_F64 storage, FP32 otherwise). */
int lbm_set_force_field(lbm_t h, const double* fxy, int on_device);

/* Set the populations to the equilibrium of the lattice's model at the given
 * density and velocity, in the transformed variable of Eq. (6):
 * f_bar = f_eq(rho, u) - S(u, F)/2, so that Eq. (26)-(27) return exactly
 * (rho, u).  The cascaded model uses the equilibrium whose central moments are
 * those of Eq. (10); BGK and raw MRT the second-order polynomial one.
 * rho [ny][nx] may be NULL (rho0 everywhere), u [2][ny][nx] may be NULL (rest).
 * Resets the step counter to 0.  _device: device pointers.  Host buffers in
 * page-locked memory mapped into the device address space (cudaHostAlloc,
 * cudaMallocHost, cudaHostRegister) are read by the kernel in place; other
 * host buffers are copied to a device staging buffer first.  Either way the
 * call is synchronous and the buffers must hold the sizes above. */
int lbm_init(lbm_t h, const double* rho, const double* u);
int lbm_init_device(lbm_t h, const double* rho, const double* u);

/* Advance n >= 0 time steps (collide Eq. 23 + stream Eq. 24 per step), one
 * fused kernel launch per step, asynchronously on the handle's stream.  Runs
 * of at least lbm_set_graph_steps steps starting at an even step are replayed
 * from a CUDA graph on an internal stream that is ordered after the handle's
 * stream and before any later work on it (the graph is recaptured whenever a
 * rate, force, force field, variant or rounding mode has changed).  With the divergence
 * check on (lbm_set_check) no graph is used, the call synchronises at every
 * check and returns LBM_EDIVERGED when it fails. */
int lbm_step(lbm_t h, long n);

/* Steps per CUDA-graph replay in lbm_step (even; 0 disables graphs; default 64). */
int lbm_set_graph_steps(lbm_t h, int steps);

/* Density [ny][nx] and velocity [2][ny][nx] of Eq. (26)-(27) at the current
 * time; either pointer may be NULL.  Host pointers: synchronous; mapped
 * page-locked buffers (as for lbm_init) are written by the kernel in place,
 * other host buffers through a device staging buffer. */
int lbm_macros(lbm_t h, double* rho, double* u);
int lbm_macros_device(lbm_t h, double* rho, double* u);

/* Local strain-rate quantities from the non-equilibrium moments of
 * f = f_bar + S/2, Eq. (28)-(30) solved exactly for the two normal
 * components: out [3][ny][nx] = (d_x j_x, d_y j_y, d_x j_y + d_y j_x).  The
 * inversion divides by the rates at which the model relaxes the second-order
 * moments: omega_3, omega_4, omega_5 (cascaded, raw MRT); omega_4 (BGK). */
int lbm_strain(lbm_t h, double* out);
int lbm_strain_device(lbm_t h, double* out);

/* Read or overwrite the populations f_bar [9][ny][nx] (FP64, full values,
 * not deviations) at the current time.  lbm_set_f resets the step counter to 0. */
int lbm_get_f(lbm_t h, double* f);
int lbm_set_f(lbm_t h, const double* f);
int lbm_get_f_device(lbm_t h, double* f);
int lbm_set_f_device(lbm_t h, const double* f);

/* Global sums in FP64 over all nodes: out = (sum rho, sum rho u_x, sum rho u_y)
 * with rho u from Eq. (27).  Synchronous; out is host memory. */
int lbm_stats(lbm_t h, double out[3]);

/* Divergence check: every `every` steps (0 = off) lbm_step computes
 * lbm_stats and fails with LBM_EDIVERGED if a sum is not finite or the mass
 * drifts from its value at the last init by more than mass_rtol (relative). */
int lbm_set_check(lbm_t h, long every, double mass_rtol);

/* Number of steps taken since create / init / set_f. */
long lbm_time(lbm_t h);

/* Layout facts: dims = (nx, ny, pitch, model, store, kernel variant, CTA
 * width of the step kernel); bytes = device bytes of the population array;
 * state = its device address (for profiling tools). */
int lbm_info(lbm_t h, long dims[7], size_t* bytes, void** state);

/* Algorithmic bytes one lattice update moves for a storage kind: 9 loads and
 * 9 stores of the stored type (144, 72, 36, 36); 0 for an unknown kind. */
size_t lbm_bytes_per_update(int store);

/* Discrete adjoint of a run (no counterpart in the paper, which has no
 * gradients): runs `nsteps` steps of the lattice from the transformed
 * equilibrium at (rho, u0) (as lbm_init_device) with the lattice's current
 * rates, uniform force and per-node force field, evaluates
 *     L = 1/2 sum_x |u(x, T) - u_target(x)|^2,   u from Eq. (26)-(27),
 * and its gradients by the exact discrete adjoint of the FP64/FP32 update:
 * reverse streaming plus the transposed cascaded collision per node, with the
 * states recomputed from checkpoints taken every `every` steps.
 *   rho [ny][nx] (NULL: rho0), u0 and u_target [2][ny][nx]: device, FP64.
 *   grad_u0, grad_force [2][ny][nx]: device, FP64, may be NULL; grad_force is
 *   dL/dF at every node (the gradient with respect to the per-node force
 *   field, whether or not one is set).
 *   loss (1 double) and grad_omega (dL/d omega_3..omega_8, 6 doubles): host.
 * Accumulation over time of dL/domega is FP64; dL/dF is summed in the
 * arithmetic type over the steps of one checkpoint segment and in FP64 across
 * segments (FP64 throughout for LBM_F64).  Requirements: the cascaded model,
 * LBM_F64 or LBM_F32 storage, four periodic edges.  The forward pass writes
 * each checkpoint directly (the step into a checkpoint runs out of place) and
 * the recomputed states of a segment are stepped out of place from it, so no
 * state is copied; every = 1 keeps every state and recomputes nothing.
 * Device memory used during the call: (ceil(nsteps/every) +
 * max(1, min(every, nsteps) - 1)) times the population array, two adjoint
 * arrays, a segment force-gradient array (FP32 storage) and small scratch,
 * allocated and released in stream order.  Synchronous.
 * Leaves the lattice at step nsteps. */
int lbm_adjoint_run(lbm_t h, long nsteps, long every, const double* rho, const double* u0, const double* u_target,
                    double* loss, double* grad_u0, double* grad_force, double grad_omega[6]);

/* ---------------------------------------------------------------------------
 * Batches: many independent lattices advanced together (no counterpart in the
 * paper).  One time step of every lattice in the batch is ONE launch of a
 * kernel whose CTAs walk a work list of (lattice, tile) items, or two steps
 * are one launch per class of lattice (lbm_batch_set_two_step); the per-node
 * update is exactly that of lbm_step, so results are bitwise equal.
 * Chunks of `graph_steps` steps (default 100, even) are replayed from a CUDA
 * graph.  All lattices must share the device and the collision model, use
 * LBM_F32, LBM_BF16DEV or LBM_F16DEV storage and have no per-node force field;
 * storage kinds, sizes, edges and uniform forces may differ.  The batch works
 * on its own stream: lbm_batch_step first waits (on the host) for the
 * lattices' streams, and later work on those streams waits for the batch.
 * A lattice must not be stepped on its own while it belongs to a live batch
 * call; lbm_step between batch calls is fine.  Destroy the batch before its
 * lattices. */
typedef struct lbm_batch_s* lbm_batch_t;

/* Errors: LBM_EINVAL (count < 1, NULL or repeated lattice, mixed devices or
 * models, FP64 storage, a force field), LBM_ENOMEM, LBM_ECUDA.  lbm_batch_step
 * fails with LBM_EINVAL if a lattice has since been given a force field. */
int lbm_batch_create(const lbm_t* lattices, int count, lbm_batch_t* out);
int lbm_batch_destroy(lbm_batch_t b);

/* Autotuner: times `trial_steps` launches of every tile shape (128x2, 256x1,
 * 64x4, 32x8 threads per 256-thread CTA, each thread updating one node row or
 * four node rows of the tile), work-list order (lattice by lattice,
 * largest first; or one tile of each lattice in turn) and scheduling policy
 * (a resident grid walking the list round robin, in contiguous chunks or
 * dynamically via an atomic counter; or one CTA per tile), and, where every
 * lattice admits it and all are at the same even step, two steps per launch
 * (lbm_batch_set_two_step); keeps the fastest.  The lattices' states are
 * snapshot and restored, so tuning leaves them unchanged.  best_ms (may be
 * NULL) receives the time per step. */
int lbm_batch_tune(lbm_batch_t b, int trial_steps, float* best_ms);

/* Advance every lattice of the batch by n >= 0 steps (asynchronous). */
int lbm_batch_step(lbm_batch_t b, long n);

/* Steps per CUDA graph (even, 0..4096; 0 disables graphs). */
int lbm_batch_set_graph_steps(lbm_batch_t b, int steps);

/* Wait for the batch's queued work.  LBM_ECUDA also if a two-step launch
 * timed out waiting for its tile load (the states are then invalid). */
int lbm_batch_sync(lbm_batch_t b);

/* Two steps per launch for the whole batch (on != 0): one CTA per 64 x 16
 * tile of any lattice takes both steps of the tile in shared memory (the tile
 * body of lbm_set_variant's variant 3, with its storage kind, edges, force and
 * rounding), so the populations cross HBM once per two steps.  Every lattice
 * gets a second population array (allocated here, kept by the lattice) and
 * the arrays trade roles at every launch.  lbm_batch_step then takes pairs of
 * steps from even steps and single batched steps for an odd start or end; a
 * call whose lattices are at steps of different parity takes single steps
 * only.  Each launch runs one kernel per class of lattice (storage kind,
 * walls, force, rounding) on streams of the batch's own, forked from and
 * joined back to the batch stream; a lattice that changes its force or
 * rounding between calls changes class, and the next call rebuilds the
 * batch's tile list (waiting for its queued work first).  Results are bit for
 * bit those of single steps.  Errors: LBM_EINVAL (a lattice smaller than
 * 4 x 4 nodes), LBM_ENOMEM, LBM_ECUDA. */
int lbm_batch_set_two_step(lbm_batch_t b, int on);

/* cfg = (tile width, tile height in nodes, policy (0 round robin, 1 chunks,
 * 2 dynamic, 3 one CTA per tile, 4 two steps per launch, one CTA per tile),
 * order, grid CTAs, tiles); stream
 * receives the batch's cudaStream_t (for timing with events).  Either may be NULL. */
int lbm_batch_info(lbm_batch_t b, int cfg[6], void** stream);

/* ---------------------------------------------------------------------------
 * Allocation-free variant of lbm_stats.  The paper has no counterpart: this is
 * an interface for callers that cannot call cudaMalloc (code running inside
 * another framework's memory pool or a fixed device-memory budget, drivers
 * that forbid allocation after start-up) and so cannot create a handle.
 *
 * The caller describes a population array it owns (the layout lbm_create
 * uses: [9][ny][pitch] deviations f - w rho0 of the stored type, in the
 * natural layout after an even number of steps, in the AA-swapped layout after
 * an odd number) and passes a device pointer `out` to 3 doubles, which
 * receives (sum rho, sum rho u_x, sum rho u_y) exactly as lbm_stats defines
 * them (uniform force only; no per-node force field).  The call is
 * asynchronous on `stream` (a cudaStream_t, NULL = legacy default stream) and
 * runs on the current device.
 *
 * Scratch: per-row partial sums live in a file-scope __device__ array of
 * 3 x LBM_NOALLOC_MAX_ROWS doubles (384 KiB) that every GPU loading this
 * library holds until the process exits.  ny > LBM_NOALLOC_MAX_ROWS is
 * rejected with LBM_EINVAL.  The array is shared by all calls and keeps the
 * last call's values; every call overwrites the rows it reads, so nothing has
 * to be cleared.  Calls that overlap on the GPU (concurrent streams or host
 * threads) race on the array and must be serialised by the caller.
 * The first call on each device looks up the array's device address
 * (cudaGetSymbolAddress, with that device current).  The address is kept per
 * device and looked up again by the first call after the device's context has
 * been replaced (for example by cudaDeviceReset).  Allocates nothing.  Errors: LBM_EINVAL (NULL
 * pointer, sizes, pitch < nx, unknown store or edge kind, one edge of an
 * opposite pair periodic and the other a wall), LBM_ECUDA. */
#define LBM_NOALLOC_MAX_ROWS 16384

typedef struct {
    int nx, ny;      /* lattice size */
    int pitch;       /* elements between consecutive rows (>= nx) */
    int store;       /* LBM_F64, LBM_F32, LBM_BF16DEV or LBM_F16DEV */
    int odd;         /* nonzero after an odd number of steps */
    double rho0;     /* reference density of the deviations */
    double force[2]; /* uniform body force (enters rho u as F/2, Eq. 27) */
    lbm_bc_t bc;     /* edges and wall speeds, as given to lbm_create */
} lbm_layout_t;

int lbm_stats_noalloc(const void* f, const lbm_layout_t* layout, double* out, void* stream);

/* Message of the last failed call on this host thread ("" if none). */
const char* lbm_last_error(void);

#ifdef __cplusplus
}
#endif

#endif /* LBM_GB300_H */
