// lbm_internal.h -- host-side declarations shared by the library's translation units.
#pragma once

#include <cuda.h>
#include <cuda_runtime.h>

#include "lbm_device.cuh"

struct lbm_s;  // the handle behind lbm_t (lbm_handle.h)

namespace lbm {

// 0: no force, 1: uniform force only, 2: per-node field (plus the uniform force).
int force_mode(const lbm_s* h);

// One fused step of any storage kind on the population array a.f.
cudaError_t launch_step_any(const Args& a, int store, int model, bool odd, int force, bool walls, cudaStream_t s);

// Launch shape of the fused step kernel: one thread per node, BX x BY threads.
constexpr int kStepBX = 128;
constexpr int kStepBY = 2;

// One fused collide-and-stream step (defined once per storage type).
cudaError_t launch_step_f64(const Args& a, int model, bool odd, int force, bool walls, cudaStream_t s);
cudaError_t launch_step_f32(const Args& a, int model, bool odd, int force, bool walls, cudaStream_t s);
cudaError_t launch_step_bf16(const Args& a, int model, bool odd, int force, bool walls, cudaStream_t s);
cudaError_t launch_step_f16(const Args& a, int model, bool odd, int force, bool walls, cudaStream_t s);

// Two fused steps (variant 3, lbm_fused.cuh) from a.f (natural layout, even
// step) into `out`; `map` describes a.f.  FP32, BF16 and FP16 storage.
cudaError_t launch_fused_f32(const CUtensorMap& map, const Args& a, void* out, int* err, int model, int force,
                             bool walls, cudaStream_t s);
cudaError_t launch_fused_bf16(const CUtensorMap& map, const Args& a, void* out, int* err, int model, int force,
                              bool walls, cudaStream_t s);
cudaError_t launch_fused_f16(const CUtensorMap& map, const Args& a, void* out, int* err, int model, int force,
                             bool walls, cudaStream_t s);

// Auxiliary kernels (lbm_aux.cu); every field argument is dense [..][ny][nx] FP64 device memory.
cudaError_t launch_init(const Args& a, int store, int model, int force, const double* rho, const double* u,
                        cudaStream_t s);
cudaError_t launch_set_f(const Args& a, int store, const double* f, cudaStream_t s);
cudaError_t launch_get_f(const Args& a, int store, bool odd, bool walls, double* f, cudaStream_t s);
cudaError_t launch_macros(const Args& a, int store, bool odd, bool walls, int force, double* rho, double* u,
                          cudaStream_t s);
cudaError_t launch_strain(const Args& a, int store, bool odd, bool walls, int force, double* out, cudaStream_t s);
// FP64 sums (rho, rho ux, rho uy) into partials[3 * nblocks] then out[3] (device).
int stats_blocks(const Args& a);
cudaError_t launch_stats(const Args& a, int store, bool odd, bool walls, int force, double* partials, double* out,
                         cudaStream_t s);

// Record the message returned by lbm_last_error() and return `code`.
int set_error(int code, const char* fmt, ...);

// dst[i] = (float)src[i], round to nearest.
cudaError_t launch_narrow(const double* src, float* dst, size_t n, cudaStream_t s);

}  // namespace lbm
