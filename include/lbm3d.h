/*
 * lbm3d.h -- C ABI of the D3Q27 central-moment lattices of the GB300 library.
 *
 * The paper (Ning & Premnath, Sec. V-VI) names three-dimensional lattices as
 * future work and gives no 3-D formulas.  The library carries the method of
 * Sec. II to D3Q27 as a statement about central moments: the 27 central
 * moments kappa_ijk (i, j, k in {0, 1, 2}) of the transformed populations
 * f_bar = f - S/2 (Eq. 6) about u = (sum e f_bar + F/2)/rho (Eq. 26-27 in
 * 3-D) relax towards the discrete Maxwellian rho m_i m_j m_k, m = (1, 0, 1/3)
 * (Eq. 10 is its 2-D case): the trace of the second-order moments at
 * omega_bulk, their deviatoric and off-diagonal parts at omega_shear, the
 * moments of order 3, 4, 5 and 6 at omega_3 .. omega_6; density and the
 * first-order moments are not relaxed, and the source whose central moments
 * are (0; F; 0 ...) (Eq. 11 in 3-D) adds F to the first-order ones.
 * Shear viscosity nu = (1/omega_shear - 1/2)/3, bulk viscosity
 * zeta = (2/3)(1/omega_bulk - 1/2)/3.
 *
 * Conventions are those of lbm.h (status codes, lbm_last_error, host
 * pointers copied synchronously, one host thread per handle).  Fields are
 * row-major with x fastest: a scalar field [nz][ny][nx], a vector field
 * [3][nz][ny][nx], populations [27][nz][ny][nx] with direction
 * a = (e_x+1) + 3 (e_y+1) + 9 (e_z+1), e in {-1, 0, 1}^3.  All six faces are
 * periodic.  Storage: LBM_F64 or LBM_F32 (deviations f - w rho0, w the D3Q27
 * weights 8/27, 2/27, 1/54, 1/216; FP32 arithmetic for LBM_F32).
 */
#ifndef LBM3D_GB300_H
#define LBM3D_GB300_H

#include <stddef.h>

#include "lbm.h"

#ifdef __cplusplus
extern "C" {
#endif

typedef struct lbm3_s* lbm3_t;

/* Create a periodic nx x ny x nz D3Q27 lattice on the current device, at rest
 * (f = w rho0).  omegas = (omega_bulk, omega_shear, omega_3, omega_4, omega_5,
 * omega_6), each in (0, 2); force = uniform (F_x, F_y, F_z) or NULL; store =
 * LBM_F64, LBM_F32, LBM_BF16DEV or LBM_F16DEV (deviations f - w rho0 as in
 * include/lbm.h; FP16 holds 4096 times the deviation; the 16-bit kinds round
 * to nearest even).  Allocates 27 * pitch * ny * nz elements (pitch = nx
 * rounded up to 32).  Errors: LBM_EINVAL (sizes < 1, nz > 65535, padded plane
 * >= 2^31 elements, omega outside (0, 2), other storage kinds, rho0 <= 0,
 * non-finite force, out == NULL), LBM_ENOMEM, LBM_ECUDA. */
int lbm3_create(int nx, int ny, int nz, const double omegas[6], const double force[3], int store, double rho0,
                lbm3_t* out);
int lbm3_destroy(lbm3_t h);                 /* NULL is a no-op */
int lbm3_set_stream(lbm3_t h, void* stream);

/* Transformed equilibrium f_bar = f_eq(rho, u) - S(u, F)/2 (so that the
 * macroscopic fields return exactly rho and u); rho [nz][ny][nx] (NULL: rho0)
 * and u [3][nz][ny][nx] (NULL: rest), host memory.  Resets the step count. */
int lbm3_init(lbm3_t h, const double* rho, const double* u);

/* n collide-and-stream steps (Eq. 23-24), one fused kernel launch per step,
 * AA-pattern streaming in place; asynchronous on the handle's stream. */
int lbm3_step(lbm3_t h, long n);

/* rho [nz][ny][nx] and u [3][nz][ny][nx] (host, FP64; either may be NULL). */
int lbm3_macros(lbm3_t h, double* rho, double* u);

/* Populations f_bar [27][nz][ny][nx] as full FP64 values (host). */
int lbm3_get_f(lbm3_t h, double* f);
int lbm3_set_f(lbm3_t h, const double* f);   /* resets the step count */

long lbm3_time(lbm3_t h);                   /* -1 for NULL */
/* dims = (nx, ny, nz, pitch, store); bytes and state of the population array */
int lbm3_info(lbm3_t h, long dims[5], size_t* bytes, void** state);
/* Algorithmic bytes of one lattice update: 27 loads and 27 stores (432 FP64,
 * 216 FP32, 108 BF16/FP16; 0 for other kinds). */
size_t lbm3_bytes_per_update(int store);

#ifdef __cplusplus
}
#endif

#endif /* LBM3D_GB300_H */
