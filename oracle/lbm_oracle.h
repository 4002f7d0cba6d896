/*
 * lbm_oracle.h -- plain FP64 CPU statement of the cascaded (central-moment MRT)
 * lattice Boltzmann method on the D2Q9 lattice (Ning & Premnath, Sec. II).
 *
 * TEST INFRASTRUCTURE ONLY.  This is the slow, obviously-correct reference that
 * the CUDA path is checked against.  Only tests/, __graft_entry__.smoke() and
 * bench.py (its cpu_baseline / reference leg) may load it.  It shares no code,
 * header, constant table or helper with the CUDA library and never calls it.
 *
 * The same source is compiled twice: with `real` = double (liblbm_oracle.so)
 * and, with -DORACLE_COMPLEX, `real` = double _Complex (liblbm_oracle_cs.so,
 * every symbol suffixed _cs) so that complex-step derivatives of a whole run
 * can be taken.  Nothing in the arithmetic branches on a value, so the complex
 * build computes the same function extended analytically.
 *
 * Population layout everywhere: f[a][y][x], a = 0..8 in the paper's order
 * (Eq. 1), x fastest, nx*ny nodes per plane.  Parameters are passed through
 * arrays of `real` so that the complex build needs no by-value complex.
 */
#ifndef LBM_ORACLE_H
#define LBM_ORACLE_H

#ifdef ORACLE_COMPLEX
#include <complex.h>
typedef double _Complex real;
#define ONAME(x) x##_cs
#else
typedef double real;
#define ONAME(x) x
#endif

/* edge kinds and edge order (west, east, south, north) */
#define ORACLE_PERIODIC 0
#define ORACLE_BOUNCEBACK 1
#define ORACLE_MOVING_WALL 2

/* collision models */
#define ORACLE_CASCADED 0
#define ORACLE_BGK 1
#define ORACLE_RAWMRT 2

typedef struct {
    int nx, ny;
    int model;            /* ORACLE_CASCADED | ORACLE_BGK | ORACLE_RAWMRT */
    int edge[4];          /* W, E, S, N */
    real omega[6];        /* omega_3 .. omega_8 (Sec. II, after Eq. 22) */
    real force[2];        /* uniform body force (F_x, F_y), Eq. 5 */
    real wall_u[4];       /* tangential wall speed per edge (x for S/N, y for W/E) */
    real rho_w;           /* density used in the moving-wall correction */
    const real* force_field; /* optional per-node force, [2][ny][nx]; NULL -> uniform */
} oracle_lattice;

/* per-node pieces (each cites its equations in the .c file) */
void ONAME(oracle_macros_node)(const real fb[9], const real F[2], real* rho, real* ux, real* uy);
void ONAME(oracle_source)(const real u[2], const real F[2], real S[9]);
void ONAME(oracle_collide_cascaded)(const real fb[9], const real F[2], const real om[6], real out[9]);
void ONAME(oracle_collide_bgk)(const real fb[9], const real F[2], const real om[6], real out[9]);
void ONAME(oracle_collide_rawmrt)(const real fb[9], const real F[2], const real om[6], real out[9]);
void ONAME(oracle_equilibrium_cascaded)(const real rho_u[3], real out[9]);
void ONAME(oracle_equilibrium_poly)(const real rho_u[3], real out[9]);
void ONAME(oracle_strain_node)(const real fb[9], const real F[2], const real om[6], real out[3]);

/* whole-lattice operations */
void ONAME(oracle_init)(const oracle_lattice* L, const real* rho, const real* u, real* f);
void ONAME(oracle_collide_all)(const oracle_lattice* L, const real* f, real* post);
void ONAME(oracle_stream_all)(const oracle_lattice* L, const real* post, real* f);
void ONAME(oracle_run)(const oracle_lattice* L, real* f, real* work, long nsteps);
void ONAME(oracle_macros)(const oracle_lattice* L, const real* f, real* rho, real* u);
void ONAME(oracle_strain)(const oracle_lattice* L, const real* f, real* out);

#endif
