/*
 * lbm3d_oracle.h -- plain FP64 CPU statement of the central-moment (cascaded)
 * lattice Boltzmann method carried to three dimensions on the D3Q27 lattice.
 *
 * TEST INFRASTRUCTURE ONLY.  Only tests/, __graft_entry__.smoke() and bench.py
 * (its cpu_baseline / reference leg) may load it.  It shares no code, header,
 * constant table or helper with the CUDA library and never calls it.
 *
 * The paper (Sec. V-VI) names three-dimensional lattices as future work and
 * gives no 3-D formulas.  This oracle takes the two-dimensional method of
 * Sec. II as a statement about central moments and writes it out for D3Q27:
 *   - the central moments kappa_ijk = sum_a (e_ax-u_x)^i (e_ay-u_y)^j
 *     (e_az-u_z)^k f_bar_a, i, j, k in {0, 1, 2}, about the velocity
 *     u = (sum_a e_a f_bar_a + F/2)/rho (Eq. 26-27 in 3-D);
 *   - their equilibrium is the discrete Maxwellian rho m_i m_j m_k with
 *     m_0 = 1, m_1 = 0, m_2 = 1/3 (Eq. 10 is its 2-D case);
 *   - the density and the first-order moments are not relaxed; every other
 *     moment relaxes towards its equilibrium: the trace of the second-order
 *     tensor at omega_bulk, its deviatoric and off-diagonal parts at
 *     omega_shear, the third-, fourth-, fifth- and sixth-order moments at
 *     omega_3 .. omega_6;
 *   - the forcing adds the source whose central moments are (0; F; 0 ...)
 *     (Eq. 11 in 3-D), and the stored variable is f_bar = f - S/2 (Eq. 6).
 * Everything is the definition written out: moments by direct summation over
 * the 27 directions, the back-transform by solving the 27 x 27 system with
 * Gaussian elimination, collide-all then stream-all in push form, periodic
 * edges in all three directions.
 *
 * Layout: f[a][z][y][x], x fastest.  Direction a = (e_x+1) + 3 (e_y+1) +
 * 9 (e_z+1) (tensor order).  Moment index m = i + 3 j + 9 k.
 */
#ifndef LBM3D_ORACLE_H
#define LBM3D_ORACLE_H

typedef struct {
    int nx, ny, nz;
    double omega[6];  /* omega_bulk, omega_shear, omega_3, omega_4, omega_5, omega_6 */
    double force[3];  /* uniform body force */
} oracle3_lattice;

void oracle3_velocities(int e[27][3], double w[27]);
void oracle3_macros_node(const double fb[27], const double F[3], double* rho, double u[3]);
void oracle3_central_moments(const double f[27], const double u[3], double c[27]);
void oracle3_from_central_moments(const double c[27], const double u[3], double f[27]);
void oracle3_collide(const double fb[27], const double F[3], const double om[6], double out[27]);
void oracle3_equilibrium(double rho, const double u[3], double out[27]);
void oracle3_source(const double u[3], const double F[3], double S[27]);

void oracle3_init(const oracle3_lattice* L, const double* rho, const double* u, double* f);
void oracle3_collide_all(const oracle3_lattice* L, const double* f, double* post);
void oracle3_stream_all(const oracle3_lattice* L, const double* post, double* f);
void oracle3_run(const oracle3_lattice* L, double* f, double* work, long nsteps);
void oracle3_macros(const oracle3_lattice* L, const double* f, double* rho, double* u);

#endif
