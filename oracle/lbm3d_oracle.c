/*
 * lbm3d_oracle.c -- plain FP64 CPU oracle of the central-moment (cascaded)
 * lattice Boltzmann method on the D3Q27 lattice: the method of Sec. II of the
 * paper (Ning & Premnath) carried to three dimensions as lbm3d_oracle.h states.
 *
 * TEST INFRASTRUCTURE ONLY -- see lbm3d_oracle.h.  Written for reading, not
 * for speed: every node is handled alone; central moments come from direct
 * sums over the 27 directions and the populations back from them by solving
 * the 27 x 27 system; collision of the whole lattice first, streaming second
 * (push form, Eq. 23-24).
 */
#include <math.h>
#include <string.h>

#include "lbm3d_oracle.h"

/* one-dimensional equilibrium moments of the discrete Maxwellian: m_0, m_1, m_2 */
static const double MEQ[3] = {1.0, 0.0, 1.0 / 3.0};

void oracle3_velocities(int e[27][3], double w[27]) {
    /* D1Q3 weights 1/6, 2/3, 1/6 for e = -1, 0, 1; D3Q27 takes their products */
    static const double w1[3] = {1.0 / 6.0, 2.0 / 3.0, 1.0 / 6.0};
    for (int a = 0; a < 27; ++a) {
        const int ix = a % 3, iy = (a / 3) % 3, iz = a / 9;
        e[a][0] = ix - 1;
        e[a][1] = iy - 1;
        e[a][2] = iz - 1;
        w[a] = w1[ix] * w1[iy] * w1[iz];
    }
}

static double ipow(double v, int n) {
    double r = 1.0;
    for (int k = 0; k < n; ++k) r *= v;
    return r;
}

/* M[m][a] = (e_ax - u_x)^i (e_ay - u_y)^j (e_az - u_z)^k, m = i + 3 j + 9 k */
static void central_matrix(const double u[3], double M[27][27]) {
    int e[27][3];
    double w[27];
    oracle3_velocities(e, w);
    for (int m = 0; m < 27; ++m) {
        const int i = m % 3, j = (m / 3) % 3, k = m / 9;
        for (int a = 0; a < 27; ++a)
            M[m][a] = ipow(e[a][0] - u[0], i) * ipow(e[a][1] - u[1], j) * ipow(e[a][2] - u[2], k);
    }
}

void oracle3_central_moments(const double f[27], const double u[3], double c[27]) {
    double M[27][27];
    central_matrix(u, M);
    for (int m = 0; m < 27; ++m) {
        double s = 0.0;
        for (int a = 0; a < 27; ++a) s += M[m][a] * f[a];
        c[m] = s;
    }
}

/* Solve M x = b by Gaussian elimination with partial pivoting (M is copied). */
static void solve27(double M[27][27], const double b[27], double x[27]) {
    double A[27][28];
    for (int r = 0; r < 27; ++r) {
        for (int q = 0; q < 27; ++q) A[r][q] = M[r][q];
        A[r][27] = b[r];
    }
    for (int col = 0; col < 27; ++col) {
        int piv = col;
        for (int r = col + 1; r < 27; ++r)
            if (fabs(A[r][col]) > fabs(A[piv][col])) piv = r;
        if (piv != col)
            for (int q = 0; q < 28; ++q) {
                const double t = A[col][q];
                A[col][q] = A[piv][q];
                A[piv][q] = t;
            }
        for (int r = col + 1; r < 27; ++r) {
            const double fct = A[r][col] / A[col][col];
            for (int q = col; q < 28; ++q) A[r][q] -= fct * A[col][q];
        }
    }
    for (int r = 26; r >= 0; --r) {
        double s = A[r][27];
        for (int q = r + 1; q < 27; ++q) s -= A[r][q] * x[q];
        x[r] = s / A[r][r];
    }
}

void oracle3_from_central_moments(const double c[27], const double u[3], double f[27]) {
    double M[27][27];
    central_matrix(u, M);
    solve27(M, c, f);
}

void oracle3_macros_node(const double fb[27], const double F[3], double* rho, double u[3]) {
    int e[27][3];
    double w[27];
    oracle3_velocities(e, w);
    double r = 0.0, j[3] = {0.0, 0.0, 0.0};
    for (int a = 0; a < 27; ++a) {
        r += fb[a];
        for (int d = 0; d < 3; ++d) j[d] += e[a][d] * fb[a];
    }
    *rho = r;
    for (int d = 0; d < 3; ++d) u[d] = (j[d] + 0.5 * F[d]) / r;
}

/* Populations whose central moments about u are (0; F; 0 ...). */
void oracle3_source(const double u[3], const double F[3], double S[27]) {
    double sigma[27];
    memset(sigma, 0, sizeof sigma);
    sigma[1] = F[0];  /* (1,0,0) */
    sigma[3] = F[1];  /* (0,1,0) */
    sigma[9] = F[2];  /* (0,0,1) */
    oracle3_from_central_moments(sigma, u, S);
}

/* Populations whose central moments about u are rho m_i m_j m_k. */
void oracle3_equilibrium(double rho, const double u[3], double out[27]) {
    double c[27];
    for (int m = 0; m < 27; ++m) c[m] = rho * MEQ[m % 3] * MEQ[(m / 3) % 3] * MEQ[m / 9];
    oracle3_from_central_moments(c, u, out);
}

void oracle3_collide(const double fb[27], const double F[3], const double om[6], double out[27]) {
    double rho, u[3];
    oracle3_macros_node(fb, F, &rho, u);
    double c[27], cp[27];
    oracle3_central_moments(fb, u, c);
    memcpy(cp, c, sizeof c);
    /* second order: trace at omega_bulk towards rho, deviators and
       off-diagonal moments at omega_shear towards 0 */
    const int xx = 2, yy = 6, zz = 18, xy = 4, xz = 10, yz = 12;
    const double ob = om[0], os = om[1];
    const double T = c[xx] + c[yy] + c[zz], D1 = c[xx] - c[yy], D2 = c[xx] - c[zz];
    const double Tp = T + ob * (rho - T), D1p = (1.0 - os) * D1, D2p = (1.0 - os) * D2;
    cp[xx] = (Tp + D1p + D2p) / 3.0;
    cp[yy] = (Tp - 2.0 * D1p + D2p) / 3.0;
    cp[zz] = (Tp + D1p - 2.0 * D2p) / 3.0;
    cp[xy] = (1.0 - os) * c[xy];
    cp[xz] = (1.0 - os) * c[xz];
    cp[yz] = (1.0 - os) * c[yz];
    /* orders 3 .. 6 towards rho m_i m_j m_k at omega_3 .. omega_6 */
    for (int m = 0; m < 27; ++m) {
        const int i = m % 3, j = (m / 3) % 3, k = m / 9, n = i + j + k;
        if (n < 3) continue;
        const double eq = rho * MEQ[i] * MEQ[j] * MEQ[k];
        cp[m] = c[m] + om[n - 1] * (eq - c[m]);
    }
    /* density and first-order moments are not relaxed; the source adds F to
       the first-order ones (its central moments are (0; F; 0 ...)) */
    cp[1] += F[0];
    cp[3] += F[1];
    cp[9] += F[2];
    oracle3_from_central_moments(cp, u, out);
}

static long idx(const oracle3_lattice* L, int a, int x, int y, int z) {
    return (((long)a * L->nz + z) * L->ny + y) * L->nx + x;
}

void oracle3_init(const oracle3_lattice* L, const double* rho, const double* u, double* f) {
    const long n = (long)L->nx * L->ny * L->nz;
    for (int z = 0; z < L->nz; ++z)
        for (int y = 0; y < L->ny; ++y)
            for (int x = 0; x < L->nx; ++x) {
                const long p = ((long)z * L->ny + y) * L->nx + x;
                const double uu[3] = {u[p], u[n + p], u[2 * n + p]};
                double feq[27], S[27];
                oracle3_equilibrium(rho[p], uu, feq);
                oracle3_source(uu, L->force, S);
                for (int a = 0; a < 27; ++a) f[idx(L, a, x, y, z)] = feq[a] - 0.5 * S[a];
            }
}

void oracle3_collide_all(const oracle3_lattice* L, const double* f, double* post) {
    for (int z = 0; z < L->nz; ++z)
        for (int y = 0; y < L->ny; ++y)
            for (int x = 0; x < L->nx; ++x) {
                double fb[27], out[27];
                for (int a = 0; a < 27; ++a) fb[a] = f[idx(L, a, x, y, z)];
                oracle3_collide(fb, L->force, L->omega, out);
                for (int a = 0; a < 27; ++a) post[idx(L, a, x, y, z)] = out[a];
            }
}

void oracle3_stream_all(const oracle3_lattice* L, const double* post, double* f) {
    int e[27][3];
    double w[27];
    oracle3_velocities(e, w);
    for (int a = 0; a < 27; ++a)
        for (int z = 0; z < L->nz; ++z)
            for (int y = 0; y < L->ny; ++y)
                for (int x = 0; x < L->nx; ++x) {
                    const int xt = (x + e[a][0] + L->nx) % L->nx;
                    const int yt = (y + e[a][1] + L->ny) % L->ny;
                    const int zt = (z + e[a][2] + L->nz) % L->nz;
                    f[idx(L, a, xt, yt, zt)] = post[idx(L, a, x, y, z)];
                }
}

void oracle3_run(const oracle3_lattice* L, double* f, double* work, long nsteps) {
    for (long s = 0; s < nsteps; ++s) {
        oracle3_collide_all(L, f, work);
        oracle3_stream_all(L, work, f);
    }
}

void oracle3_macros(const oracle3_lattice* L, const double* f, double* rho, double* u) {
    const long n = (long)L->nx * L->ny * L->nz;
    for (int z = 0; z < L->nz; ++z)
        for (int y = 0; y < L->ny; ++y)
            for (int x = 0; x < L->nx; ++x) {
                const long p = ((long)z * L->ny + y) * L->nx + x;
                double fb[27], r, uu[3];
                for (int a = 0; a < 27; ++a) fb[a] = f[idx(L, a, x, y, z)];
                oracle3_macros_node(fb, L->force, &r, uu);
                rho[p] = r;
                for (int d = 0; d < 3; ++d) u[d * n + p] = uu[d];
            }
}
