/*
 * lbm_oracle.c -- plain FP64 CPU oracle of the cascaded central-moment LBM
 * (Ning & Premnath, "Numerical study of the properties of the central moment
 * lattice Boltzmann method", Sec. II), plus the two sibling collision models
 * the paper compares against in Sec. IV-V (SRT-BGK and raw-moment MRT).
 *
 * TEST INFRASTRUCTURE ONLY -- see lbm_oracle.h.  Written for reading, not for
 * speed: every node is handled alone, collision of the whole lattice is done
 * first and streaming second, in the push form in which Eq. (23)-(24) are
 * written.  No blocking, fusion or reordering.
 *
 * Readings of the paper that this file takes:
 *   - weights w_a (used in Sec. III-C but never printed) are the unique D2Q9
 *     populations whose central moments are (1,0,0,1/3,1/3,0,0,0,1/9) at u = 0,
 *     i.e. Eq. (10) with rho = 1: (4/9, 1/9 x4, 1/36 x4).
 *   - in Eq. (20)-(21) the source moments written without a prime are the raw
 *     moments sigma'_xxy, sigma'_xyy of Eq. (13) (the central ones vanish by
 *     Eq. (11)); only this reading makes the post-collision central moments
 *     equal their relaxation targets.
 *   - the moving-wall correction of Sec. III-C is applied along the wall:
 *     f_b(x) = f~_bbar(x) + 6 w_b rho_w (e_b . U_wall), with rho_w = rho_0.
 *   - a diagonal link that crosses the corner point where two walls meet
 *     (e.g. the lid and a side wall of the cavity) is bounced back with no
 *     moving-wall term.  Sec. III-C lists the lid's incoming directions
 *     without saying which wall owns such a link; giving it the lid term
 *     makes the cavity converge at first order, not the second order that
 *     Sec. III-C reports for it.
 *   - initial populations are the transformed equilibrium of Eq. (12),
 *     i.e. f_bar = f_eq(rho, u) - S/2.
 *   - SRT-BGK and raw-moment MRT are only named by the paper; they are
 *     defined here with the second-order polynomial equilibrium and the same
 *     source S_a of Eq. (14).
 *   - the strain rates of Eq. (28)-(30) divide by the rate at which each
 *     non-equilibrium moment relaxes; under BGK that is omega_4 for all three.
 */
#include <string.h>
#include "lbm_oracle.h"

/* D2Q9 particle velocities: the rows |e_ax>, |e_ay> of Eq. (1). */
static const int EX[9] = {0, 1, 0, -1, 0, 1, -1, -1, 1};
static const int EY[9] = {0, 0, 1, 0, -1, 1, 1, -1, -1};
/* opposite direction abar: e_abar = -e_a */
static const int OPP[9] = {0, 3, 4, 1, 2, 7, 8, 5, 6};
/* weights (reading above) */
static const double W[9] = {4.0 / 9, 1.0 / 9, 1.0 / 9, 1.0 / 9, 1.0 / 9,
                            1.0 / 36, 1.0 / 36, 1.0 / 36, 1.0 / 36};

/* The orthogonal basis matrix K of Eq. (3): row a = population, column b = K_b. */
static const int KMAT[9][9] = {
    {1, 0, 0, -4, 0, 0, 0, 0, 4},
    {1, 1, 0, -1, 1, 0, 0, 2, -2},
    {1, 0, 1, -1, -1, 0, 2, 0, -2},
    {1, -1, 0, -1, 1, 0, 0, -2, -2},
    {1, 0, -1, -1, -1, 0, -2, 0, -2},
    {1, 1, 1, 2, 0, 1, -1, -1, 1},
    {1, -1, 1, 2, 0, -1, -1, 1, 1},
    {1, -1, -1, 2, 0, 1, 1, 1, 1},
    {1, 1, -1, 2, 0, -1, 1, -1, 1},
};

/* ------------------------------------------------------------------------ */
/* Macroscopic fields, Eq. (26)-(27): rho = sum f_bar, rho u = sum f_bar e + F/2 */
void ONAME(oracle_macros_node)(const real fb[9], const real F[2], real* rho, real* ux, real* uy)
{
    real r = 0, jx = 0, jy = 0;
    for (int a = 0; a < 9; ++a) {
        r += fb[a];
        jx += EX[a] * fb[a];
        jy += EY[a] * fb[a];
    }
    *rho = r;
    *ux = (jx + 0.5 * F[0]) / r;
    *uy = (jy + 0.5 * F[1]) / r;
}

/* Source term in velocity space: orthogonal source moments m^s (the list before Eq. 14)
 * inverted with K^-1 = D^-1 K^T into S_0..S_8 of Eq. (14). */
void ONAME(oracle_source)(const real u[2], const real F[2], real S[9])
{
    const real ux = u[0], uy = u[1], Fx = F[0], Fy = F[1];
    /* the m^s list before Eq. (14) */
    const real m1 = Fx;
    const real m2 = Fy;
    const real m3 = 6.0 * (Fx * ux + Fy * uy);
    const real m4 = 2.0 * (Fx * ux - Fy * uy);
    const real m5 = Fx * uy + Fy * ux;
    const real m6 = (2.0 - 3.0 * ux * ux) * Fy - 6.0 * Fx * ux * uy;
    const real m7 = (2.0 - 3.0 * uy * uy) * Fx - 6.0 * Fy * uy * ux;
    const real m8 = 6.0 * ((3.0 * uy * uy - 2.0) * Fx * ux + (3.0 * ux * ux - 2.0) * Fy * uy);
    /* Eq. (14) */
    S[0] = (1.0 / 9.0) * (-m3 + m8);
    S[1] = (1.0 / 36.0) * (6.0 * m1 - m3 + 9.0 * m4 + 6.0 * m7 - 2.0 * m8);
    S[2] = (1.0 / 36.0) * (6.0 * m2 - m3 - 9.0 * m4 + 6.0 * m6 - 2.0 * m8);
    S[3] = (1.0 / 36.0) * (-6.0 * m1 - m3 + 9.0 * m4 - 6.0 * m7 - 2.0 * m8);
    S[4] = (1.0 / 36.0) * (-6.0 * m2 - m3 - 9.0 * m4 - 6.0 * m6 - 2.0 * m8);
    S[5] = (1.0 / 36.0) * (6.0 * m1 + 6.0 * m2 + 2.0 * m3 + 9.0 * m5 - 3.0 * m6 - 3.0 * m7 + m8);
    S[6] = (1.0 / 36.0) * (-6.0 * m1 + 6.0 * m2 + 2.0 * m3 - 9.0 * m5 - 3.0 * m6 + 3.0 * m7 + m8);
    S[7] = (1.0 / 36.0) * (-6.0 * m1 - 6.0 * m2 + 2.0 * m3 + 9.0 * m5 + 3.0 * m6 + 3.0 * m7 + m8);
    S[8] = (1.0 / 36.0) * (6.0 * m1 - 6.0 * m2 + 2.0 * m3 - 9.0 * m5 + 3.0 * m6 - 3.0 * m7 + m8);
}

/* ------------------------------------------------------------------------ */
/* Cascaded collision, Sec. II: f~_bar = f_bar + K g^ + S  (Eq. 23, 25). */
void ONAME(oracle_collide_cascaded)(const real fb[9], const real F[2], const real om[6], real out[9])
{
    const real w3 = om[0], w4 = om[1], w5 = om[2], w6 = om[3], w7 = om[4], w8 = om[5];
    const real Fx = F[0], Fy = F[1];

    /* Eq. (26)-(27) */
    real rho, ux, uy;
    ONAME(oracle_macros_node)(fb, F, &rho, &ux, &uy);

    /* Eq. (15): raw moments of the transformed populations f_bar */
    const real kxx = fb[1] + fb[3] + fb[5] + fb[6] + fb[7] + fb[8];
    const real kyy = fb[2] + fb[4] + fb[5] + fb[6] + fb[7] + fb[8];
    const real kxy = (fb[5] + fb[7]) - (fb[6] + fb[8]);
    const real kxxy = (fb[5] + fb[6]) - (fb[7] + fb[8]);
    const real kxyy = (fb[5] + fb[8]) - (fb[6] + fb[7]);
    const real kxxyy = fb[5] + fb[6] + fb[7] + fb[8];

    /* Eq. (13): raw moments of the source */
    const real sxx = 2.0 * Fx * ux;
    const real syy = 2.0 * Fy * uy;
    const real sxy = Fx * uy + Fy * ux;
    const real sxxy = Fy * ux * ux + 2.0 * Fx * ux * uy;
    const real sxyy = Fx * uy * uy + 2.0 * Fy * uy * ux;
    const real sxxyy = 2.0 * Fx * ux * uy * uy + 2.0 * Fy * uy * ux * ux;

    /* Eq. (17)-(22): the collision kernel, in cascade order */
    const real g3 = (w3 / 12.0) * ((2.0 / 3.0) * rho + rho * (ux * ux + uy * uy)
                                   - (kxx + kyy) - 0.5 * (sxx + syy));
    const real g4 = (w4 / 4.0) * (rho * (ux * ux - uy * uy) - (kxx - kyy) - 0.5 * (sxx - syy));
    const real g5 = (w5 / 4.0) * (rho * ux * uy - kxy - 0.5 * sxy);
    const real g6 = (w6 / 4.0) * (2.0 * rho * ux * ux * uy + kxxy - 2.0 * ux * kxy - uy * kxx - 0.5 * sxxy)
                    - 0.5 * uy * (3.0 * g3 + g4) - 2.0 * ux * g5;
    const real g7 = (w7 / 4.0) * (2.0 * rho * ux * uy * uy + kxyy - 2.0 * uy * kxy - ux * kyy - 0.5 * sxyy)
                    - 0.5 * ux * (3.0 * g3 - g4) - 2.0 * uy * g5;
    const real g8 = (w8 / 4.0) * ((1.0 / 9.0) * rho + 3.0 * rho * ux * ux * uy * uy
                                  - (kxxyy - 2.0 * ux * kxyy - 2.0 * uy * kxxy + ux * ux * kyy
                                     + uy * uy * kxx + 4.0 * ux * uy * kxy)
                                  - 0.5 * sxxyy)
                    - 2.0 * g3 - 0.5 * uy * uy * (3.0 * g3 + g4) - 0.5 * ux * ux * (3.0 * g3 - g4)
                    - 4.0 * ux * uy * g5 - 2.0 * uy * g6 - 2.0 * ux * g7;

    /* Eq. (14) source in velocity space */
    real S[9];
    const real u[2] = {ux, uy};
    ONAME(oracle_source)(u, F, S);

    /* Eq. (25): explicit post-collision populations (g0 = g1 = g2 = 0) */
    out[0] = fb[0] + (-4.0 * (g3 - g8)) + S[0];
    out[1] = fb[1] + (-g3 + g4 + 2.0 * (g7 - g8)) + S[1];
    out[2] = fb[2] + (-g3 - g4 + 2.0 * (g6 - g8)) + S[2];
    out[3] = fb[3] + (-g3 + g4 - 2.0 * (g7 + g8)) + S[3];
    out[4] = fb[4] + (-g3 - g4 - 2.0 * (g6 + g8)) + S[4];
    out[5] = fb[5] + (2.0 * g3 + g5 - g6 - g7 + g8) + S[5];
    out[6] = fb[6] + (2.0 * g3 - g5 - g6 + g7 + g8) + S[6];
    out[7] = fb[7] + (2.0 * g3 + g5 + g6 + g7 + g8) + S[7];
    out[8] = fb[8] + (2.0 * g3 - g5 + g6 - g7 + g8) + S[8];
}

/* ------------------------------------------------------------------------ */
/* Populations from the nine raw moments r[m][n] = sum_a e_ax^m e_ay^n f_a
 * (m, n in 0..2): the inverse of the monomial basis of Eq. (1). */
static void pops_from_raw(const real r[3][3], real f[9])
{
    f[0] = r[0][0] - r[2][0] - r[0][2] + r[2][2];
    f[1] = 0.5 * (r[1][0] + r[2][0] - r[1][2] - r[2][2]);
    f[2] = 0.5 * (r[0][1] + r[0][2] - r[2][1] - r[2][2]);
    f[3] = 0.5 * (-r[1][0] + r[2][0] + r[1][2] - r[2][2]);
    f[4] = 0.5 * (-r[0][1] + r[0][2] + r[2][1] - r[2][2]);
    f[5] = 0.25 * (r[1][1] + r[2][1] + r[1][2] + r[2][2]);
    f[6] = 0.25 * (-r[1][1] + r[2][1] - r[1][2] + r[2][2]);
    f[7] = 0.25 * (r[1][1] - r[2][1] - r[1][2] + r[2][2]);
    f[8] = 0.25 * (-r[1][1] - r[2][1] + r[1][2] + r[2][2]);
}

static real ipow(real x, int n)
{
    real p = 1;
    for (int i = 0; i < n; ++i) p *= x;
    return p;
}

/* Binomial formula of Sec. II (between Eq. 12 and 13): raw moments from central
 * moments c[i][j] about u:  r_mn = sum_{i<=m, j<=n} C(m,i) C(n,j) u_x^(m-i) u_y^(n-j) c_ij. */
static void raw_from_central(const real c[3][3], real ux, real uy, real r[3][3])
{
    static const int C[3][3] = {{1, 0, 0}, {1, 1, 0}, {1, 2, 1}}; /* C[p][q] = p choose q */
    for (int m = 0; m < 3; ++m)
        for (int n = 0; n < 3; ++n) {
            real s = 0;
            for (int i = 0; i <= m; ++i)
                for (int j = 0; j <= n; ++j)
                    s += C[m][i] * C[n][j] * ipow(ux, m - i) * ipow(uy, n - j) * c[i][j];
            r[m][n] = s;
        }
}

/* Cascaded (central-moment) equilibrium of f: the populations whose central
 * moments about u are those of Eq. (10), (rho,0,0,rho/3,rho/3,0,0,0,rho/9). */
void ONAME(oracle_equilibrium_cascaded)(const real rho_u[3], real out[9])
{
    const real rho = rho_u[0];
    real c[3][3];
    memset(c, 0, sizeof c);
    c[0][0] = rho;
    c[2][0] = rho / 3.0;
    c[0][2] = rho / 3.0;
    c[2][2] = rho / 9.0;
    real r[3][3];
    raw_from_central(c, rho_u[1], rho_u[2], r);
    pops_from_raw(r, out);
}

/* Second-order polynomial equilibrium used by the SRT and raw-MRT siblings:
 * f_eq = w rho (1 + 3 e.u + 9/2 (e.u)^2 - 3/2 u.u). */
void ONAME(oracle_equilibrium_poly)(const real rho_u[3], real out[9])
{
    const real rho = rho_u[0], ux = rho_u[1], uy = rho_u[2];
    const real uu = ux * ux + uy * uy;
    for (int a = 0; a < 9; ++a) {
        const real eu = EX[a] * ux + EY[a] * uy;
        out[a] = W[a] * rho * (1.0 + 3.0 * eu + 4.5 * eu * eu - 1.5 * uu);
    }
}

/* SRT-BGK sibling: f~_bar = f_bar - w (f_bar - f_eq) + (1 - w/2) S, with the
 * single rate w = omega_4 (the shear rate). */
void ONAME(oracle_collide_bgk)(const real fb[9], const real F[2], const real om[6], real out[9])
{
    const real w = om[1];
    real rho, ux, uy;
    ONAME(oracle_macros_node)(fb, F, &rho, &ux, &uy);
    const real ru[3] = {rho, ux, uy};
    real feq[9], S[9];
    ONAME(oracle_equilibrium_poly)(ru, feq);
    const real u[2] = {ux, uy};
    ONAME(oracle_source)(u, F, S);
    for (int a = 0; a < 9; ++a)
        out[a] = fb[a] - w * (fb[a] - feq[a]) + (1.0 - 0.5 * w) * S[a];
}

/* Raw-moment MRT sibling in the orthogonal basis K of Eq. (3):
 * f~_bar = f_bar - K D^-1 [ L (K^T f_bar - K^T f_eq) - (I - L/2) K^T S ],
 * L = diag(0,0,0,omega_3..omega_8), D = diag(K^T K). */
void ONAME(oracle_collide_rawmrt)(const real fb[9], const real F[2], const real om[6], real out[9])
{
    real rho, ux, uy;
    ONAME(oracle_macros_node)(fb, F, &rho, &ux, &uy);
    const real ru[3] = {rho, ux, uy};
    real feq[9], S[9];
    ONAME(oracle_equilibrium_poly)(ru, feq);
    const real u[2] = {ux, uy};
    ONAME(oracle_source)(u, F, S);

    real lam[9];
    lam[0] = lam[1] = lam[2] = 0;
    for (int b = 3; b < 9; ++b) lam[b] = om[b - 3];

    real dm[9];
    for (int b = 0; b < 9; ++b) {
        real m = 0, meq = 0, ms = 0;
        double d = 0;
        for (int a = 0; a < 9; ++a) {
            m += KMAT[a][b] * fb[a];
            meq += KMAT[a][b] * feq[a];
            ms += KMAT[a][b] * S[a];
            d += KMAT[a][b] * KMAT[a][b];
        }
        dm[b] = (lam[b] * (m - meq) - (1.0 - 0.5 * lam[b]) * ms) / d;
    }
    for (int a = 0; a < 9; ++a) {
        real s = 0;
        for (int b = 0; b < 9; ++b) s += KMAT[a][b] * dm[b];
        out[a] = fb[a] - s;
    }
}

/* Local strain rate from non-equilibrium moments, Eq. (28)-(33).  The
 * moments are those of the untransformed f = f_bar + S/2.  The three relations
 * of Eq. (28)-(30) are solved exactly for the two normal components, which
 * differs from Eq. (31)-(32) as printed only when omega_3 != omega_4.
 * out = (d_x j_x, d_y j_y, d_x j_y + d_y j_x). */
void ONAME(oracle_strain_node)(const real fb[9], const real F[2], const real om[6], real out[3])
{
    real rho, ux, uy;
    ONAME(oracle_macros_node)(fb, F, &rho, &ux, &uy);
    real S[9], f[9];
    const real u[2] = {ux, uy};
    ONAME(oracle_source)(u, F, S);
    for (int a = 0; a < 9; ++a) f[a] = fb[a] + 0.5 * S[a];
    real kxx = 0, kyy = 0, kxy = 0;
    for (int a = 0; a < 9; ++a) {
        kxx += EX[a] * EX[a] * f[a];
        kyy += EY[a] * EY[a] * f[a];
        kxy += EX[a] * EY[a] * f[a];
    }
    /* non-equilibrium raw moments f^_3, f^_4, f^_5 (text after Eq. 30) */
    const real n3 = (kxx + kyy) - ((2.0 / 3.0) * rho + rho * (ux * ux + uy * uy));
    const real n4 = (kxx - kyy) - rho * (ux * ux - uy * uy);
    const real n5 = kxy - rho * ux * uy;
    const real div = -1.5 * om[0] * n3;   /* Eq. (28): d_x j_x + d_y j_y */
    const real dif = -1.5 * om[1] * n4;   /* Eq. (29): d_x j_x - d_y j_y */
    out[0] = 0.5 * (div + dif);
    out[1] = 0.5 * (div - dif);
    out[2] = -3.0 * om[2] * n5;           /* Eq. (30) */
}

/* ------------------------------------------------------------------------ */
/* whole-lattice operations */

static void node_force(const oracle_lattice* L, long node, long plane, real F[2])
{
    F[0] = L->force[0];
    F[1] = L->force[1];
    if (L->force_field) {
        F[0] += L->force_field[node];
        F[1] += L->force_field[plane + node];
    }
}

/* Initial state: the transformed equilibrium f_bar = f_eq - S/2 (Eq. 6, 12),
 * with the model's own f_eq.  rho may be NULL (rho = 1 is not assumed: the
 * caller passes it), u is [2][ny][nx] and may be NULL (rest). */
void ONAME(oracle_init)(const oracle_lattice* L, const real* rho, const real* u, real* f)
{
    const long plane = (long)L->nx * L->ny;
    for (long n = 0; n < plane; ++n) {
        real F[2];
        node_force(L, n, plane, F);
        const real ru[3] = {rho ? rho[n] : 1.0, u ? u[n] : 0.0, u ? u[plane + n] : 0.0};
        real feq[9], S[9];
        if (L->model == ORACLE_CASCADED)
            ONAME(oracle_equilibrium_cascaded)(ru, feq);
        else
            ONAME(oracle_equilibrium_poly)(ru, feq);
        const real uu[2] = {ru[1], ru[2]};
        ONAME(oracle_source)(uu, F, S);
        for (int a = 0; a < 9; ++a) f[a * plane + n] = feq[a] - 0.5 * S[a];
    }
}

/* Collision at every node, Eq. (23). */
void ONAME(oracle_collide_all)(const oracle_lattice* L, const real* f, real* post)
{
    const long plane = (long)L->nx * L->ny;
    for (long n = 0; n < plane; ++n) {
        real fb[9], out[9], F[2];
        for (int a = 0; a < 9; ++a) fb[a] = f[a * plane + n];
        node_force(L, n, plane, F);
        if (L->model == ORACLE_CASCADED)
            ONAME(oracle_collide_cascaded)(fb, F, L->omega, out);
        else if (L->model == ORACLE_BGK)
            ONAME(oracle_collide_bgk)(fb, F, L->omega, out);
        else
            ONAME(oracle_collide_rawmrt)(fb, F, L->omega, out);
        for (int a = 0; a < 9; ++a) post[a * plane + n] = out[a];
    }
}

/* Streaming, Eq. (24), in push form: f_bar(x + e_a) <- f~_bar_a(x).  A link
 * leaving the lattice through a periodic edge re-enters on the other side; one
 * leaving through a wall is reflected into the opposite direction at the same
 * node (half-way bounce-back, Sec. III-A), with the moving-wall correction of
 * Sec. III-C.  A diagonal link that leaves through the corner point of two
 * walls is reflected with no moving-wall term (reading in the header). */
void ONAME(oracle_stream_all)(const oracle_lattice* L, const real* post, real* f)
{
    const int nx = L->nx, ny = L->ny;
    const long plane = (long)nx * ny;
    for (int y = 0; y < ny; ++y)
        for (int x = 0; x < nx; ++x)
            for (int a = 0; a < 9; ++a) {
                const real v = post[a * plane + (long)y * nx + x];
                int dx = x + EX[a], dy = y + EY[a];
                const int yw = dy < 0 ? 2 : (dy >= ny ? 3 : -1);
                const int xw = dx < 0 ? 0 : (dx >= nx ? 1 : -1);
                const int ywall = yw >= 0 && L->edge[yw] != ORACLE_PERIODIC;
                const int xwall = xw >= 0 && L->edge[xw] != ORACLE_PERIODIC;
                const int corner = ywall && xwall;
                const int wall = ywall ? yw : (xwall ? xw : -1);
                if (wall >= 0) {
                    const int b = OPP[a];
                    real corr = 0;
                    if (!corner && L->edge[wall] == ORACLE_MOVING_WALL) {
                        /* tangential wall velocity: along x on S/N, along y on W/E */
                        const real Ux = (wall >= 2) ? L->wall_u[wall] : 0.0;
                        const real Uy = (wall >= 2) ? 0.0 : L->wall_u[wall];
                        corr = 6.0 * W[b] * L->rho_w * (EX[b] * Ux + EY[b] * Uy);
                    }
                    f[b * plane + (long)y * nx + x] = v + corr;
                } else {
                    dx = (dx + nx) % nx;
                    dy = (dy + ny) % ny;
                    f[a * plane + (long)dy * nx + dx] = v;
                }
            }
}

void ONAME(oracle_run)(const oracle_lattice* L, real* f, real* work, long nsteps)
{
    for (long s = 0; s < nsteps; ++s) {
        ONAME(oracle_collide_all)(L, f, work);
        ONAME(oracle_stream_all)(L, work, f);
    }
}

void ONAME(oracle_macros)(const oracle_lattice* L, const real* f, real* rho, real* u)
{
    const long plane = (long)L->nx * L->ny;
    for (long n = 0; n < plane; ++n) {
        real fb[9], F[2], r, ux, uy;
        for (int a = 0; a < 9; ++a) fb[a] = f[a * plane + n];
        node_force(L, n, plane, F);
        ONAME(oracle_macros_node)(fb, F, &r, &ux, &uy);
        if (rho) rho[n] = r;
        if (u) {
            u[n] = ux;
            u[plane + n] = uy;
        }
    }
}

void ONAME(oracle_strain)(const oracle_lattice* L, const real* f, real* out)
{
    const long plane = (long)L->nx * L->ny;
    /* Eq. (28)-(30) divide by the rates at which the second-order moments relax:
     * omega_3, omega_4, omega_5 for the cascaded and raw-MRT collisions, the
     * single rate omega_4 for BGK. */
    real om[6];
    for (int k = 0; k < 6; ++k) om[k] = L->omega[k];
    if (L->model == ORACLE_BGK) om[0] = om[2] = om[1];
    for (long n = 0; n < plane; ++n) {
        real fb[9], F[2], s[3];
        for (int a = 0; a < 9; ++a) fb[a] = f[a * plane + n];
        node_force(L, n, plane, F);
        ONAME(oracle_strain_node)(fb, F, om, s);
        for (int k = 0; k < 3; ++k) out[k * plane + n] = s[k];
    }
}
