// lbm_adjoint.cuh -- reverse mode of the cascaded collision (per node, in registers).
//
// The forward map is d~ = d + K g(d, F) + S(u, F) (Sec. II, Eq. 13-25, on
// deviations).  Given mu = dL/dd~ at one node, collide_cascaded_vjp returns
// dL/dd = (d d~/d d)^T mu, dL/dF (the node's force) and dL/dc (the six
// coefficients c3 = omega_3/12, c4..c8 = omega_4..8/4).  It recomputes the
// forward intermediates, then walks the cascade backwards: g8, then g7 and g6
// (which feed g8), then g5, g4, g3, then the raw source moments, the velocity
// u = (j + F/2)/rho and finally the raw moments of d, whose transposes are
// signed sums over the nine directions.  No matrix is formed.
#pragma once

#include "lbm_device.cuh"

namespace lbm {

// Adds (dS/du)^T mu and (dS/dF)^T mu to the four accumulators, for the source
// S = K D^-1 m^s(u, F) of Eq. (14) with the m^s list before it: dL/dm^s_b = (K^T mu)_b / D_b, with
// D = (9, 6, 6, 36, 4, 4, 12, 12, 36), then through the polynomials m^s_b.
template <typename R>
LBM_HD void source_vjp(R ux, R uy, R Fx, R Fy, const R mu[9], R& ux_a, R& uy_a, R& Fx_a, R& Fy_a) {
    const R m5p6 = mu[5] + mu[6], m7p8 = mu[7] + mu[8];
    const R diag = m5p6 + m7p8, axis = mu[1] + mu[2] + mu[3] + mu[4];
    const R uxx = ux * ux, uyy = uy * uy, uxy = ux * uy;
    const R s1 = ((mu[1] - mu[3]) + (mu[5] + mu[8]) - (mu[6] + mu[7])) * R(1.0 / 6.0);
    const R s2 = ((mu[2] - mu[4]) + m5p6 - m7p8) * R(1.0 / 6.0);
    const R s3 = (R(-4) * mu[0] - axis + R(2) * diag) * R(1.0 / 36.0);
    const R s4 = ((mu[1] + mu[3]) - (mu[2] + mu[4])) * R(0.25);
    const R s5 = ((mu[5] + mu[7]) - (mu[6] + mu[8])) * R(0.25);
    const R s6 = (R(2) * (mu[2] - mu[4]) - m5p6 + m7p8) * R(1.0 / 12.0);
    const R s7 = (R(2) * (mu[1] - mu[3]) - (mu[5] + mu[8]) + (mu[6] + mu[7])) * R(1.0 / 12.0);
    const R s8 = (R(4) * mu[0] - R(2) * axis + diag) * R(1.0 / 36.0);
    // m1 = Fx, m2 = Fy
    Fx_a += s1;
    Fy_a += s2;
    // m3 = 6 (Fx ux + Fy uy)
    Fx_a += R(6) * ux * s3; ux_a += R(6) * Fx * s3; Fy_a += R(6) * uy * s3; uy_a += R(6) * Fy * s3;
    // m4 = 2 (Fx ux - Fy uy)
    Fx_a += R(2) * ux * s4; ux_a += R(2) * Fx * s4; Fy_a -= R(2) * uy * s4; uy_a -= R(2) * Fy * s4;
    // m5 = Fx uy + Fy ux
    Fx_a += uy * s5; uy_a += Fx * s5; Fy_a += ux * s5; ux_a += Fy * s5;
    // m6 = (2 - 3 ux^2) Fy - 6 Fx ux uy
    ux_a += (R(-6) * ux * Fy - R(6) * Fx * uy) * s6;
    uy_a += R(-6) * Fx * ux * s6;
    Fx_a += R(-6) * uxy * s6;
    Fy_a += (R(2) - R(3) * uxx) * s6;
    // m7 = (2 - 3 uy^2) Fx - 6 Fy uy ux
    ux_a += R(-6) * Fy * uy * s7;
    uy_a += (R(-6) * uy * Fx - R(6) * Fy * ux) * s7;
    Fx_a += (R(2) - R(3) * uyy) * s7;
    Fy_a += R(-6) * uxy * s7;
    // m8 = 6 ((3 uy^2 - 2) Fx ux + (3 ux^2 - 2) Fy uy)
    ux_a += R(6) * ((R(3) * uyy - R(2)) * Fx + R(6) * ux * Fy * uy) * s8;
    uy_a += R(6) * (R(6) * uy * Fx * ux + (R(3) * uxx - R(2)) * Fy) * s8;
    Fx_a += R(6) * (R(3) * uyy - R(2)) * ux * s8;
    Fy_a += R(6) * (R(3) * uxx - R(2)) * uy * s8;
}

template <typename R>
struct CollideAdjoint {
    R d[9];        // dL/dd (pre-collision deviations)
    R Fx, Fy;      // dL/dF at the node
    R c[6];        // dL/dc3 .. dL/dc8
};

template <typename R>
LBM_HD void collide_cascaded_vjp(const R d[9], R Fx, R Fy, const Coef<R>& c, const R mu[9], CollideAdjoint<R>& out) {
    // ---------------- forward recompute (same statements as collide_cascaded)
    const Moments<R> m = moments(d, c.rho0);
    const R inv = recip(m.rho);  // as the forward kernel: IEEE in FP64, rcp.approx in FP32
    const R px = m.jx + R(0.5) * Fx, py = m.jy + R(0.5) * Fy;
    const R ux = px * inv, uy = py * inv;
    const R uxx = rmul(ux, ux), uyy = rmul(uy, uy), uxy = rmul(ux, uy);
    const R r3 = rmul(c.rho0, R(1.0 / 3.0));
    const R P = rmul(Fx, uy) + rmul(Fy, ux);
    const R sxx = R(2) * Fx * ux, syy = R(2) * Fy * uy, sxy = P;
    const R sxxy = Fy * uxx + R(2) * Fx * uxy, sxyy = Fx * uyy + R(2) * Fy * uxy;
    const R sxxyy = R(2) * uxy * P;
    const R kxx_t = r3 + m.kxx, kyy_t = r3 + m.kyy;
    const R G3 = R(2.0 / 3.0) * m.drho + m.rho * (uxx + uyy) - (m.kxx + m.kyy) - R(0.5) * (sxx + syy);
    const R G4 = m.rho * (uxx - uyy) - (m.kxx - m.kyy) - R(0.5) * (sxx - syy);
    const R G5 = m.rho * uxy - m.kxy - R(0.5) * sxy;
    const R g3 = rmul(c.c3, G3), g4 = rmul(c.c4, G4), g5 = rmul(c.c5, G5);
    const R A = R(3) * g3 + g4, B = R(3) * g3 - g4;
    const R G6 = R(2) * m.rho * uxx * uy + m.kxxy - R(2) * ux * m.kxy - uy * kxx_t - R(0.5) * sxxy;
    const R g6 = c.c6 * G6 - R(0.5) * uy * A - R(2) * ux * g5;
    const R G7 = R(2) * m.rho * ux * uyy + m.kxyy - R(2) * uy * m.kxy - ux * kyy_t - R(0.5) * sxyy;
    const R g7 = c.c7 * G7 - R(0.5) * ux * B - R(2) * uy * g5;
    const R G8 = R(1.0 / 9.0) * m.drho - m.kxxyy + R(3) * m.rho * uxx * uyy + R(2) * (ux * m.kxyy + uy * m.kxxy)
               - uxx * kyy_t - uyy * kxx_t - R(4) * uxy * m.kxy - R(0.5) * sxxyy;

    // ---------------- adjoints of g3..g8 through d~ = d + K g: (K^T mu)_b
    const R m5p6 = mu[5] + mu[6], m7p8 = mu[7] + mu[8];
    const R diag = m5p6 + m7p8, axis = mu[1] + mu[2] + mu[3] + mu[4];
    R a3 = R(-4) * mu[0] - axis + R(2) * diag;
    R a4 = (mu[1] + mu[3]) - (mu[2] + mu[4]);
    R a5 = (mu[5] + mu[7]) - (mu[6] + mu[8]);
    R a6 = R(2) * (mu[2] - mu[4]) - m5p6 + m7p8;
    R a7 = R(2) * (mu[1] - mu[3]) - (mu[5] + mu[8]) + (mu[6] + mu[7]);
    const R a8 = R(4) * mu[0] - R(2) * axis + diag;

    R ux_a = 0, uy_a = 0, uxx_a = 0, uyy_a = 0, uxy_a = 0, rho_a = 0, drho_a = 0;
    R kxx_a = 0, kyy_a = 0, kxy_a = 0, kxxy_a = 0, kxyy_a = 0, kxxyy_a = 0;
    R sxx_a = 0, syy_a = 0, sxy_a = 0, sxxy_a = 0, sxyy_a = 0, sxxyy_a = 0;
    R Fx_a = 0, Fy_a = 0, A_a = 0, B_a = 0;

    // g8 = c8 G8 - 2 g3 - (uyy A + uxx B)/2 - 4 uxy g5 - 2 (uy g6 + ux g7)
    out.c[5] = a8 * G8;
    const R G8a = c.c8 * a8;
    a3 += R(-2) * a8;
    A_a += R(-0.5) * uyy * a8;
    B_a += R(-0.5) * uxx * a8;
    uyy_a += R(-0.5) * A * a8;
    uxx_a += R(-0.5) * B * a8;
    uxy_a += R(-4) * g5 * a8;
    a5 += R(-4) * uxy * a8;
    uy_a += R(-2) * g6 * a8;
    a6 += R(-2) * uy * a8;
    ux_a += R(-2) * g7 * a8;
    a7 += R(-2) * ux * a8;
    // G8
    drho_a += R(1.0 / 9.0) * G8a;
    kxxyy_a -= G8a;
    rho_a += R(3) * uxx * uyy * G8a;
    uxx_a += (R(3) * m.rho * uyy - kyy_t) * G8a;
    uyy_a += (R(3) * m.rho * uxx - kxx_t) * G8a;
    ux_a += R(2) * m.kxyy * G8a;
    kxyy_a += R(2) * ux * G8a;
    uy_a += R(2) * m.kxxy * G8a;
    kxxy_a += R(2) * uy * G8a;
    kyy_a -= uxx * G8a;
    kxx_a -= uyy * G8a;
    uxy_a -= R(4) * m.kxy * G8a;
    kxy_a -= R(4) * uxy * G8a;
    sxxyy_a -= R(0.5) * G8a;

    // g7 = c7 G7 - ux B / 2 - 2 uy g5
    out.c[4] = a7 * G7;
    const R G7a = c.c7 * a7;
    ux_a -= R(0.5) * B * a7;
    B_a -= R(0.5) * ux * a7;
    uy_a -= R(2) * g5 * a7;
    a5 -= R(2) * uy * a7;
    rho_a += R(2) * ux * uyy * G7a;
    ux_a += (R(2) * m.rho * uyy - kyy_t) * G7a;
    uyy_a += R(2) * m.rho * ux * G7a;
    kxyy_a += G7a;
    uy_a -= R(2) * m.kxy * G7a;
    kxy_a -= R(2) * uy * G7a;
    kyy_a -= ux * G7a;
    sxyy_a -= R(0.5) * G7a;

    // g6 = c6 G6 - uy A / 2 - 2 ux g5
    out.c[3] = a6 * G6;
    const R G6a = c.c6 * a6;
    uy_a -= R(0.5) * A * a6;
    A_a -= R(0.5) * uy * a6;
    ux_a -= R(2) * g5 * a6;
    a5 -= R(2) * ux * a6;
    rho_a += R(2) * uxx * uy * G6a;
    uxx_a += R(2) * m.rho * uy * G6a;
    uy_a += (R(2) * m.rho * uxx - kxx_t) * G6a;
    kxxy_a += G6a;
    ux_a -= R(2) * m.kxy * G6a;
    kxy_a -= R(2) * ux * G6a;
    kxx_a -= uy * G6a;
    sxxy_a -= R(0.5) * G6a;

    // A = 3 g3 + g4, B = 3 g3 - g4
    a3 += R(3) * (A_a + B_a);
    a4 += A_a - B_a;

    // g5 = c5 G5
    out.c[2] = a5 * G5;
    const R G5a = c.c5 * a5;
    rho_a += uxy * G5a;
    uxy_a += m.rho * G5a;
    kxy_a -= G5a;
    sxy_a -= R(0.5) * G5a;
    // g4 = c4 G4
    out.c[1] = a4 * G4;
    const R G4a = c.c4 * a4;
    rho_a += (uxx - uyy) * G4a;
    uxx_a += m.rho * G4a;
    uyy_a -= m.rho * G4a;
    kxx_a -= G4a;
    kyy_a += G4a;
    sxx_a -= R(0.5) * G4a;
    syy_a += R(0.5) * G4a;
    // g3 = c3 G3
    out.c[0] = a3 * G3;
    const R G3a = c.c3 * a3;
    drho_a += R(2.0 / 3.0) * G3a;
    rho_a += (uxx + uyy) * G3a;
    uxx_a += m.rho * G3a;
    uyy_a += m.rho * G3a;
    kxx_a -= G3a;
    kyy_a -= G3a;
    sxx_a -= R(0.5) * G3a;
    syy_a -= R(0.5) * G3a;

    // raw source moments (Eq. 13)
    Fx_a += R(2) * ux * sxx_a;  ux_a += R(2) * Fx * sxx_a;
    Fy_a += R(2) * uy * syy_a;  uy_a += R(2) * Fy * syy_a;
    Fx_a += uy * sxy_a;  uy_a += Fx * sxy_a;  Fy_a += ux * sxy_a;  ux_a += Fy * sxy_a;
    Fy_a += uxx * sxxy_a;  uxx_a += Fy * sxxy_a;  Fx_a += R(2) * uxy * sxxy_a;  uxy_a += R(2) * Fx * sxxy_a;
    Fx_a += uyy * sxyy_a;  uyy_a += Fx * sxyy_a;  Fy_a += R(2) * uxy * sxyy_a;  uxy_a += R(2) * Fy * sxyy_a;
    uxy_a += R(2) * P * sxxyy_a;
    {
        const R Pa = R(2) * uxy * sxxyy_a;
        Fx_a += uy * Pa;  uy_a += Fx * Pa;  Fy_a += ux * Pa;  ux_a += Fy * Pa;
    }

    // source in velocity space, S = K D^-1 m^s (Eq. 14 with the m^s list before it)
    source_vjp(ux, uy, Fx, Fy, mu, ux_a, uy_a, Fx_a, Fy_a);

    // uxx = ux^2, uyy = uy^2, uxy = ux uy
    ux_a += R(2) * ux * uxx_a + uy * uxy_a;
    uy_a += R(2) * uy * uyy_a + ux * uxy_a;
    // ux = (jx + Fx/2)/rho, uy = (jy + Fy/2)/rho
    const R jx_a = ux_a * inv, jy_a = uy_a * inv;
    Fx_a += R(0.5) * jx_a;
    Fy_a += R(0.5) * jy_a;
    rho_a -= (ux * ux_a + uy * uy_a) * inv;
    drho_a += rho_a;
    // kxx_t, kyy_t carry their adjoints into kxx, kyy (already accumulated there)

    // raw moments of d -> d (each moment is a signed sum over directions)
    const R xx = kxx_a, yy = kyy_a, b = kxxyy_a;
    out.d[0] = mu[0] + drho_a;
    out.d[1] = mu[1] + drho_a + jx_a + xx;
    out.d[2] = mu[2] + drho_a + jy_a + yy;
    out.d[3] = mu[3] + drho_a - jx_a + xx;
    out.d[4] = mu[4] + drho_a - jy_a + yy;
    const R c0 = drho_a + xx + yy + b;
    out.d[5] = mu[5] + c0 + jx_a + jy_a + kxy_a + kxxy_a + kxyy_a;
    out.d[6] = mu[6] + c0 - jx_a + jy_a - kxy_a + kxxy_a - kxyy_a;
    out.d[7] = mu[7] + c0 - jx_a - jy_a + kxy_a - kxxy_a - kxyy_a;
    out.d[8] = mu[8] + c0 + jx_a - jy_a - kxy_a - kxxy_a + kxyy_a;
    out.Fx = Fx_a;
    out.Fy = Fy_a;
}

}  // namespace lbm
