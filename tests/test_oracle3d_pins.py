"""Pins of the D3Q27 central-moment oracle (oracle/lbm3d_oracle.c) against what
the mathematics fixes, independently of the oracle's own code: the discrete
Maxwellian at rest and in product form, conservation, the relaxation of every
central moment computed by direct summation, exact streaming, cubic symmetry,
and closed-form flows (shear-wave decay at the shear viscosity with second-order
convergence, Galilean invariance of that decay, the 2-D Taylor-Green vortex
embedded in 3-D, the attenuation of sound by the shear and bulk viscosities).

The paper (Sec. V-VI) names 3-D lattices as future work; the oracle's header
states how the 2-D method of Sec. II is carried to D3Q27."""
import math

import numpy as np
import pytest

from oracle import d3q27 as D

RATES = (1.15, 1.62, 1.3, 0.9, 1.1, 1.25)  # omega_bulk, omega_shear, omega_3 .. omega_6


def _velocities():
    """D3Q27 velocities in the oracle's order, built here: a = (ex+1) + 3 (ey+1) + 9 (ez+1)."""
    return np.array([[a % 3 - 1, (a // 3) % 3 - 1, a // 9 - 1] for a in range(27)])


E = _velocities()


def _central(f, u):
    """kappa_ijk = sum_a (e_ax-u_x)^i (e_ay-u_y)^j (e_az-u_z)^k f_a, as an array [k][j][i]."""
    c = np.zeros((3, 3, 3))
    for i in range(3):
        for j in range(3):
            for k in range(3):
                c[k, j, i] = ((E[:, 0] - u[0]) ** i * (E[:, 1] - u[1]) ** j * (E[:, 2] - u[2]) ** k * f).sum()
    return c


def _random_node(rng, amp=0.05):
    w = np.array([np.prod([(2 / 3 if e == 0 else 1 / 6) for e in ea]) for ea in E])
    return w * (1 + amp * rng.standard_normal(27))


def test_velocity_set_and_weights():
    """The 27 velocities of {-1,0,1}^3 in tensor order and the textbook D3Q27
    weights 8/27, 2/27, 1/54, 1/216 by |e|^2 = 0, 1, 2, 3."""
    e, w = D.velocities()
    np.testing.assert_array_equal(e, E)
    expect = {0: 8 / 27, 1: 2 / 27, 2: 1 / 54, 3: 1 / 216}
    for a in range(27):
        assert w[a] == pytest.approx(expect[int((E[a] ** 2).sum())], rel=1e-15)


def test_equilibrium_is_the_product_maxwellian():
    """At rest the equilibrium is rho w; at any u it is the product of 1-D
    distributions with moments (1, u, 1/3 + u^2): rho prod_d phi(e_d; u_d),
    phi(0) = 2/3 - u^2, phi(+-1) = (1/3 + u^2 +- u)/2; its central moments are
    rho m_i m_j m_k with m = (1, 0, 1/3)."""
    _, w = D.velocities()
    np.testing.assert_allclose(D.equilibrium_node(1.3, (0, 0, 0)), 1.3 * w, rtol=1e-12)

    def phi(e, u):
        return 2 / 3 - u * u if e == 0 else 0.5 * (1 / 3 + u * u + e * u)

    rng = np.random.default_rng(3)
    for _ in range(20):
        rho, u = 1 + 0.1 * rng.standard_normal(), 0.1 * rng.standard_normal(3)
        feq = D.equilibrium_node(rho, u)
        prod = np.array([rho * phi(ea[0], u[0]) * phi(ea[1], u[1]) * phi(ea[2], u[2]) for ea in E])
        np.testing.assert_allclose(feq, prod, rtol=1e-12, atol=1e-15)
        m = np.array([1, 0, 1 / 3])
        np.testing.assert_allclose(_central(feq, u), rho * np.einsum("k,j,i->kji", m, m, m), atol=1e-14)


def test_collision_conserves_mass_and_gains_momentum_F():
    rng = np.random.default_rng(7)
    for _ in range(50):
        fb = _random_node(rng)
        F = 1e-3 * rng.standard_normal(3)
        out = D.collide_node(fb, F, RATES)
        assert out.sum() == pytest.approx(fb.sum(), rel=1e-14)
        np.testing.assert_allclose(E.T @ out - E.T @ fb, F, atol=1e-15)


def test_post_collision_central_moments_relax_to_their_targets():
    """Sec. II carried to 3-D: with u = (j + F/2)/rho, the central moments of
    f~_bar - S equal (1 - omega) kappa + omega kappa_eq group by group: the trace
    of the second-order tensor at omega_bulk (target rho), its deviators and
    off-diagonal moments at omega_shear (target 0), orders 3..6 at
    omega_3..omega_6 (targets rho m_i m_j m_k); density and first-order moments
    are kept (the latter equal -F/2 for f_bar).  S has central moments
    (0; F; 0 ...)."""
    rng = np.random.default_rng(11)
    m = np.array([1, 0, 1 / 3])
    for _ in range(40):
        fb = _random_node(rng, 0.08)
        F = 2e-3 * rng.standard_normal(3)
        om = 0.3 + 1.5 * rng.random(6)
        rho = fb.sum()
        u = (E.T @ fb + 0.5 * F) / rho
        S = D.source_node(u, F)
        cs = _central(S, u)
        sig = np.zeros((3, 3, 3))
        sig[0, 0, 1], sig[0, 1, 0], sig[1, 0, 0] = F
        np.testing.assert_allclose(cs, sig, atol=1e-15)
        pre = _central(fb, u)
        post = _central(D.collide_node(fb, F, om) - S, u)
        np.testing.assert_allclose(pre[0, 0, 1], -F[0] / 2, atol=1e-15)
        want = pre.copy()
        tr = pre[0, 0, 2] + pre[0, 2, 0] + pre[2, 0, 0]
        tr_t = tr + om[0] * (rho - tr)
        d1 = (1 - om[1]) * (pre[0, 0, 2] - pre[0, 2, 0])
        d2 = (1 - om[1]) * (pre[0, 0, 2] - pre[2, 0, 0])
        want[0, 0, 2] = (tr_t + d1 + d2) / 3
        want[0, 2, 0] = (tr_t - 2 * d1 + d2) / 3
        want[2, 0, 0] = (tr_t + d1 - 2 * d2) / 3
        for (k, j, i) in ((0, 1, 1), (1, 0, 1), (1, 1, 0)):
            want[k, j, i] = (1 - om[1]) * pre[k, j, i]
        for k in range(3):
            for j in range(3):
                for i in range(3):
                    n = i + j + k
                    if n >= 3:
                        want[k, j, i] = pre[k, j, i] + om[n - 1] * (rho * m[i] * m[j] * m[k] - pre[k, j, i])
        np.testing.assert_allclose(post, want, atol=2e-14)


def test_unit_rates_give_the_equilibrium_and_rest_is_a_fixed_point():
    rng = np.random.default_rng(5)
    fb = _random_node(rng)
    F = np.array([1e-3, -2e-3, 5e-4])
    out = D.collide_node(fb, F, (1.0,) * 6)
    rho = fb.sum()
    u = (E.T @ fb + 0.5 * F) / rho
    np.testing.assert_allclose(out, D.equilibrium_node(rho, u) + 0.5 * D.source_node(u, F), atol=1e-15)
    _, w = D.velocities()
    np.testing.assert_allclose(D.collide_node(1.1 * w, (0, 0, 0), RATES), 1.1 * w, atol=1e-16)


def test_streaming_is_a_periodic_shift_of_each_population():
    rng = np.random.default_rng(2)
    L = D.Lattice3(5, 4, 3, RATES)
    post = rng.standard_normal((27, 3, 4, 5))
    L.stream(post)
    for a in range(27):
        np.testing.assert_array_equal(L.f[a], np.roll(post[a], shift=(E[a, 2], E[a, 1], E[a, 0]), axis=(0, 1, 2)))


def test_start_state_returns_the_requested_fields():
    rng = np.random.default_rng(9)
    shape = (3, 4, 5)
    rho = 1 + 0.02 * rng.standard_normal(shape)
    u = 0.05 * rng.standard_normal((3,) + shape)
    L = D.Lattice3(5, 4, 3, RATES, force=(1e-4, -2e-4, 3e-4)).init(rho, u)
    r, v = L.macros()
    np.testing.assert_allclose(r, rho, rtol=1e-14)
    np.testing.assert_allclose(v, u, atol=1e-15)


def test_cubic_symmetry_of_whole_runs():
    """Exchanging two axes of the start state exchanges them in the result (the
    method treats x, y and z alike), for every pair of axes."""
    rng = np.random.default_rng(4)
    n = 4
    rho = 1 + 0.02 * rng.standard_normal((n, n, n))
    u = 0.04 * rng.standard_normal((3, n, n, n))
    base = D.Lattice3(n, n, n, RATES).init(rho, u).run(3).macros()
    # array axes are (z, y, x): velocity component d lives on array axis 2 - d
    for d1, d2 in ((0, 1), (0, 2), (1, 2)):
        perm = list(range(3))
        perm[2 - d1], perm[2 - d2] = perm[2 - d2], perm[2 - d1]
        rho_p = np.transpose(rho, perm)
        u_p = np.transpose(u, [0] + [p + 1 for p in perm])[[{d1: d2, d2: d1}.get(d, d) for d in range(3)]]
        r2, v2 = D.Lattice3(n, n, n, RATES).init(rho_p, u_p).run(3).macros()
        np.testing.assert_allclose(r2, np.transpose(base[0], perm), atol=1e-15)
        v_back = np.transpose(base[1], [0] + [p + 1 for p in perm])[[{d1: d2, d2: d1}.get(d, d) for d in range(3)]]
        np.testing.assert_allclose(v2, v_back, atol=1e-16)


def _shear_wave_error(n, om_shear, steps, advect=0.0):
    """Shear wave u_x = U sin(2 pi z / n) on a 1 x 1 x n lattice (a quasi-1-D
    run of the 3-D method), optionally advected along z; returns the
    fitted decay rate and the decay rate nu k^2 of the Navier-Stokes equations."""
    rates = (1.0, om_shear, 1.0, 1.0, 1.0, 1.0)
    U = 1e-4
    k = 2 * math.pi / n
    z = np.arange(n, dtype=float)
    u = np.zeros((3, n, 1, 1))
    u[0, :, 0, 0] = U * np.sin(k * z)
    u[2] += advect
    L = D.Lattice3(1, 1, n, rates).init(np.ones((n, 1, 1)), u)
    amps = []
    for s in range(steps + 1):
        _, v = L.macros()
        # amplitude of the mode in the frame moving with the flow
        amps.append(2 / n * np.abs((v[0, :, 0, 0] * np.exp(-1j * k * (z - advect * s))).sum()))
        L.run(1)
    t = np.arange(steps + 1)
    rate = -np.polyfit(t[steps // 4:], np.log(amps[steps // 4:]), 1)[0]
    return rate, D.nu_from_omega(om_shear) * k * k


def test_shear_wave_decays_at_the_shear_viscosity_with_second_order_accuracy():
    """A shear wave decays at nu k^2, nu = (1/omega_shear - 1/2)/3; the relative
    error of the rate falls as n^-2."""
    errs = []
    for n in (16, 32, 64):
        rate, exact = _shear_wave_error(n, 1.4, 3 * n)
        errs.append(abs(rate / exact - 1))
    slopes = [math.log2(errs[k] / errs[k + 1]) for k in range(2)]
    assert errs[-1] < 2e-3
    assert all(1.8 < s < 2.3 for s in slopes), (errs, slopes)


def test_shear_wave_decay_is_galilean_invariant():
    """Advected by a uniform flow along the wave vector, the central-moment
    collision keeps the decay rate (the property Sec. I-II build the method
    for): the rate at U = 0.1 matches the rate at rest to 1e-3."""
    r0, _ = _shear_wave_error(32, 1.4, 96)
    r1, _ = _shear_wave_error(32, 1.4, 96, advect=0.1)
    assert abs(r1 / r0 - 1) < 1e-3


def test_embedded_taylor_green_vortex_decays_at_second_order():
    """The 2-D Taylor-Green vortex (Sec. III-B) on an n x n x 1 lattice is an
    exact solution of the 3-D equations; after one decay time the velocity
    error falls as n^-2."""
    om = 1.6
    nu = D.nu_from_omega(om)
    errs = []
    for n in (16, 32, 64):
        u0 = 0.04 * 16 / n
        k = 2 * math.pi / n
        x = np.arange(n, dtype=float)
        Y, X = np.meshgrid(x, x, indexing="ij")
        u = np.zeros((3, 1, n, n))
        u[0, 0] = -u0 * np.cos(k * X) * np.sin(k * Y)
        u[1, 0] = u0 * np.sin(k * X) * np.cos(k * Y)
        rho = (1 - 0.75 * u0 * u0 * (np.cos(2 * k * X) + np.cos(2 * k * Y)))[None]
        T = int(round(1 / (2 * nu * k * k)))
        L = D.Lattice3(n, n, 1, (1.0, om, 1.0, 1.0, 1.0, 1.0)).init(rho, u).run(T)
        _, v = L.macros()
        ua = u * math.exp(-2 * nu * k * k * T)
        errs.append(float(np.sqrt(((v - ua) ** 2).sum() / (ua ** 2).sum())))
    slopes = [math.log2(errs[k] / errs[k + 1]) for k in range(2)]
    assert all(1.85 < s < 2.2 for s in slopes), (errs, slopes)


def test_sound_attenuation_follows_the_shear_and_bulk_viscosities():
    """A standing density wave along z oscillates as A e^{-Gamma t} cos(Omega t)
    with Gamma = k^2 (4 nu / 3 + zeta) / 2, nu = (1/omega_shear - 1/2)/3 and bulk
    viscosity zeta = (2/3)(1/omega_bulk - 1/2)/3 (the trace of the second-order
    moments relaxes at omega_bulk), Omega = sqrt(k^2/3 - Gamma^2)."""
    scipy_opt = pytest.importorskip("scipy.optimize")
    n, eps = 128, 1e-4
    ob, os_ = 1.3, 1.7
    k = 2 * math.pi / n
    z = np.arange(n, dtype=float)
    rho = (1 + eps * np.cos(k * z)).reshape(n, 1, 1)
    L = D.Lattice3(1, 1, n, (ob, os_, 1.0, 1.0, 1.0, 1.0)).init(rho, np.zeros((3, n, 1, 1)))
    amp = []
    for _ in range(2500):
        r, _ = L.macros()
        amp.append(2 / n * ((r[:, 0, 0] - 1) * np.cos(k * z)).sum())
        L.run(1)
    amp, t = np.array(amp), np.arange(len(amp))
    nu = (1 / os_ - 0.5) / 3
    zeta = (2 / 3) * (1 / ob - 0.5) / 3
    gamma = k * k * (4 * nu / 3 + zeta) / 2
    omega = math.sqrt(k * k / 3 - gamma ** 2)
    wave = lambda t, A, G, W, p: A * np.exp(-G * t) * np.cos(W * t + p)  # noqa: E731
    p, _ = scipy_opt.curve_fit(wave, t, amp, p0=[eps, gamma, omega, 0.0])
    assert abs(p[1] / gamma - 1) < 3e-3, (p[1], gamma)
    assert abs(p[2] / omega - 1) < 1e-3
