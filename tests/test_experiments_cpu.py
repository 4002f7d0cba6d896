"""Host-side post-processing of the cavity experiments (no GPU): the stream
function, the primary and secondary vortex finders, the centre-line extraction
and the strain-rate probes, checked on synthetic fields whose answers are known
in closed form."""

import numpy as np
import pytest

from paper_1202_6351_gb300 import experiments as X


def _velocity_from_psi(psi_fn, n):
    """u = d psi / dy, v = -d psi / dx sampled at the nodes x_i = (i + 1/2)/n
    (spacing 1/n) of an n x n cavity; psi in lattice units (node spacing 1)."""
    c = (np.arange(n) + 0.5) / n
    X_, Y_ = np.meshgrid(c, c, indexing="xy")
    h = 1e-6
    u = (psi_fn(X_, Y_ + h) - psi_fn(X_, Y_ - h)) / (2 * h) / n
    v = -(psi_fn(X_ + h, Y_) - psi_fn(X_ - h, Y_)) / (2 * h) / n
    return np.stack([u, v])


def test_stream_function_integrates_u_from_the_bottom_wall_to_each_node():
    """The wall is half a spacing below node row 0: psi there is half of that
    row's u, and each further row adds the two half cells between nodes."""
    rng = np.random.default_rng(3)
    u = rng.standard_normal((2, 7, 5))
    psi = X.stream_function(u)
    assert psi.shape == (7, 5)
    np.testing.assert_allclose(psi[0], 0.5 * u[0][0])
    np.testing.assert_allclose(psi[1] - psi[0], 0.5 * (u[0][0] + u[0][1]))
    np.testing.assert_allclose(psi[-1], u[0].sum(axis=0) - 0.5 * u[0][-1])
    # a uniform flow u = U gives psi = U (y - y_wall) at the nodes
    uu = np.zeros((2, 7, 5))
    uu[0] = 0.3
    np.testing.assert_allclose(X.stream_function(uu)[:, 2], 0.3 * (np.arange(7) + 0.5))


@pytest.mark.parametrize("centre", [(0.6148, 0.7354), (0.5307, 0.5651), (0.47, 0.31)])
def test_primary_vortex_centre_of_a_gaussian_vortex(centre):
    """A clockwise Gaussian vortex (psi has a minimum at the centre): the finder
    returns the centre to a small fraction of a cell."""
    n = 129
    xc, yc = centre
    u = _velocity_from_psi(lambda x, y: -np.exp(-((x - xc) ** 2 + (y - yc) ** 2) / 0.05) * n, n)
    x, y = X.vortex_centre(u)
    assert abs(x - xc) < 0.2 / n and abs(y - yc) < 0.2 / n


def test_secondary_vortices_found_only_where_they_exist():
    """A clockwise primary vortex plus a small counter-clockwise one in the
    bottom-right corner: the finder locates the corner vortex and reports none
    in the other corner regions."""
    n = 257
    xc, yc = 0.86, 0.11

    def g(x, y):
        primary = -np.exp(-((x - 0.55) ** 2 + (y - 0.6) ** 2) / 0.08)
        corner = 0.02 * np.exp(-((x - xc) ** 2 + (y - yc) ** 2) / 0.002)
        return (primary + corner) * n

    def psi(x, y):  # psi = 0 along the bottom wall: no flow through it, as in the cavity
        return g(x, y) - g(x, 0.0 * y)

    from scipy.optimize import minimize

    u = _velocity_from_psi(psi, n)
    # the vortex centre is the maximum of the whole psi near the corner vortex,
    # which the primary vortex's slope moves away from (xc, yc)
    best = minimize(lambda p: -psi(p[0], p[1]), x0=[xc, yc], method="Nelder-Mead",
                    options={"xatol": 1e-9, "fatol": 1e-12})
    ex, ey = best.x
    got = X.secondary_vortex(u, "bottom_right")
    assert got is not None
    assert abs(got[0] - ex) < 0.2 / n and abs(got[1] - ey) < 0.2 / n
    assert X.secondary_vortex(u, "bottom_left") is None
    assert X.secondary_vortex(u, "top_left") is None


def test_centre_lines_pass_through_the_middle_nodes():
    n = 13
    rng = np.random.default_rng(5)
    u = rng.standard_normal((2, n, n))
    pos, uc, vc = X.centreline_profiles(u)
    np.testing.assert_allclose(pos, (np.arange(n) + 0.5) / n)
    np.testing.assert_array_equal(uc, u[0][:, 6])
    np.testing.assert_array_equal(vc, u[1][6, :])
    assert pos[6] == pytest.approx(0.5)


def test_strain_probes_use_central_differences_at_the_table_III_points():
    """A linear velocity field u = (a y, b y + c x): the central differences are
    exact, and the moment-based values are the strain array divided by rho."""
    n = 64
    a, b, c = 0.3, -0.2, 0.7
    j, i = np.mgrid[0:n, 0:n].astype(float)
    u = np.stack([a * j, b * j + c * i])
    rho = np.full((n, n), 2.0)
    strain = np.stack([np.zeros((n, n)), np.full((n, n), 2.0 * b), np.full((n, n), 2.0 * (a + c))])
    pts = X.strain_at_points(rho, u, strain)
    assert set(pts) == set("ABCDE")
    for name, (dvdy_m, dvdy_fd, shear_m, shear_fd) in pts.items():
        assert dvdy_fd == pytest.approx(b) and shear_fd == pytest.approx(a + c)
        assert dvdy_m == pytest.approx(b) and shear_m == pytest.approx(a + c)


def test_cavity_omega_follows_the_stated_reynolds_number():
    om = X.cavity_omega(257, 1000.0, 0.1)
    nu = (1.0 / om - 0.5) / 3.0
    assert 0.1 * 256 / nu == pytest.approx(1000.0)
