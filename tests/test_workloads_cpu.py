"""The seeded input generators, checked against properties they must have.

The generators hold no lattice Boltzmann arithmetic; what they promise is about
the continuum fields (incompressibility, the Taylor-Green pressure of
Sec. III-B, band limits) and the recipes of the workloads (sizes, mixes,
seeds).  Derivatives here are spectral (FFT), independent of the generators'
closed forms.
"""
import numpy as np
import pytest

from paper_1202_6351_gb300 import workloads as W


def _spectral_grad(f):
    """(d/dx, d/dy) of a periodic field f[y, x] with unit node spacing."""
    ny, nx = f.shape
    kx = 2 * np.pi * np.fft.fftfreq(nx)
    ky = 2 * np.pi * np.fft.fftfreq(ny)
    F = np.fft.fft2(f)
    return (np.fft.ifft2(1j * kx[None, :] * F).real, np.fft.ifft2(1j * ky[:, None] * F).real)


@pytest.mark.parametrize("n", [16, 64])
def test_taylor_green_start_is_divergence_free_and_in_pressure_balance(n):
    """Sec. III-B: the start field is incompressible and its pressure
    p = rho / 3 balances the advection of the steady inviscid vortex,
    grad p = -rho0 (u . grad) u."""
    u0, rho0 = 0.01, 1.0
    rho, u = W.taylor_green_init(n, u0, rho0)
    ux_x, ux_y = _spectral_grad(u[0])
    uy_x, uy_y = _spectral_grad(u[1])
    assert np.abs(ux_x + uy_y).max() < 1e-15 * n
    # central differences cancel exactly as well (the lattice's own derivative)
    cd = lambda f, ax: (np.roll(f, -1, ax) - np.roll(f, 1, ax)) / 2  # noqa: E731
    assert np.abs(cd(u[0], 1) + cd(u[1], 0)).max() < 1e-17
    px, py = _spectral_grad(rho / 3)
    adv_x = u[0] * ux_x + u[1] * ux_y
    adv_y = u[0] * uy_x + u[1] * uy_y
    tol = 1e-9 * rho0 * np.abs(adv_x).max()      # rho ~ 1 is stored to ~1e-16
    np.testing.assert_allclose(px, -rho0 * adv_x, rtol=0, atol=tol)
    np.testing.assert_allclose(py, -rho0 * adv_y, rtol=0, atol=tol)
    assert rho.mean() == pytest.approx(rho0, abs=1e-15)


def test_diffusive_scaling_keeps_u0_times_n():
    assert W.diffusive_u0(64) == pytest.approx(0.04)
    for n in (16, 128, 4096):
        assert W.diffusive_u0(n) * n == pytest.approx(0.04 * 64)


@pytest.mark.parametrize("seed", [20261202, 7])
def test_fourier_modes_field_is_solenoidal_band_limited_and_bounded(seed):
    """The adjoint workload's start field: divergence-free, only wave vectors
    with 1 <= max(|kx|, |ky|) <= 8 (in cycles per box), |u| <= 0.02 everywhere
    with the bound reached, and reproducible from its seed."""
    n = 128
    u = W.fourier_modes_field(seed, n)
    ux_x, _ = _spectral_grad(u[0])
    _, uy_y = _spectral_grad(u[1])
    assert np.abs(ux_x + uy_y).max() < 1e-14
    speed = np.sqrt((u ** 2).sum(axis=0))
    assert speed.max() <= 0.02 * (1 + 1e-12)
    assert speed.max() >= 0.02 * (1 - 1e-12)
    m = np.fft.fftfreq(n) * n
    power = np.abs(np.fft.fft2(u[0])) ** 2 + np.abs(np.fft.fft2(u[1])) ** 2
    band = np.maximum(np.abs(m)[None, :], np.abs(m)[:, None])
    assert power[(band < 1) | (band > 8)].sum() < 1e-20 * power.sum()
    assert (power > 1e-12 * power.max()).sum() >= 2          # not a single mode
    np.testing.assert_array_equal(W.fourier_modes_field(seed, n), u)


def test_batch_domains_recipe():
    """The batched ensemble: 96 domains, sides log-uniform in [64, 2048], Re in
    [100, 5000], cavity and Taylor-Green alternating, FP32 and FP16 in pairs,
    fixed by the seed."""
    d = W.batch_domains()
    assert len(d) == 96
    sides = np.array([x["side"] for x in d])
    assert sides.min() >= 64 and sides.max() <= 2048
    # log-uniform: the median side is near the geometric mean of the range
    assert 200 < np.median(sides) < 700
    assert all(100 <= x["re"] <= 5000 for x in d)
    assert [x["kind"] for x in d[:4]] == ["cavity", "taylor_green"] * 2
    assert [x["store"] for x in d[:4]] == ["f32", "f32", "f16", "f16"]
    assert W.batch_domains() == d
    assert W.batch_domains(seed=1) != d


def test_random_generators_are_seeded():
    a = W.random_fields(3, 7, 5)
    b = W.random_fields(3, 7, 5)
    assert a[0].shape == (5, 7) and a[1].shape == (2, 5, 7)
    np.testing.assert_array_equal(a[0], b[0])
    np.testing.assert_array_equal(a[1], b[1])
    assert W.random_force_field(4, 7, 5, 1e-3).shape == (2, 5, 7)
    np.testing.assert_array_equal(W.random_noise(5, (9, 3), 0.1), W.random_noise(5, (9, 3), 0.1))
    assert not np.array_equal(W.random_noise(5, (9, 3), 0.1), W.random_noise(6, (9, 3), 0.1))
