"""The D3Q27 central-moment lattices on the CUDA path against the D3Q27 oracle
(oracle/lbm3d_oracle.c): FP64 storage element by element per step, FP32 storage
after many steps, sampled nodes of a large lattice one by one, and mass and
momentum over a long run."""
import math

import numpy as np
import pytest

from oracle import d3q27 as D
from paper_1202_6351_gb300 import lbm, workloads

pytestmark = pytest.mark.gpu

RATES = (1.15, 1.62, 1.3, 0.9, 1.1, 1.25)


@pytest.fixture(scope="module", autouse=True)
def cuda():
    import torch

    assert torch.cuda.is_available(), "GPU tests need a CUDA device"
    torch.cuda.set_device(0)
    yield


def _noisy_start(L, O, rho, u, seed):
    """Both lattices at the same state off equilibrium (multiplicative noise on f)."""
    O.init(rho, u)
    f = O.f * (1.0 + workloads.random_noise(seed, O.f.shape, 0.02))
    O.set_f(f)
    L.set_f(f)


@pytest.mark.parametrize("shape", [(7, 5, 6), (33, 4, 3), (1, 1, 9), (16, 16, 2)])
@pytest.mark.parametrize("force", [(0.0, 0.0, 0.0), (2e-5, -1e-5, 3e-5)], ids=["unforced", "forced"])
def test_f64_steps_match_the_oracle(shape, force):
    nx, ny, nz = shape
    rho, u = workloads.random_fields_3d(3, nx, ny, nz, u_amp=0.03, rho_amp=0.01)
    O = D.Lattice3(nx, ny, nz, RATES, force=force)
    with lbm.Lattice3(nx, ny, nz, RATES, force=force, store=lbm.F64) as L:
        _noisy_start(L, O, rho, u, 5)
        for n in (1, 1, 1, 4):  # both AA parities, then a few more
            L.step(n)
            O.run(n)
            f = L.get_f()
            err = np.abs(f - O.f).max() / np.abs(O.f).max()
            assert err <= 1e-12, (shape, L.time, err)
        r, v = L.macros()
        r0, v0 = O.macros()
        np.testing.assert_allclose(r, r0, rtol=1e-12)
        np.testing.assert_allclose(v, v0, atol=1e-13)


def test_f64_start_state_matches_the_oracle():
    nx, ny, nz = 9, 6, 5
    force = (1e-4, 2e-4, -1e-4)
    rho, u = workloads.random_fields_3d(8, nx, ny, nz, u_amp=0.05, rho_amp=0.02)
    O = D.Lattice3(nx, ny, nz, RATES, force=force).init(rho, u)
    with lbm.Lattice3(nx, ny, nz, RATES, force=force, store=lbm.F64) as L:
        L.init(rho, u)
        np.testing.assert_allclose(L.get_f(), O.f, rtol=0, atol=1e-15)
        r, v = L.macros()
        np.testing.assert_allclose(r, rho, rtol=1e-14)
        np.testing.assert_allclose(v, u, atol=1e-15)


def test_f32_taylor_green_3d_after_many_steps():
    """FP32 storage (deviations, FP32 arithmetic) on the 3-D Taylor-Green
    vortex, 16^3, 150 steps: relative L2 velocity error against the FP64 oracle
    at most 1e-5."""
    n = 16
    rho, u = workloads.taylor_green_3d_init(n, 0.04)
    rates = (1.0, 1.6, 1.0, 1.0, 1.0, 1.0)
    O = D.Lattice3(n, n, n, rates).init(rho, u).run(150)
    _, u_ref = O.macros()
    with lbm.Lattice3(n, n, n, rates, store=lbm.F32) as L:
        L.init(rho, u).step(150)
        _, v = L.macros()
    err = float(np.sqrt(((v - u_ref) ** 2).sum() / (u_ref ** 2).sum()))
    print("FP32 D3Q27 Taylor-Green 16^3, 150 steps: relative L2 velocity error %.3e" % err)
    assert err <= 1e-5


# relative L2 velocity error bounds of the 16-bit storage kinds after 150 steps
# of the 16^3 Taylor-Green vortex (measured and stated; the paper has no
# reduced precision): FP16 keeps 4096 x the deviation, BF16 has an 8-bit
# significand
REDUCED_BOUNDS_3D = {lbm.F16DEV: 1e-3, lbm.BF16DEV: 1e-2}  # measured 2.3e-4 and 1.9e-3


@pytest.mark.parametrize("store", [lbm.F16DEV, lbm.BF16DEV], ids=["f16", "bf16"])
def test_16bit_taylor_green_3d_against_the_oracle(store):
    """16-bit deviation storage (FP32 arithmetic, round to nearest even) on the
    3-D Taylor-Green vortex, 16^3, 150 steps, against the FP64 oracle; the
    stored state reads back within one 16-bit rounding of the FP64 start."""
    n = 16
    rho, u = workloads.taylor_green_3d_init(n, 0.04)
    rates = (1.0, 1.6, 1.0, 1.0, 1.0, 1.0)
    O = D.Lattice3(n, n, n, rates).init(rho, u)
    f0 = O.f.copy()
    O.run(150)
    _, u_ref = O.macros()
    with lbm.Lattice3(n, n, n, rates, store=store) as L:
        L.init(rho, u)
        dev = f0 - L.get_f()  # both are f = d + w rho0; only the rounding of d differs
        rel = 2.0 ** -11 if store == lbm.F16DEV else 2.0 ** -8
        assert np.abs(dev).max() <= rel * np.abs(f0 - D.velocities()[1][:, None, None, None]).max() * 1.01
        L.step(150)
        r, v = L.macros()
    err = float(np.sqrt(((v - u_ref) ** 2).sum() / (u_ref ** 2).sum()))
    print("%s D3Q27 Taylor-Green 16^3, 150 steps: relative L2 velocity error %.3e" % (lbm.STORE_NAMES[store], err))
    assert err <= REDUCED_BOUNDS_3D[store]
    assert abs(r.mean() - 1.0) < 1e-3


def test_large_lattice_sampled_nodes_match_the_oracle():
    """128^3 FP32 (the launch shape of the 3-D bench lattice): after one step,
    64 sampled nodes agree with the oracle's collision of their pulled
    neighbours to FP32 rounding (relative 1e-6 of the populations)."""
    n = 128
    rho, u = workloads.taylor_green_3d_init(n, 0.05)
    rates = (1.0, 1.7, 1.0, 1.0, 1.0, 1.0)
    with lbm.Lattice3(n, n, n, rates, store=lbm.F32) as L:
        L.init(rho, u)
        f0 = L.get_f()
        L.step(1)
        f1 = L.get_f()
    e, _ = D.velocities()
    rng = np.random.default_rng(1)
    for _ in range(64):
        x, y, z = (int(v) for v in rng.integers(0, n, 3))
        want = np.empty(27)
        for q in range(27):  # pull: f_q(x, t+1) = collide(f(x - e_q, t))_q
            xs, ys, zs = (x - e[q, 0]) % n, (y - e[q, 1]) % n, (z - e[q, 2]) % n
            want[q] = D.collide_node(f0[:, zs, ys, xs], (0, 0, 0), rates)[q]
        np.testing.assert_allclose(f1[:, z, y, x], want, rtol=0, atol=1e-6 * np.abs(want).max())


def test_mass_and_momentum_over_a_long_run():
    """Periodic FP32 lattice with a uniform force: mass is kept and the total
    momentum grows by F per node and step (to FP32 accumulation error)."""
    n = 64
    F = (1e-6, -2e-6, 5e-7)
    rho, u = workloads.taylor_green_3d_init(n, 0.03)
    with lbm.Lattice3(n, n, n, (1.0, 1.5, 1.0, 1.0, 1.0, 1.0), force=F, store=lbm.F32) as L:
        L.init(rho, u)
        r0, v0 = L.macros()
        L.step(1000)
        r1, v1 = L.macros()
    m0, m1 = r0.sum(), r1.sum()
    assert abs(m1 / m0 - 1) < 1e-6
    p0 = (r0 * v0).reshape(3, -1).sum(1)
    p1 = (r1 * v1).reshape(3, -1).sum(1)
    np.testing.assert_allclose(p1 - p0, np.array(F) * n ** 3 * 1000, rtol=2e-3)


def test_rejects_bad_arguments():
    with pytest.raises(lbm.LBMError):
        lbm.Lattice3(0, 4, 4, RATES)
    with pytest.raises(lbm.LBMError):
        lbm.Lattice3(4, 4, 4, (1.0, 2.5, 1.0, 1.0, 1.0, 1.0))
    with pytest.raises(lbm.LBMError):
        lbm.Lattice3(4, 4, 4, RATES, store=7)  # no such storage kind
