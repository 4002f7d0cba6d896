"""The CUDA adjoint (lbm_adjoint_run, through the C ABI) against complex-step
derivatives of the FP64 oracle and central finite differences.

Loss: L = 1/2 sum_x |u(x, T) - u_target(x)|^2 after T steps of a periodic
cascaded lattice started at the transformed equilibrium with velocity u0.
Gradients: dL/du0, dL/dF (per-node body force field), dL/domega_3..8.
"""

import numpy as np
import pytest

import oracle as O
from paper_1202_6351_gb300 import lbm, workloads

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def cuda():
    import torch

    assert torch.cuda.is_available(), "GPU tests need a CUDA device"
    torch.cuda.set_device(0)
    yield


def _t(a):
    import torch

    return torch.from_numpy(np.ascontiguousarray(a, dtype=np.float64)).cuda()


def oracle_loss(nx, ny, omegas, u0, F, target, steps):
    cplx = any(np.iscomplexobj(v) for v in (u0, F, omegas))
    L = O.Lattice(nx, ny, omegas, force_field=F, complex=cplx)
    L.init(np.ones((ny, nx)), u0).run(steps)
    _, u = L.macros()
    return 0.5 * ((u - target) ** 2).sum()


def gpu_adjoint(nx, ny, omegas, u0, F, target, steps, every, store=lbm.F64):
    with lbm.Lattice(nx, ny, omegas, store=store) as L:
        L.set_force_field(F)
        loss, gu, gf, gom = L.adjoint_run(steps, every, _t(u0), _t(target))
        return loss, gu.cpu().numpy(), gf.cpu().numpy(), gom


def test_full_gradient_matches_oracle_complex_step_small_lattice():
    nx, ny, steps, every = 7, 6, 5, 2
    rng = np.random.default_rng(31)
    u0 = 0.05 * rng.standard_normal((2, ny, nx))
    F = 1e-3 * rng.standard_normal((2, ny, nx))
    target = 0.03 * rng.standard_normal((2, ny, nx))
    om = rng.uniform(0.6, 1.8, 6)
    loss, gu, gf, gom = gpu_adjoint(nx, ny, om, u0, F, target, steps, every)
    assert loss == pytest.approx(oracle_loss(nx, ny, om, u0, F, target, steps), rel=1e-13)
    h = 1e-30
    cs_u = np.zeros_like(u0)
    cs_f = np.zeros_like(F)
    for idx in np.ndindex(*u0.shape):
        du = u0.astype(complex)
        du[idx] += 1j * h
        cs_u[idx] = oracle_loss(nx, ny, om, du, F, target, steps).imag / h
        dF = F.astype(complex)
        dF[idx] += 1j * h
        cs_f[idx] = oracle_loss(nx, ny, om, u0, dF, target, steps).imag / h
    cs_om = np.zeros(6)
    for k in range(6):
        o = om.astype(complex)
        o[k] += 1j * h
        cs_om[k] = oracle_loss(nx, ny, o, u0, F, target, steps).imag / h
    assert np.abs(gu - cs_u).max() <= 1e-10 * np.abs(cs_u).max()
    assert np.abs(gf - cs_f).max() <= 1e-10 * np.abs(cs_f).max()
    np.testing.assert_allclose(gom, cs_om, rtol=1e-10, atol=1e-10 * np.abs(cs_om).max())


def test_directional_derivatives_match_oracle_complex_step_64():
    n, steps, every = 64, 200, 50
    om = (1.0, 1.6, 1.6, 1.0, 1.0, 1.0)
    u0 = workloads.fourier_modes_field(5, n, modes=16, amp=0.02, kmax=8)
    F = np.zeros((2, n, n))
    _, ua, _ = O.taylor_green(n, 0.04, 1.0 / 24.0, steps)
    loss, gu, gf, gom = gpu_adjoint(n, n, om, u0, F, ua, steps, every)
    rng = np.random.default_rng(64)
    h = 1e-30
    for k in range(3):
        v = rng.standard_normal(u0.shape)
        cs = oracle_loss(n, n, om, u0 + 1j * h * v, F, ua, steps).imag / h
        assert (gu * v).sum() == pytest.approx(cs, rel=1e-9)
        w = 1e-4 * rng.standard_normal(F.shape)
        cs = oracle_loss(n, n, om, u0, F + 1j * h * w, ua, steps).imag / h
        assert (gf * w).sum() == pytest.approx(cs, rel=1e-9)
    o = np.array(om, dtype=complex)
    o[1] += 1j * h
    o[2] += 1j * h
    cs = oracle_loss(n, n, o, u0, F, ua, steps).imag / h
    assert gom[1] + gom[2] == pytest.approx(cs, rel=1e-9)


# ---------------------------------------------------------------- the 512 x 512, 2000-step configuration

N, STEPS, EVERY, OMEGA = 512, 2000, 100, 1.6


def _config():
    u0 = workloads.fourier_modes_field(20261202, N, modes=16, amp=0.02, kmax=8)
    F = np.zeros((2, N, N))
    nu = (1.0 / OMEGA - 0.5) / 3.0
    _, target, _ = O.taylor_green(N, 0.04 * 64 / N, nu, STEPS)
    return u0, F, target


def _fd_loss(u0, F, omega_shear, target):
    """Forward-only FP64 loss through the C ABI (the parity-pinned FP64 path)."""
    import torch

    with lbm.Lattice(N, N, (1.0, omega_shear, omega_shear, 1.0, 1.0, 1.0), store=lbm.F64) as L:
        L.set_force_field(_t(F))
        L.init_device(None, _t(u0)).step(STEPS)
        _, u = L.macros_device()
        torch.cuda.synchronize()
        return 0.5 * float(((u - _t(target)) ** 2).sum())


@pytest.fixture(scope="module")
def adjoint_512():
    u0, F, target = _config()
    om = (1.0, OMEGA, OMEGA, 1.0, 1.0, 1.0)
    out = {}
    for store in (lbm.F32, lbm.F64):
        out[store] = gpu_adjoint(N, N, om, u0, F, target, STEPS, EVERY, store)
    return u0, F, target, out


def test_adjoint_512_matches_central_differences(adjoint_512):
    u0, F, target, out = adjoint_512
    rng = np.random.default_rng(512)
    checks = []
    for k in range(4):  # random directions in u0
        v = 0.02 * rng.standard_normal(u0.shape)
        eps = 1e-3
        fd = (_fd_loss(u0 + eps * v, F, OMEGA, target) - _fd_loss(u0 - eps * v, F, OMEGA, target)) / (2 * eps)
        checks.append(("u0", lambda g, v=v: (g[1] * v).sum(), fd))
    for k in range(3):  # random directions in F
        w = 1e-5 * rng.standard_normal(F.shape)
        eps = 1e-2
        fd = (_fd_loss(u0, F + eps * w, OMEGA, target) - _fd_loss(u0, F - eps * w, OMEGA, target)) / (2 * eps)
        checks.append(("F", lambda g, w=w: (g[2] * w).sum(), fd))
    eps = 1e-5  # the tied shear rate
    fd = (_fd_loss(u0, F, OMEGA + eps, target) - _fd_loss(u0, F, OMEGA - eps, target)) / (2 * eps)
    checks.append(("omega", lambda g: g[3][1] + g[3][2], fd))
    for store, tol in ((lbm.F64, 1e-6), (lbm.F32, 1e-4)):
        for name, proj, fd in checks:
            got = proj(out[store])
            assert abs(got - fd) <= tol * abs(fd), (lbm.STORE_NAMES[store], name, got, fd)


def test_adjoint_512_individual_entries(adjoint_512):
    u0, F, target, out = adjoint_512
    rng = np.random.default_rng(16)
    g64 = out[lbm.F64]
    g32 = out[lbm.F32]
    for k in range(16):
        c, y, x = int(rng.integers(0, 2)), int(rng.integers(0, N)), int(rng.integers(0, N))
        if k < 8:
            e = np.zeros_like(u0)
            e[c, y, x] = 1.0
            eps = 1e-4
            fd = (_fd_loss(u0 + eps * e, F, OMEGA, target) - _fd_loss(u0 - eps * e, F, OMEGA, target)) / (2 * eps)
            got64, got32 = g64[1][c, y, x], g32[1][c, y, x]
        else:
            e = np.zeros_like(F)
            e[c, y, x] = 1.0
            eps = 1e-6
            fd = (_fd_loss(u0, F + eps * e, OMEGA, target) - _fd_loss(u0, F - eps * e, OMEGA, target)) / (2 * eps)
            got64, got32 = g64[2][c, y, x], g32[2][c, y, x]
        scale = max(abs(fd), 1e-3 * np.abs(g64[1 if k < 8 else 2]).max())
        assert abs(got64 - fd) <= 1e-5 * scale, (k, got64, fd)
        assert abs(got32 - fd) <= 1e-3 * scale, (k, got32, fd)


def test_adjoint_512_f32_agrees_with_f64(adjoint_512):
    _, _, _, out = adjoint_512
    l32, gu32, gf32, go32 = out[lbm.F32]
    l64, gu64, gf64, go64 = out[lbm.F64]
    assert l32 == pytest.approx(l64, rel=1e-5)
    assert np.sqrt(((gu32 - gu64) ** 2).sum() / (gu64 ** 2).sum()) <= 1e-4
    assert np.sqrt(((gf32 - gf64) ** 2).sum() / (gf64 ** 2).sum()) <= 1e-4


@pytest.mark.parametrize("every", [1, 7, 40, 100])
def test_f32_force_gradient_folding_for_any_checkpoint_interval(every):
    """FP32 storage sums the force gradient in FP32 within a checkpoint segment
    and folds it into FP64 once per segment: one step per segment, a ragged
    last segment (40 = 5 x 7 + 5) and a single segment longer than the run must
    all give the FP64 adjoint's gradients to FP32 accuracy."""
    n, steps = 32, 40
    om = (1.0, 1.6, 1.6, 1.0, 1.0, 1.0)
    rng = np.random.default_rng(11)
    u0 = 0.02 * rng.standard_normal((2, n, n))
    F = 1e-5 * rng.standard_normal((2, n, n))
    target = 0.02 * rng.standard_normal((2, n, n))
    ref = gpu_adjoint(n, n, om, u0, F, target, steps, 7, store=lbm.F64)
    got = gpu_adjoint(n, n, om, u0, F, target, steps, every, store=lbm.F32)
    assert got[0] == pytest.approx(ref[0], rel=1e-5)
    for a, b in zip(got[1:3], ref[1:3]):
        assert np.abs(a - b).max() <= 1e-4 * np.abs(b).max()
    np.testing.assert_allclose(got[3], ref[3], rtol=1e-3, atol=1e-6 * np.abs(ref[3]).max())


def test_autograd_function_returns_the_adjoint_gradients():
    import torch

    from paper_1202_6351_gb300.adjoint import final_velocity_loss

    n, steps = 48, 60
    u0 = _t(workloads.fourier_modes_field(9, n, modes=8, amp=0.02, kmax=4)).requires_grad_(True)
    F = torch.zeros((2, n, n), dtype=torch.float64, device="cuda", requires_grad=True)
    w = torch.tensor(1.6, dtype=torch.float64, device="cuda", requires_grad=True)
    target = torch.zeros((2, n, n), dtype=torch.float64, device="cuda")
    loss = final_velocity_loss(u0, F, w, target, steps, every=16, store=lbm.F64)
    loss.backward()
    l_ref, gu, gf, gom = gpu_adjoint(n, n, (1.0, 1.6, 1.6, 1.0, 1.0, 1.0), u0.detach().cpu().numpy(),
                                     np.zeros((2, n, n)), np.zeros((2, n, n)), steps, 16)
    assert float(loss.detach()) == pytest.approx(l_ref, rel=1e-14)
    np.testing.assert_allclose(u0.grad.cpu().numpy(), gu, rtol=1e-12, atol=1e-15)
    np.testing.assert_allclose(F.grad.cpu().numpy(), gf, rtol=1e-12, atol=1e-15)
    assert float(w.grad) == pytest.approx(gom[1] + gom[2], rel=1e-12)
    # one step of gradient descent on the shear rate lowers the loss
    with torch.no_grad():
        w2 = w - 1e-3 * torch.sign(w.grad)
    assert float(final_velocity_loss(u0.detach(), F.detach(), w2, target, steps, 16, store=lbm.F64)) < float(loss.detach())
