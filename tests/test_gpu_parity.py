"""Parity of the CUDA path (through the C ABI) with the FP64 oracle.

Bars: FP64 storage/arithmetic <= 1e-12 relative (max-norm of f) per step and
<= 1e-10 after 1000 steps; FP32 <= 1e-5 relative L2 velocity error after 1000
steps; reduced-precision storage within the bounds stated in the test.
Inputs are seeded; expected values come from the oracle only.
"""

import numpy as np
import pytest

import oracle as O
from paper_1202_6351_gb300 import lbm, workloads

pytestmark = pytest.mark.gpu

EDGES = {
    "periodic": ((lbm.PERIODIC,) * 4, (0, 0, 0, 0)),
    "channel": ((lbm.PERIODIC, lbm.PERIODIC, lbm.BOUNCEBACK, lbm.BOUNCEBACK), (0, 0, 0, 0)),
    "ychannel": ((lbm.BOUNCEBACK, lbm.BOUNCEBACK, lbm.PERIODIC, lbm.PERIODIC), (0, 0, 0, 0)),
    "cavity": ((lbm.BOUNCEBACK, lbm.BOUNCEBACK, lbm.BOUNCEBACK, lbm.MOVING_WALL), (0, 0, 0, 0.1)),
    "allmoving": ((lbm.MOVING_WALL,) * 4, (0.03, -0.02, 0.05, 0.08)),
    "couette": ((lbm.PERIODIC, lbm.PERIODIC, lbm.MOVING_WALL, lbm.MOVING_WALL), (0, 0, -0.04, 0.06)),
}
MODELS = [lbm.CASCADED, lbm.BGK, lbm.RAWMRT]
OMEGAS = (1.3, 1.7, 1.6, 0.9, 1.1, 1.2)


@pytest.fixture(scope="module", autouse=True)
def cuda():
    import torch

    assert torch.cuda.is_available(), "GPU tests need a CUDA device"
    torch.cuda.set_device(0)
    lbm.load_library()
    yield


def pair(nx, ny, model=lbm.CASCADED, store=lbm.F64, edges="periodic", omegas=OMEGAS, force=(0.0, 0.0),
         force_field=None):
    e, wu = EDGES[edges]
    gpu = lbm.Lattice(nx, ny, omegas, force=force, edges=e, wall_u=wu, model=model, store=store)
    if force_field is not None:
        gpu.set_force_field(force_field)
    ref = O.Lattice(nx, ny, omegas, force=force, edges=e, wall_u=wu, model=model, force_field=force_field)
    return gpu, ref


def random_state(ref, seed, noise=0.02):
    rho, u = workloads.random_fields(seed, ref.nx, ref.ny)
    ref.init(rho, u)
    ref.f *= 1.0 + workloads.random_noise(seed + 1, ref.f.shape, noise)
    return ref.f.copy()


def rel_max(a, b):
    return float(np.abs(a - b).max() / np.abs(b).max())


def rel_l2(a, b):
    return float(np.sqrt(((a - b) ** 2).sum() / (b ** 2).sum()))


# ---------------------------------------------------------------- FP64 per-step parity

@pytest.mark.parametrize("model", MODELS, ids=["cascaded", "bgk", "rawmrt"])
@pytest.mark.parametrize("edges", list(EDGES))
@pytest.mark.parametrize("forced", [False, True], ids=["unforced", "forced"])
def test_f64_steps_match_oracle_from_random_state(model, edges, forced):
    """37 x 23 (ragged against the 128 x 2 block and the 32-wide pitch), random
    non-equilibrium state; 1, 2 and 3 steps cover both AA parities."""
    force = (2e-4, -1e-4) if forced else (0.0, 0.0)
    gpu, ref = pair(37, 23, model, lbm.F64, edges, force=force)
    f0 = random_state(ref, 100 + model)
    gpu.set_f(f0)
    for k in range(3):
        gpu.step(1)
        ref.run(1)
        assert rel_max(gpu.get_f(), ref.f) <= 1e-12, f"step {k + 1}"
    rho_g, u_g = gpu.macros()
    rho_r, u_r = ref.macros()
    assert rel_max(rho_g, rho_r) <= 1e-13
    assert rel_max(u_g, u_r) <= 1e-11
    gpu.close()


def test_f64_force_field_matches_oracle():
    ff = workloads.random_force_field(7, 40, 30, 1e-4)
    for model in MODELS:
        gpu, ref = pair(40, 30, model, lbm.F64, "channel", force=(1e-5, 0.0), force_field=ff)
        f0 = random_state(ref, 11)
        gpu.set_f(f0)
        gpu.step(5)
        ref.run(5)
        assert rel_max(gpu.get_f(), ref.f) <= 1e-12
        np.testing.assert_allclose(gpu.strain(), ref.strain(), rtol=0, atol=1e-13)
        gpu.close()


@pytest.mark.parametrize("shape", [(1, 1), (1, 7), (7, 1), (2, 2), (33, 1), (1, 33), (3, 5)])
@pytest.mark.parametrize("edges", ["periodic", "cavity", "allmoving", "channel"])
def test_f64_degenerate_sizes(shape, edges):
    nx, ny = shape
    gpu, ref = pair(nx, ny, lbm.CASCADED, lbm.F64, edges, force=(1e-4, 2e-4))
    f0 = random_state(ref, 5)
    gpu.set_f(f0)
    gpu.step(4)
    ref.run(4)
    assert rel_max(gpu.get_f(), ref.f) <= 1e-12
    gpu.close()


def test_f64_taylor_green_1000_steps():
    n = 64
    om = 1.6
    oms = (1.0, om, om, 1.0, 1.0, 1.0)
    rho, u = workloads.taylor_green_init(n, workloads.diffusive_u0(n))
    gpu = lbm.Lattice(n, n, oms, store=lbm.F64).init(rho, u)
    ref = O.Lattice(n, n, oms).init(rho, u)
    assert rel_max(gpu.get_f(), ref.f) <= 1e-15
    gpu.step(1000)
    ref.run(1000)
    assert rel_max(gpu.get_f(), ref.f) <= 1e-10
    gpu.close()


def test_f64_poiseuille_config_matches_oracle_and_parabola():
    om = 1 / 0.8
    nu = O.nu_from_omega(om)
    fx = 8 * nu * 0.01 / 32 ** 2
    oms = (1.0, om, om, 1.0, 1.0, 1.0)
    gpu, ref = pair(4, 32, lbm.CASCADED, lbm.F64, "channel", omegas=oms, force=(fx, 0.0))
    gpu.init()
    ref.init()
    gpu.step(20000)
    ref.run(20000)
    assert rel_max(gpu.get_f(), ref.f) <= 1e-12
    _, u = gpu.macros()
    ua = O.poiseuille_profile(32, fx, nu)
    assert np.abs(u[0][:, 0] - ua).max() / ua.max() < 0.0022
    gpu.close()


@pytest.mark.parametrize("model", MODELS, ids=["cascaded", "bgk", "rawmrt"])
def test_cavity_parity_f64_and_f32(model):
    n, U, re = 65, 0.1, 400.0
    nu = U * (n - 1) / re
    om = O.omega_from_nu(nu)
    oms = (1.0, om, om, 1.0, 1.0, 1.0)
    ref = O.Lattice(n, n, oms, edges=EDGES["cavity"][0], wall_u=EDGES["cavity"][1], model=model).init()
    ref.run(2000)
    _, u_ref = ref.macros()
    for store, tol in ((lbm.F64, 1e-10), (lbm.F32, 1e-5)):
        gpu = lbm.Lattice(n, n, oms, edges=EDGES["cavity"][0], wall_u=EDGES["cavity"][1], model=model,
                          store=store).init()
        gpu.step(2000)
        _, u = gpu.macros()
        if store == lbm.F64:
            assert rel_max(gpu.get_f(), ref.f) <= tol
        else:
            assert rel_l2(u, u_ref) <= tol
        gpu.close()


# ---------------------------------------------------------------- FP32 and reduced precision

def test_f32_taylor_green_1000_steps_velocity_error():
    n = 128
    om = 1.6
    oms = (1.0, om, om, 1.0, 1.0, 1.0)
    rho, u = workloads.taylor_green_init(n, workloads.diffusive_u0(n))
    ref = O.Lattice(n, n, oms).init(rho, u).run(1000)
    _, u_ref = ref.macros()
    gpu = lbm.Lattice(n, n, oms, store=lbm.F32).init(rho, u).step(1000)
    _, u_g = gpu.macros()
    assert rel_l2(u_g, u_ref) <= 1e-5
    gpu.close()


# Stated bounds for deviation storage (relative L2 velocity error against the
# FP64 oracle, Taylor-Green, 1000 steps, N = 128 under diffusive scaling).
REDUCED_BOUNDS = {lbm.BF16DEV: 8e-2, lbm.F16DEV: 2e-3}


@pytest.mark.parametrize("store", [lbm.BF16DEV, lbm.F16DEV], ids=["bf16", "f16"])
def test_reduced_precision_taylor_green_error_is_bounded(store):
    n = 128
    om = 1.6
    oms = (1.0, om, om, 1.0, 1.0, 1.0)
    rho, u = workloads.taylor_green_init(n, workloads.diffusive_u0(n))
    ref = O.Lattice(n, n, oms).init(rho, u).run(1000)
    _, u_ref = ref.macros()
    gpu = lbm.Lattice(n, n, oms, store=store).init(rho, u).step(1000)
    _, u_g = gpu.macros()
    err = rel_l2(u_g, u_ref)
    print(f"store {lbm.STORE_NAMES[store]}: relative L2 velocity error {err:.3e}")
    assert err <= REDUCED_BOUNDS[store]
    gpu.close()


# ---------------------------------------------------------------- diagnostics

def test_macros_strain_stats_at_both_parities():
    gpu, ref = pair(50, 41, lbm.CASCADED, lbm.F64, "couette", force=(3e-5, 1e-5))
    gpu.set_f(random_state(ref, 21))
    for k in range(2):
        gpu.step(1)
        ref.run(1)
        rho_g, u_g = gpu.macros()
        rho_r, u_r = ref.macros()
        np.testing.assert_allclose(rho_g, rho_r, rtol=1e-13, atol=0)
        np.testing.assert_allclose(u_g, u_r, rtol=0, atol=1e-13)
        np.testing.assert_allclose(gpu.strain(), ref.strain(), rtol=0, atol=1e-13)
        st = gpu.stats()
        mom_x = (rho_r * u_r[0]).sum()
        mom_y = (rho_r * u_r[1]).sum()
        np.testing.assert_allclose(st, [rho_r.sum(), mom_x, mom_y], rtol=1e-12, atol=1e-12)
    gpu.close()


def test_device_pointer_entry_points_agree_with_host_ones():
    import torch

    n = 40
    rho, u = workloads.random_fields(3, n, n, u_amp=0.03)
    a = lbm.Lattice(n, n, OMEGAS, store=lbm.F32, edges=EDGES["cavity"][0], wall_u=EDGES["cavity"][1])
    b = lbm.Lattice(n, n, OMEGAS, store=lbm.F32, edges=EDGES["cavity"][0], wall_u=EDGES["cavity"][1],
                    stream=torch.cuda.current_stream().cuda_stream)
    a.init(rho, u).step(7)
    b.init_device(torch.from_numpy(rho).cuda(), torch.from_numpy(u).cuda()).step(7)
    r_b, u_b = b.macros_device()
    torch.cuda.synchronize()
    r_a, u_a = a.macros()
    np.testing.assert_array_equal(r_b.cpu().numpy(), r_a)
    np.testing.assert_array_equal(u_b.cpu().numpy(), u_a)
    f = b.get_f_device()
    c = lbm.Lattice(n, n, OMEGAS, store=lbm.F32, edges=EDGES["cavity"][0], wall_u=EDGES["cavity"][1])
    c.set_f_device(f)
    torch.cuda.synchronize()
    np.testing.assert_array_equal(c.get_f(), a.get_f())
    for x in (a, b, c):
        x.close()


def test_divergence_check_stops_an_unstable_run_cleanly():
    """SRT at a cell Reynolds number far above its stability limit (Sec. V,
    Table IV) blows up; the check reports it and the context stays usable."""
    n = 64
    gpu = lbm.Lattice(n, n, (1.0, 1.995, 1.995, 1.0, 1.0, 1.0), edges=EDGES["cavity"][0],
                      wall_u=(0, 0, 0, 0.4), model=lbm.BGK, store=lbm.F32).init()
    gpu.set_check(50, 1e-3)
    with pytest.raises(lbm.LBMError) as ei:
        gpu.step(200000)
    assert ei.value.code == lbm.LBM_EDIVERGED
    gpu.close()
    ok = lbm.Lattice(8, 8, OMEGAS, store=lbm.F64).init().step(3)
    assert np.isfinite(ok.get_f()).all()
    ok.close()


# ---------------------------------------------------------------- full size (the bench workload)

def _patch_reference(fields, om, ix, iy, steps):
    """Post-step populations of node (ix, iy) of the n x n Taylor-Green lattice
    with initial (rho, u) = fields, from the oracle on the (2 steps + 1)^2 patch
    around it (periodic wrap)."""
    rho, u = fields
    n = rho.shape[0]
    r = steps
    xs = [(ix + k) % n for k in range(-r, r + 1)]
    ys = [(iy + k) % n for k in range(-r, r + 1)]
    prho = rho[np.ix_(ys, xs)]
    pu = u[:, ys][:, :, xs]
    m = 2 * r + 1
    L = O.Lattice(m, m, (1.0, om, om, 1.0, 1.0, 1.0)).init(prho, pu)
    L.run(steps)
    return L.f[:, r, r]


# absolute tolerance on f after one or two steps from the analytic start: FP32
# rounding of the arithmetic, FP16 / BF16 rounding of the stored deviations
FULL_SIZE_TOL = {lbm.F32: 2e-9, lbm.F16DEV: 5e-7, lbm.BF16DEV: 5e-6}


@pytest.mark.parametrize("store", [lbm.F32, lbm.F16DEV, lbm.BF16DEV], ids=["f32", "f16", "bf16"])
def test_full_size_taylor_green_4096_sampled_nodes(store):
    """The bench workload (4096^2, one launch per step) against the oracle on
    sampled nodes, plus global mass conservation after 100 steps."""
    import torch

    n, om = 4096, 1.6
    u0 = workloads.diffusive_u0(n)
    rho, u = workloads.taylor_green_init(n, u0)
    gpu = lbm.Lattice(n, n, (1.0, om, om, 1.0, 1.0, 1.0), store=store)
    gpu.init(rho, u)
    m0 = gpu.stats()[0]
    rng = np.random.default_rng(4096)
    pts = [(0, 0), (n - 1, n - 1), (0, n - 1), (n - 1, 0)] + [tuple(v) for v in rng.integers(0, n, (60, 2))]
    for steps in (1, 2):
        gpu.step(1)
        f = gpu.get_f()
        for ix, iy in pts:
            ref = _patch_reference((rho, u), om, ix, iy, steps)
            dev = f[:, iy, ix] - ref
            assert np.abs(dev).max() <= FULL_SIZE_TOL[store], (ix, iy, steps, np.abs(dev).max())
    gpu.step(98)
    m1 = gpu.stats()[0]
    assert abs(m1 - m0) / m0 <= (1e-9 if store == lbm.F32 else 1e-6)
    gpu.close()
    torch.cuda.synchronize()


def test_full_size_taylor_green_4096_two_steps_per_launch():
    """The bench's tuned FP32 configuration (variant 3: two steps per launch,
    node pairs in packed FP32x2, a graph replay of 64 steps among the 100) on
    the bench workload: bit for bit the states of one step per launch after 2
    and 102 steps, and sampled nodes (tile corners among them) after the first
    two-step launch against the oracle."""
    import torch

    n, om = 4096, 1.6
    rho, u = workloads.taylor_green_init(n, workloads.diffusive_u0(n))
    out = {}
    for variant in (0, 3):
        g = lbm.Lattice(n, n, (1.0, om, om, 1.0, 1.0, 1.0), store=lbm.F32)
        g.set_variant(variant).init(rho, u)
        assert g.info()["variant"] == variant
        g.step(2)
        f2 = g.get_f()
        g.step(100)
        out[variant] = (f2, g.get_f())
        g.close()
    np.testing.assert_array_equal(out[3][0], out[0][0])
    np.testing.assert_array_equal(out[3][1], out[0][1])
    f = out[3][0]
    rng = np.random.default_rng(4097)
    pts = [(0, 0), (n - 1, n - 1), (63, 15), (64, 16)] + [tuple(v) for v in rng.integers(0, n, (40, 2))]
    for ix, iy in pts:
        ref = _patch_reference((rho, u), om, ix, iy, 2)
        assert np.abs(f[:, iy, ix] - ref).max() <= FULL_SIZE_TOL[lbm.F32], (ix, iy)
    torch.cuda.synchronize()


# ---------------------------------------------------------------- packed two-rows-per-thread variant

@pytest.mark.parametrize("model", MODELS, ids=["cascaded", "bgk", "rawmrt"])
@pytest.mark.parametrize("edges,force", [("periodic", (0.0, 0.0)), ("cavity", (0.0, 0.0)),
                                         ("channel", (2e-5, 1e-5)), ("allmoving", (0.0, 0.0))])
def test_pair_variant_matches_oracle_and_scalar_variant(model, edges, force):
    """Variant 1 (two rows per thread, packed FP32x2) on a 67 x 45 lattice (odd
    row count: the last thread holds one row) against the oracle and variant 0."""
    nx, ny, steps = 67, 45, 300
    e, wu = EDGES[edges]
    rho, u = workloads.random_fields(8, nx, ny, u_amp=0.03, rho_amp=0.01)
    ref = O.Lattice(nx, ny, OMEGAS, force=force, edges=e, wall_u=wu, model=model).init(rho, u).run(steps)
    _, u_ref = ref.macros()
    out = {}
    for variant in (0, 1):
        g = lbm.Lattice(nx, ny, OMEGAS, force=force, edges=e, wall_u=wu, model=model, store=lbm.F32)
        g.set_variant(variant).init(rho, u).step(steps)
        out[variant] = g.get_f()
        _, ug = g.macros()
        assert rel_l2(ug, u_ref) <= 1e-5, variant
        g.close()
    assert rel_max(out[1], out[0]) <= 1e-6


@pytest.mark.parametrize("store", [lbm.BF16DEV, lbm.F16DEV], ids=["bf16", "f16"])
def test_pair_variant_reduced_precision_bound(store):
    n, om = 128, 1.6
    oms = (1.0, om, om, 1.0, 1.0, 1.0)
    rho, u = workloads.taylor_green_init(n, workloads.diffusive_u0(n))
    ref = O.Lattice(n, n, oms).init(rho, u).run(1000)
    _, u_ref = ref.macros()
    g = lbm.Lattice(n, n, oms, store=store).set_variant(1).init(rho, u).step(1000)
    _, ug = g.macros()
    assert rel_l2(ug, u_ref) <= REDUCED_BOUNDS[store]
    g.close()


# ---------------------------------------------------------------- four-nodes-per-thread vector variant

@pytest.mark.parametrize("store", [lbm.F16DEV, lbm.BF16DEV], ids=["f16", "bf16"])
@pytest.mark.parametrize("model", MODELS, ids=["cascaded", "bgk", "rawmrt"])
@pytest.mark.parametrize("edges,force", [("periodic", (0.0, 0.0)), ("cavity", (0.0, 0.0)),
                                         ("channel", (2e-5, 1e-5)), ("allmoving", (0.0, 0.0)),
                                         ("periodic", (1e-5, -2e-5))])
@pytest.mark.parametrize("shape", [(70, 37), (64, 9), (13, 5), (17, 3)])
def test_vector_variant_is_bitwise_equal_to_the_scalar_kernel(store, model, edges, force, shape):
    """Variant 2 (four nodes of a row per thread, 64-bit accesses, lane
    exchanges at vector edges, the per-node path at wrapped and wall neighbours
    and in the partial last vector) runs the scalar kernel's arithmetic, so the
    state must match variant 0 bit for bit after 1, 2 and 5 steps (both AA
    parities)."""
    nx, ny = shape
    e, wu = EDGES[edges]
    rho, u = workloads.random_fields(21, nx, ny, u_amp=0.03, rho_amp=0.01)
    states = {}
    for variant in (0, 2):
        g = lbm.Lattice(nx, ny, OMEGAS, force=force, edges=e, wall_u=wu, model=model, store=store)
        g.set_graph_steps(0)
        g.set_variant(variant).init(rho, u)
        states[variant] = []
        for n in (1, 1, 3):
            g.step(n)
            states[variant].append(g.get_f())
        g.close()
    for k, (a, b) in enumerate(zip(states[2], states[0])):
        np.testing.assert_array_equal(a, b, err_msg=f"chunk {k}")


@pytest.mark.parametrize("store", [lbm.F16DEV, lbm.BF16DEV], ids=["f16", "bf16"])
def test_vector_variant_with_a_force_field_runs_the_scalar_path(store):
    nx, ny = 40, 24
    rho, u = workloads.random_fields(5, nx, ny, u_amp=0.02, rho_amp=0.01)
    fxy = workloads.random_force_field(6, nx, ny, amp=1e-5)
    out = {}
    for variant in (0, 2):
        g = lbm.Lattice(nx, ny, OMEGAS, store=store).set_variant(variant)
        g.set_force_field(fxy)
        g.init(rho, u).step(3)
        out[variant] = g.get_f()
        g.close()
    np.testing.assert_array_equal(out[2], out[0])


@pytest.mark.parametrize("store", [lbm.BF16DEV, lbm.F16DEV], ids=["bf16", "f16"])
@pytest.mark.parametrize("variant", [0, 2])
def test_vector_variants_reduced_precision_bound(store, variant):
    n, om = 128, 1.6
    oms = (1.0, om, om, 1.0, 1.0, 1.0)
    rho, u = workloads.taylor_green_init(n, workloads.diffusive_u0(n))
    ref = O.Lattice(n, n, oms).init(rho, u).run(1000)
    _, u_ref = ref.macros()
    g = lbm.Lattice(n, n, oms, store=store).set_variant(variant).init(rho, u).step(1000)
    _, ug = g.macros()
    assert rel_l2(ug, u_ref) <= REDUCED_BOUNDS[store]
    g.close()


@pytest.mark.parametrize("store", [lbm.F64, lbm.F32, lbm.F16DEV], ids=["f64", "f32", "f16"])
def test_init_and_macros_read_and_write_pinned_host_buffers_in_place(store):
    """lbm_init / lbm_macros access mapped page-locked host buffers from the
    kernels directly and pageable ones through a staging copy; both paths must
    give the same state and fields, with NULL for either field."""
    import torch

    nx, ny = 70, 45
    e, wu = EDGES["cavity"]
    rho, u = workloads.random_fields(31, nx, ny, u_amp=0.03, rho_amp=0.01)
    lib = lbm.load_library()
    results = []
    for pinned in (False, True):
        g = lbm.Lattice(nx, ny, OMEGAS, edges=e, wall_u=wu, store=store)
        if pinned:
            rho_h = torch.from_numpy(rho).pin_memory()
            u_h = torch.from_numpy(u).pin_memory()
            lbm._check(lib.lbm_init(g.h, rho_h.data_ptr(), u_h.data_ptr()))
        else:
            g.init(rho, u)
        f0 = g.get_f()
        g.step(7)
        out_r = torch.zeros((ny, nx), dtype=torch.float64).pin_memory() if pinned else np.zeros((ny, nx))
        out_u = torch.zeros((2, ny, nx), dtype=torch.float64).pin_memory() if pinned else np.zeros((2, ny, nx))
        ptr = (lambda t: t.data_ptr()) if pinned else (lambda a: a.ctypes.data)
        lbm._check(lib.lbm_macros(g.h, ptr(out_r), ptr(out_u)))
        only_u = torch.zeros((2, ny, nx), dtype=torch.float64).pin_memory() if pinned else np.zeros((2, ny, nx))
        lbm._check(lib.lbm_macros(g.h, None, ptr(only_u)))
        if pinned:
            lbm._check(lib.lbm_init(g.h, None, u_h.data_ptr()))  # rho defaults to rho0
        else:
            g.init(None, u)
        f_rest = g.get_f()
        g.close()
        as_np = (lambda t: t.numpy()) if pinned else (lambda a: a)
        results.append((f0, as_np(out_r).copy(), as_np(out_u).copy(), as_np(only_u).copy(), f_rest))
    for a, b in zip(results[0], results[1]):
        np.testing.assert_array_equal(a, b)
    np.testing.assert_array_equal(results[1][2], results[1][3])


# ---------------------------------------------------------------- stochastic rounding of the stores

@pytest.mark.parametrize("store", [lbm.F16DEV, lbm.BF16DEV, lbm.F32], ids=["f16", "bf16", "f32"])
@pytest.mark.parametrize("model", MODELS, ids=["cascaded", "bgk", "rawmrt"])
@pytest.mark.parametrize("edges,force", [("periodic", (0.0, 0.0)), ("cavity", (0.0, 0.0)),
                                         ("channel", (2e-5, 1e-5))])
def test_stochastic_rounding_is_the_same_in_every_variant_and_graph_length(store, model, edges, force):
    """The random bits depend only on (seed, step, node, population): the
    four-node kernel, the one-node kernel and CUDA-graph replays of any length
    give the same states bit for bit; the same seed repeats a run, another seed
    does not."""
    nx, ny = 70, 37
    e, wu = EDGES[edges]
    rho, u = workloads.random_fields(41, nx, ny, u_amp=0.03, rho_amp=0.01)

    def run(variant, graph_steps, seed):
        g = lbm.Lattice(nx, ny, OMEGAS, force=force, edges=e, wall_u=wu, model=model, store=store)
        g.set_variant(variant).set_graph_steps(graph_steps).set_rounding(lbm.ROUND_STOCHASTIC, seed)
        g.init(rho, u)
        out = []
        for n in (3, 8, 21):
            g.step(n)
            out.append(g.get_f())
        g.close()
        return out

    ref = run(0, 0, 7)
    # FP32 storage has variants 0 and 1 (variant 1 runs variant 0 in this mode)
    others = ((1, 0), (0, 8), (1, 8), (0, 64)) if store == lbm.F32 else ((2, 0), (0, 8), (2, 8), (2, 64))
    for variant, graph_steps in others:
        for k, (a, b) in enumerate(zip(run(variant, graph_steps, 7), ref)):
            np.testing.assert_array_equal(a, b, err_msg=f"variant {variant}, graph {graph_steps}, chunk {k}")
    other = run(0, 0, 8)
    assert not np.array_equal(other[-1], ref[-1])
    nearest = lbm.Lattice(nx, ny, OMEGAS, force=force, edges=e, wall_u=wu, model=model, store=store)
    nearest.init(rho, u).step(32)
    f_rn = nearest.get_f()
    nearest.close()
    assert not np.array_equal(f_rn, ref[-1])
    # the same flow, rounded differently
    assert np.abs(ref[-1] - f_rn).max() <= (1e-3 if store != lbm.F32 else 1e-6)


@pytest.mark.parametrize("store", [lbm.F16DEV, lbm.BF16DEV, lbm.F32], ids=["f16", "bf16", "f32"])
def test_stochastic_rounding_keeps_mass_and_rejects_misuse(store):
    n = 128
    rho, u = workloads.taylor_green_init(n, workloads.diffusive_u0(n))
    g = lbm.Lattice(n, n, OMEGAS, store=store).set_rounding(lbm.ROUND_STOCHASTIC, 3).init(rho, u)
    m0 = g.stats()[0]
    g.step(1000)
    m1 = g.stats()[0]
    assert abs(m1 - m0) / m0 <= {lbm.F16DEV: 2e-6, lbm.BF16DEV: 2e-5, lbm.F32: 1e-10}[store]
    with pytest.raises(lbm.LBMError):
        g.set_rounding(5)
    g.set_rounding(lbm.ROUND_NEAREST)
    g.close()
    f64 = lbm.Lattice(16, 16, OMEGAS, store=lbm.F64)
    with pytest.raises(lbm.LBMError):
        f64.set_rounding(lbm.ROUND_STOCHASTIC, 1)
    f64.set_rounding(lbm.ROUND_NEAREST)
    f64.close()


def test_fp32_stochastic_rounding_removes_the_storage_drift():
    """Taylor-Green on 4096^2 (the bench workload, U0 = 6.25e-4): the viscous
    change of a stored deviation per step is only a few FP32 units in the last
    place, and round to nearest loses part of it every step, so the decay drifts
    away from the analytic one.  With the collision's last addition formed as an
    error-free sum and its remainder rounded in stochastically the stored state
    is unbiased.  After T/50 steps (Sec. III-B: T = 1 / (2 nu k^2)) the
    stochastic run's velocity error against the analytic decay stays below
    1e-6 (the discretisation error at this size is about 2e-7, relative L2),
    several times smaller than the round-to-nearest run's."""
    n = 4096
    om = OMEGAS[1]
    nu = (1.0 / om - 0.5) / 3.0
    u0 = workloads.diffusive_u0(n)
    steps = workloads.taylor_green_decay_steps(n, nu) // 50
    rho, u = workloads.taylor_green_init(n, u0)
    ua = workloads.taylor_green_velocity(n, u0, nu, steps)
    res = {}
    for mode in (lbm.ROUND_NEAREST, lbm.ROUND_STOCHASTIC):
        with lbm.Lattice(n, n, (1.0, om, om, 1.0, 1.0, 1.0), store=lbm.F32) as g:
            g.set_rounding(mode, 11).init(rho, u).step(steps)
            _, ug = g.macros()
        res[mode] = (float(np.sqrt(((ug - ua) ** 2).sum() / (ua ** 2).sum())), float((ug * ua).sum() / (ua * ua).sum()))
        print("FP32", "stochastic" if mode else "nearest", steps, "steps: u error %.3e, amplitude %.8f" % res[mode])
    err_sr, _ = res[lbm.ROUND_STOCHASTIC]
    err_rn, _ = res[lbm.ROUND_NEAREST]
    assert err_sr < 1e-6
    assert err_rn > 3 * err_sr  # measured: 2.6e-6 against 3.8e-7


def test_tune_keeps_state_and_picks_a_variant():
    n = 256
    rho, u = workloads.taylor_green_init(n, workloads.diffusive_u0(n))
    g = lbm.Lattice(n, n, OMEGAS, store=lbm.F16DEV).init(rho, u).step(3)
    before = g.get_f()
    ms = g.tune(10)
    assert all(m > 0 for m in ms)  # 16-bit storage admits variants 0..3
    np.testing.assert_array_equal(g.get_f(), before)
    assert g.time == 3
    g.close()


# ---------------------------------------------------------------- CUDA-graph replay in lbm_step

@pytest.mark.parametrize("store", [lbm.F32, lbm.F16DEV, lbm.F64], ids=["f32", "f16", "f64"])
def test_graph_replay_is_bitwise_equal_to_single_launches(store):
    """lbm_step replays chunks of steps from a CUDA graph; the result must not
    depend on it, also across an odd start, a rate change and a force change
    (each forces a new capture)."""
    nx, ny = 70, 45
    e, wu = EDGES["channel"]
    rho, u = workloads.random_fields(12, nx, ny, u_amp=0.03, rho_amp=0.01)
    runs = []
    for graph_steps in (0, 8):
        g = lbm.Lattice(nx, ny, OMEGAS, force=(1e-5, 0.0), edges=e, wall_u=wu, store=store)
        g.set_graph_steps(graph_steps).init(rho, u)
        g.step(3)     # odd: the next chunk starts with single launches
        g.step(37)
        g.set_omegas((1.0, 1.5, 1.5, 1.0, 1.1, 1.0))
        g.step(20)
        g.set_force((0.0, 2e-5))
        g.step(33)
        assert g.time == 93
        runs.append(g.get_f())
        g.close()
    np.testing.assert_array_equal(runs[0], runs[1])


# ---------------------------------------------------------------- two fused steps per launch (variant 3)

FUSED_CASES = [  # (nx, ny, edges, force, force field, store, rounding)
    (200, 70, "periodic", (0.0, 0.0), False, lbm.F32, False),
    (128, 32, "periodic", (0.0, 0.0), False, lbm.F16DEV, False),
    (131, 45, "cavity", (0.0, 0.0), False, lbm.F32, False),
    (131, 45, "cavity", (0.0, 0.0), False, lbm.BF16DEV, False),
    (70, 37, "channel", (2e-5, 1e-5), False, lbm.F32, False),
    (70, 37, "channel", (2e-5, 1e-5), False, lbm.F16DEV, True),
    (66, 17, "periodic", (0.0, 0.0), True, lbm.F32, False),
    (100, 33, "cavity", (0.0, 0.0), False, lbm.F32, True),
    (5, 7, "periodic", (1e-5, 0.0), False, lbm.F32, False),
    (4, 4, "cavity", (0.0, 0.0), False, lbm.F16DEV, False),
    (90, 40, "allmoving", (1e-5, -2e-5), False, lbm.F32, False),
    (77, 50, "ychannel", (0.0, 3e-5), False, lbm.BF16DEV, True),
    # tiles away from every wall (the odd step's body without wall links) beside tiles at the walls
    (260, 70, "cavity", (0.0, 0.0), False, lbm.F32, True),
    (200, 70, "channel", (2e-5, 1e-5), False, lbm.F16DEV, False),
    # periodic, unforced FP32: the cascaded collision runs in packed FP32x2 pairs here
    (130, 33, "periodic", (0.0, 0.0), False, lbm.F32, False),
    (64, 16, "periodic", (0.0, 0.0), False, lbm.F32, False),
    (4, 4, "periodic", (0.0, 0.0), False, lbm.F32, False),
]


@pytest.mark.parametrize("model", MODELS, ids=["cascaded", "bgk", "rawmrt"])
@pytest.mark.parametrize("case", FUSED_CASES, ids=[f"{c[0]}x{c[1]}-{c[2]}-{lbm.STORE_NAMES[c[5]]}"
                                                   f"{'-field' if c[4] else ''}{'-sr' if c[6] else ''}"
                                                   for c in FUSED_CASES])
def test_fused_two_step_variant_is_bitwise_equal_to_single_steps(model, case):
    """Variant 3 takes two steps per launch in shared memory (TMA tile load,
    halo of two nodes, ping-pong arrays); every node's arithmetic and every
    rounding of the stored values are those of two single steps, so the states
    agree bit for bit: across ragged tiles, lattice edges with periodic wrap,
    walls and moving walls, forces and force fields, stochastic rounding, an odd
    start, and CUDA-graph replays; also where the kernel collides node pairs in
    packed FP32x2 arithmetic (periodic, unforced, FP32, cascaded)."""
    nx, ny, edges, force, field, store, sr = case
    e, wu = EDGES[edges]
    rho, u = workloads.random_fields(71, nx, ny, u_amp=0.03, rho_amp=0.01)
    ff = workloads.random_force_field(5, nx, ny, 1e-5) if field else None

    def run(variant, graph_steps):
        g = lbm.Lattice(nx, ny, OMEGAS, force=force, edges=e, wall_u=wu, model=model, store=store)
        g.set_variant(variant).set_graph_steps(graph_steps)
        if sr:
            g.set_rounding(lbm.ROUND_STOCHASTIC, 9)
        if ff is not None:
            g.set_force_field(ff)
        g.init(rho, u)
        out = []
        for n in (1, 6, 2, 13, 40):  # odd start after the first call; graph replays in the last
            g.step(n)
            out.append(g.get_f())
        info = g.info()
        g.close()
        return out, info

    ref, _ = run(0, 0)
    for graph_steps in (0, 8, 64):
        got, info = run(3, graph_steps)
        assert info["variant"] == 3
        for k, (a, b) in enumerate(zip(got, ref)):
            np.testing.assert_array_equal(a, b, err_msg=f"graph {graph_steps}, chunk {k}")


def test_fused_variant_is_rejected_for_fp64_and_tuned_elsewhere():
    n = 256
    rho, u = workloads.taylor_green_init(n, workloads.diffusive_u0(n))
    g = lbm.Lattice(n, n, OMEGAS, store=lbm.F64).set_variant(3)
    assert g.info()["variant"] == 0  # FP64 admits variant 0 only
    g.close()
    g = lbm.Lattice(n, n, OMEGAS, store=lbm.F32).init(rho, u).step(3)
    before = g.get_f()
    ms = g.tune(10)
    assert ms[0] > 0 and ms[1] > 0 and ms[2] == 0 and ms[3] > 0  # FP32: variants 0, 1, 3
    np.testing.assert_array_equal(g.get_f(), before)
    assert g.time == 3
    g.close()
