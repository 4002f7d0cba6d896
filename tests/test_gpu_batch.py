"""Batched persistent launch (lbm_batch_*, through the C ABI).

The batch runs the same per-node update as lbm_step, so every lattice of a
batch must end bit-for-bit where the same lattice stepped alone ends; that
single-lattice path is itself pinned to the oracle (test_gpu_parity).
"""
import numpy as np
import pytest

import oracle as O
from paper_1202_6351_gb300 import lbm, workloads

pytestmark = pytest.mark.gpu

P, BB, MW = lbm.PERIODIC, lbm.BOUNCEBACK, lbm.MOVING_WALL
OM = (1.1, 1.7, 1.7, 1.0, 1.2, 0.9)

# (nx, ny, store, edges, wall_u, force, init)
DOMAINS = [
    (64, 64, lbm.F32, (P, P, P, P), (0, 0, 0, 0), (0, 0), "tg"),
    (50, 37, lbm.F16DEV, (BB, BB, BB, MW), (0, 0, 0, 0.1), (0, 0), "rest"),
    (33, 20, lbm.BF16DEV, (P, P, BB, BB), (0, 0, 0, 0), (2e-5, 0), "rest"),
    (100, 100, lbm.F16DEV, (P, P, P, P), (0, 0, 0, 0), (0, 0), "tg"),
    (129, 97, lbm.F32, (BB, BB, BB, MW), (0, 0, 0, 0.08), (0, 0), "random"),
    (5, 3, lbm.F32, (P, P, P, P), (0, 0, 0, 0), (1e-4, -1e-4), "random"),
    (1, 1, lbm.F32, (P, P, P, P), (0, 0, 0, 0), (0, 0), "random"),
    (260, 7, lbm.F16DEV, (MW, MW, P, P), (0.02, -0.03, 0, 0), (0, 1e-5), "random"),
]


@pytest.fixture(scope="module", autouse=True)
def cuda():
    import torch

    assert torch.cuda.is_available(), "GPU tests need a CUDA device"
    torch.cuda.set_device(0)
    yield


def make(spec, seed):
    nx, ny, store, edges, wall_u, force, init = spec
    L = lbm.Lattice(nx, ny, OM, force=force, edges=edges, wall_u=wall_u, store=store)
    if init == "tg":
        rho, u = workloads.taylor_green_init(nx, 0.03)
        L.init(rho, u)
    elif init == "random":
        rho, u = workloads.random_fields(seed, nx, ny, u_amp=0.03, rho_amp=0.01)
        L.init(rho, u)
    else:
        L.init()
    return L


def with_rounding(L, i):
    """Stochastic rounding on the 16-bit lattices except domain 3 and on the
    FP32 lattices 4 and 5 (seed = index)."""
    if (L.store in (lbm.F16DEV, lbm.BF16DEV) and i != 3) or i in (4, 5):
        L.set_rounding(lbm.ROUND_STOCHASTIC, i)
    return L


@pytest.mark.parametrize("rounding", [False, True], ids=["nearest", "mixed_stochastic"])
@pytest.mark.parametrize("tune", [False, True], ids=["default", "tuned"])
def test_batch_is_bitwise_equal_to_single_lattice_steps(tune, rounding):
    alone = [make(s, i) for i, s in enumerate(DOMAINS)]
    batched = [make(s, i) for i, s in enumerate(DOMAINS)]
    if rounding:  # the batch's per-domain round table must reproduce lbm_step's hashes
        alone = [with_rounding(L, i) for i, L in enumerate(alone)]
        batched = [with_rounding(L, i) for i, L in enumerate(batched)]
        assert {L.store for i, L in enumerate(batched) if L.store != lbm.F32 and i != 3} == {lbm.F16DEV, lbm.BF16DEV}
    # start two lattices one step ahead: the batch handles mixed parities
    for k in (1, 4):
        alone[k].step(1)
        batched[k].step(1)
    with lbm.Batch(batched) as B:
        B.set_graph_steps(10)
        if tune:
            before = [L.get_f() for L in batched]
            B.tune(3)
            for L, f in zip(batched, before):
                np.testing.assert_array_equal(L.get_f(), f)  # tuning leaves the states unchanged
        B.step(37)  # three graphs of 10 steps and 7 single launches
        B.step(3)
        B.sync()
    for L in alone:
        L.step(40)
    for i, (a, b) in enumerate(zip(alone, batched)):
        assert a.time == b.time
        np.testing.assert_array_equal(a.get_f(), b.get_f(), err_msg=f"domain {i}")
    for L in alone + batched:
        L.close()


# lattices of at least 4 x 4 nodes: every one admits two steps per launch
DOMAINS_TWO_STEP = [d for d in DOMAINS if d[0] >= 4 and d[1] >= 4] + [
    (200, 70, lbm.F32, (P, P, P, P), (0, 0, 0, 0), (0, 0), "random"),
    (64, 16, lbm.F16DEV, (BB, BB, MW, MW), (0, 0, -0.05, 0.05), (0, 0), "random"),
    (4, 4, lbm.BF16DEV, (P, P, P, P), (0, 0, 0, 0), (1e-5, 0), "random"),
]


@pytest.mark.parametrize("rounding", [False, True], ids=["nearest", "mixed_stochastic"])
@pytest.mark.parametrize("start", [0, 1], ids=["even_start", "odd_start"])
def test_batch_two_steps_per_launch_is_bitwise_equal_to_single_steps(start, rounding):
    """lbm_batch_set_two_step: one CTA per 64 x 16 tile of any lattice takes two
    steps in shared memory, the lattices' arrays trading roles at every launch;
    an odd start or end takes one single batched step.  Every lattice ends bit for
    bit where it ends stepped alone, across graph replays and single launches."""
    alone = [make(s, i) for i, s in enumerate(DOMAINS_TWO_STEP)]
    batched = [make(s, i) for i, s in enumerate(DOMAINS_TWO_STEP)]
    if rounding:
        alone = [with_rounding(L, i) for i, L in enumerate(alone)]
        batched = [with_rounding(L, i) for i, L in enumerate(batched)]
    for L in alone + batched:
        L.step(start)
    with lbm.Batch(batched) as B:
        B.set_graph_steps(12)
        B.set_two_step(True)
        assert B.info()["policy"] == "two_steps_per_launch"
        B.step(29)  # [a single step,] two replays of 6 two-step launches, single launches[, a single step]
        B.step(4)
        B.sync()
    for L in alone:
        L.step(33)
    for i, (a, b) in enumerate(zip(alone, batched)):
        assert a.time == b.time
        np.testing.assert_array_equal(a.get_f(), b.get_f(), err_msg=f"domain {i}")
    for L in alone + batched:
        L.close()


def test_batch_two_step_follows_lattices_that_change_force_or_rounding():
    """The two-step batch runs one kernel per class of lattice (storage kind,
    walls, force, rounding).  A lattice that turns its force or stochastic
    rounding on or off between batch calls moves to another class; the
    following launches (graph replays included) must take it along and still
    match single steps bit for bit."""
    alone = [make(s, i) for i, s in enumerate(DOMAINS_TWO_STEP)]
    batched = [make(s, i) for i, s in enumerate(DOMAINS_TWO_STEP)]

    def change(Ls, phase):
        if phase == 0:
            Ls[0].set_rounding(lbm.ROUND_STOCHASTIC, 11)  # FP32 periodic: leaves the packed class
            Ls[3].set_force((3e-5, -1e-5))  # FP16 periodic, now forced
            Ls[2].set_force((0.0, 0.0))  # BF16 with walls, now unforced
        else:
            Ls[0].set_rounding(lbm.ROUND_NEAREST)
            Ls[7].set_rounding(lbm.ROUND_STOCHASTIC, 5)

    with lbm.Batch(batched) as B:
        B.set_graph_steps(8)
        B.set_two_step(True)
        B.step(10)
        change(batched, 0)
        B.step(12)
        change(batched, 1)
        B.step(8)
        B.sync()
    for L in alone:
        L.step(10)
    change(alone, 0)
    for L in alone:
        L.step(12)
    change(alone, 1)
    for L in alone:
        L.step(8)
    for i, (a, b) in enumerate(zip(alone, batched)):
        assert a.time == b.time
        np.testing.assert_array_equal(a.get_f(), b.get_f(), err_msg=f"domain {i}")
    for L in alone + batched:
        L.close()


def test_batch_tuner_with_the_two_step_candidate_leaves_states_unchanged():
    """The batch tuner also times two steps per launch when every lattice admits
    it and all are at the same even step; its trial launches swap each
    lattice's two arrays an even number of times and the states are restored,
    so tuning changes nothing, and the steps after it match single steps bit
    for bit whichever configuration it keeps."""
    alone = [make(s, i) for i, s in enumerate(DOMAINS_TWO_STEP)]
    batched = [make(s, i) for i, s in enumerate(DOMAINS_TWO_STEP)]
    with lbm.Batch(batched) as B:
        before = [L.get_f() for L in batched]
        B.tune(4)
        for L, f in zip(batched, before):
            np.testing.assert_array_equal(L.get_f(), f)
        assert B.info()["policy"] in ("round_robin", "chunked", "dynamic", "one_cta_per_tile", "two_steps_per_launch")
        B.step(22)
        B.sync()
    for L in alone:
        L.step(22)
    for i, (a, b) in enumerate(zip(alone, batched)):
        np.testing.assert_array_equal(a.get_f(), b.get_f(), err_msg=f"domain {i}")
    for L in alone + batched:
        L.close()


def test_batch_two_step_needs_4x4_lattices_and_falls_back_on_mixed_parity():
    small = [make(DOMAINS[6], 0), make(DOMAINS[0], 1)]  # a 1 x 1 lattice
    with lbm.Batch(small) as B:
        with pytest.raises(lbm.LBMError):
            B.set_two_step(True)
    alone = [make(DOMAINS[0], 1), make(DOMAINS[3], 2)]
    batched = [make(DOMAINS[0], 1), make(DOMAINS[3], 2)]
    alone[0].step(1)
    batched[0].step(1)
    with lbm.Batch(batched) as B:
        B.set_two_step(True)
        B.step(6)  # parities differ: single batched steps
        B.sync()
    for L in alone:
        L.step(6)
    for a, b in zip(alone, batched):
        np.testing.assert_array_equal(a.get_f(), b.get_f())
    for L in alone + batched:
        L.close()


def test_batch_cavity_matches_oracle():
    n, U, re = 65, 0.1, 400.0
    om = O.omega_from_nu(U * (n - 1) / re)
    oms = (1.0, om, om, 1.0, 1.0, 1.0)
    edges = (BB, BB, BB, MW)
    Ls = [lbm.Lattice(n, n, oms, edges=edges, wall_u=(0, 0, 0, U), store=lbm.F32).init(),
          lbm.Lattice(40, 40, oms, store=lbm.F16DEV).init()]
    with lbm.Batch(Ls) as B:
        B.tune(2)
        B.step(1000)
        B.sync()
    _, u = Ls[0].macros()
    ref = O.Lattice(n, n, oms, edges=edges, wall_u=(0, 0, 0, U)).init().run(1000)
    _, u_ref = ref.macros()
    assert np.sqrt(((u - u_ref) ** 2).sum() / (u_ref ** 2).sum()) <= 1e-5
    for L in Ls:
        L.close()


def test_batch_rejects_unsupported_lattices():
    a = lbm.Lattice(8, 8, OM, store=lbm.F64)
    b = lbm.Lattice(8, 8, OM, store=lbm.F32)
    c = lbm.Lattice(8, 8, OM, store=lbm.F32, model=lbm.BGK)
    for group in ([a], [b, c], [b, b]):
        with pytest.raises(lbm.LBMError) as ei:
            lbm.Batch(group)
        assert ei.value.code == lbm.LBM_EINVAL
    for L in (a, b, c):
        L.close()


def test_full_size_96_domain_ensemble_two_steps_per_launch():
    """The batched ensemble at full size (the 96 domains of
    workloads.batch_domains(): sides 64..2048, lid-driven cavities at Re
    100..5000 and Taylor-Green vortices, FP32 and FP16 storage, 52.9 M nodes)
    in the configuration the bench's batch tuner keeps, two steps per launch
    (one kernel per class of lattice, a graph replay among the launches):
    every lattice ends bit for bit where it ends stepped alone."""
    def build():
        Ls = []
        for d in workloads.batch_domains():
            n = d["side"]
            st = lbm.F32 if d["store"] == "f32" else lbm.F16DEV
            if d["kind"] == "cavity":
                U = 0.1
                om = 1.0 / (3.0 * U * (n - 1) / d["re"] + 0.5)
                L = lbm.Lattice(n, n, (1.0, om, om, 1.0, 1.0, 1.0), edges=(BB, BB, BB, MW), wall_u=(0, 0, 0, U),
                                store=st).init()
            else:
                rho, u = workloads.taylor_green_init(n, workloads.diffusive_u0(n))
                L = lbm.Lattice(n, n, (1.0, 1.6, 1.6, 1.0, 1.0, 1.0), store=st).init(rho, u)
            Ls.append(L)
        return Ls

    batched = build()
    with lbm.Batch(batched) as B:
        B.set_graph_steps(8)
        B.set_two_step(True)
        B.step(10)  # one replay of four two-step launches, then one more launch
        B.sync()
    alone = build()
    for i, (a, b) in enumerate(zip(alone, batched)):
        a.step(10)
        assert a.time == b.time == 10
        np.testing.assert_array_equal(a.get_f(), b.get_f(), err_msg=f"domain {i} ({a.shape})")
        a.close()
        b.close()
