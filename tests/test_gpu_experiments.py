"""Results of Sec. III-V reproduced on the CUDA path: Taylor-Green decay and
grid convergence, and the lid-driven cavity (context pins: the paper's own
printed numbers, at a coarser grid than the paper's)."""
import math

import numpy as np
import pytest

import oracle as O
from paper_1202_6351_gb300 import experiments as X
from paper_1202_6351_gb300 import lbm, workloads
from tests import _pins as P

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def cuda():
    import torch

    assert torch.cuda.is_available(), "GPU tests need a CUDA device"
    torch.cuda.set_device(0)
    yield


@pytest.mark.parametrize("re", [100, 1000])
def test_primary_vortex_centre_matches_table_I(re):
    """Sec. IV-C, Table I: cascaded (x, y) of the primary vortex at 401^2; here
    257^2 in FP32 storage, run to max |du| < 1e-7 per 1000 steps."""
    table = P.PAPER["primary_vortex"]
    k = table["re"].index(re)
    u, steps = X.cavity_steady(257, re, model=lbm.CASCADED)
    xc, yc = X.vortex_centre(u)
    px, py = table["cascaded"][k]
    print(f"Re {re}: cascaded centre ({xc:.5f}, {yc:.5f}) after {steps} steps; paper ({px}, {py})")
    assert abs(xc - px) < 0.01 and abs(yc - py) < 0.01
    # Table II: first secondary vortices in the bottom corners (no top-left one below Re 3200)
    sec = P.PAPER["secondary_vortices"]["cascaded"][str(re)]
    for region in ("bottom_left", "bottom_right"):
        got = X.secondary_vortex(u, region)
        print(f"Re {re}: {region} vortex {got}; paper {sec[region]}")
        assert got is not None
        assert abs(got[0] - sec[region][0]) < 0.01 and abs(got[1] - sec[region][1]) < 0.01
    assert X.secondary_vortex(u, "top_left") is None
    if re == 1000:  # the raw-moment MRT lands on the same centre (the paper: within 0.014 %)
        um, _ = X.cavity_steady(257, re, model=lbm.RAWMRT)
        xm, ym = X.vortex_centre(um)
        print(f"Re {re}: raw-MRT centre ({xm:.5f}, {ym:.5f})")
        assert abs(xm - xc) < 2e-3 and abs(ym - yc) < 2e-3


def test_stability_ordering_of_table_IV():
    """Sec. V, Table IV: the maximum stable cell Reynolds number grows from SRT to
    raw MRT to cascaded (14.14 / 59.40 / 148.50 at 101^2 in the paper; raw MRT
    3-4 times SRT and cascaded 2-3 times raw MRT); a run is stable unless it
    blows up within 20 convective times."""
    th = {}
    for model in (lbm.BGK, lbm.RAWMRT, lbm.CASCADED):
        th[model], _ = X.max_stable_cell_reynolds(model, 101)
    print("max stable cell Re at 101^2: SRT %.1f, raw MRT %.1f, cascaded %.1f" % (th[lbm.BGK], th[lbm.RAWMRT],
                                                                                  th[lbm.CASCADED]))
    assert 12.0 <= th[lbm.BGK] <= 17.0
    assert th[lbm.RAWMRT] >= 3.0 * th[lbm.BGK]
    assert th[lbm.CASCADED] >= 1.8 * th[lbm.RAWMRT]


def test_max_stable_lid_velocity_on_a_coarse_grid():
    """Sec. V's alternative test: 26 x 26 cavity, fixed viscosity, largest lid
    speed stable for 50,000 steps; the cascaded model reaches a considerably
    higher speed than the other two (here nu = 0.005)."""
    th = {}
    for model in (lbm.BGK, lbm.RAWMRT, lbm.CASCADED):
        th[model], _ = X.max_stable_lid_velocity(model, 0.005)
    print("max stable lid speed at 26^2, nu 0.005: SRT %.4f, raw MRT %.4f, cascaded %.4f" % (
        th[lbm.BGK], th[lbm.RAWMRT], th[lbm.CASCADED]))
    assert th[lbm.BGK] < th[lbm.RAWMRT] < th[lbm.CASCADED]
    assert th[lbm.CASCADED] >= 1.5 * th[lbm.RAWMRT]


@pytest.mark.parametrize("re", [100, 1000])
def test_strain_rate_from_moments_agrees_with_finite_differences(re):
    """Sec. IV-C, Table III: the strain rate from local non-equilibrium moments
    (Eq. 28-30) agrees with central differences of the velocity at the five
    probe points (the paper: within 2 %)."""
    rho, u, strain, steps = X.cavity_steady(257, re, fields=True)
    pts = X.strain_at_points(rho, u, strain)
    scale = max(max(abs(v[1]), abs(v[3])) for v in pts.values())
    paper = P.PAPER["strain_rate_points"][str(re)]
    for name, (dm, dfd, sm, sfd) in pts.items():
        print(f"Re {re} point {name}: dv/dy {dm:.4e} (moments) {dfd:.4e} (FD) paper {paper['dvdy'][name]:.4e}; "
              f"du/dy+dv/dx {sm:.4e} (moments) {sfd:.4e} (FD) paper {paper['shear'][name]:.4e}")
        assert abs(dm - dfd) <= 0.02 * max(abs(dfd), 0.1 * scale)
        assert abs(sm - sfd) <= 0.02 * max(abs(sfd), 0.1 * scale)
        # Table III's grid is not stated, so its magnitudes (lattice units, ~U/N) are
        # not comparable; the sign of each component at each point is.
        assert np.sign(dm) == np.sign(paper["dvdy"][name]) and np.sign(sm) == np.sign(paper["shear"][name])


def test_taylor_green_strain_rate_converges_at_second_order_on_the_gpu():
    """Sec. III-B: S_xx from the non-equilibrium moments falls as N^-2 against
    Eq. 41 under diffusive scaling (FP64 storage, one decay time)."""
    import math

    import oracle as O
    from paper_1202_6351_gb300 import workloads

    om = 1.6
    nu = O.nu_from_omega(om)
    errs = []
    for n in (32, 64, 128):
        u0 = workloads.diffusive_u0(n)
        steps = int(round(O.taylor_green_decay_time(n, nu)))
        rho0, u_init = workloads.taylor_green_init(n, u0)
        with lbm.Lattice(n, n, (1.0, om, om, 1.0, 1.0, 1.0), store=lbm.F64) as L:
            L.init(rho0, u_init).step(steps)
            rho, _ = L.macros()
            sxx = L.strain()[0] / rho
        _, _, sa = O.taylor_green(n, u0, nu, steps)
        errs.append(float(np.sqrt(((sxx - sa) ** 2).sum() / (sa ** 2).sum())))
    slopes = [math.log2(errs[k] / errs[k + 1]) for k in range(2)]
    print("S_xx errors", errs, "slopes", slopes)
    assert all(1.9 < s < 2.15 for s in slopes)


# Relative L2 velocity error at one decay time for 16-bit storage, as measured
# (stated bounds with some margin): round to nearest drops every per-step change
# below half a spacing of the stored type, which stalls part of the slow viscous
# decay, so the error grows with the number of steps and is not monotone in N.
ONE_DECAY_TIME_BOUNDS = {lbm.F16DEV: {64: 5e-3, 128: 1.5e-2, 256: 0.3, 1024: 6e-2},
                         lbm.BF16DEV: {64: 0.1, 128: 0.3, 256: 0.1, 1024: 0.7}}


def test_taylor_green_to_one_decay_time():
    """The Taylor-Green configuration (Sec. III-B) on N = 64, 128, 256, 1024, run
    to one decay time T = N^2 / (8 pi^2 nu) (1245 .. 318729 steps) and checked
    against the analytic decay: in FP32 the velocity error falls at second order
    (the paper: slopes 1.98-1.99), and S_xx from the moments (Eq. 28-30) too up
    to N = 256 (at 1024 FP32 rounding of the small non-equilibrium moments sets a
    floor near 1e-5); the 16-bit stores meet their stated bounds."""
    om = 1.6
    nu = O.nu_from_omega(om)
    oms = (1.0, om, om, 1.0, 1.0, 1.0)
    sides = (64, 128, 256, 1024)
    errs = {}
    for st in (lbm.F32, lbm.F16DEV, lbm.BF16DEV):
        for n in sides:
            u0 = workloads.diffusive_u0(n)
            T = int(round(O.taylor_green_decay_time(n, nu)))
            rho, u = workloads.taylor_green_init(n, u0)
            with lbm.Lattice(n, n, oms, store=st) as L:
                L.init(rho, u).step(T)
                r, ug = L.macros()
                sxx = L.strain()[0] / r
            _, ua, sa = O.taylor_green(n, u0, nu, T)
            errs[st, n] = (float(np.sqrt(((ug - ua) ** 2).sum() / (ua ** 2).sum())),
                           float(np.sqrt(((sxx - sa) ** 2).sum() / (sa ** 2).sum())))
            print(lbm.STORE_NAMES[st], n, T, "u error %.3e, S_xx error %.3e" % errs[st, n])
    for a, b in zip(sides, sides[1:]):
        slope_u = math.log(errs[lbm.F32, a][0] / errs[lbm.F32, b][0]) / math.log(b / a)
        assert 1.85 < slope_u < 2.2, (a, b, slope_u)
        if b <= 256:
            slope_s = math.log(errs[lbm.F32, a][1] / errs[lbm.F32, b][1]) / math.log(b / a)
            assert 1.85 < slope_s < 2.2, (a, b, slope_s)
    assert errs[lbm.F32, 1024][1] < 2e-5
    for st, bounds in ONE_DECAY_TIME_BOUNDS.items():
        for n, bound in bounds.items():
            assert errs[st, n][0] <= bound, (lbm.STORE_NAMES[st], n, errs[st, n][0])


@pytest.mark.parametrize("store", [lbm.F16DEV, lbm.BF16DEV], ids=["f16", "bf16"])
def test_stochastic_rounding_keeps_16bit_storage_accurate_to_one_decay_time(store):
    """With stochastic rounding of the stored deviations the 16-bit runs no
    longer drift: the Taylor-Green velocity error at one decay time stays at the
    storage's noise level on every grid (round to nearest: up to 0.22 in FP16 and
    0.53 in BF16, ONE_DECAY_TIME_BOUNDS)."""
    om = 1.6
    nu = O.nu_from_omega(om)
    oms = (1.0, om, om, 1.0, 1.0, 1.0)
    bound = 2.5e-3 if store == lbm.F16DEV else 1e-2
    for n in (64, 128, 256, 1024):
        u0 = workloads.diffusive_u0(n)
        T = int(round(O.taylor_green_decay_time(n, nu)))
        rho, u = workloads.taylor_green_init(n, u0)
        with lbm.Lattice(n, n, oms, store=store) as L:
            L.set_rounding(lbm.ROUND_STOCHASTIC, 2026).init(rho, u).step(T)
            _, ug = L.macros()
        _, ua, _ = O.taylor_green(n, u0, nu, T)
        err = float(np.sqrt(((ug - ua) ** 2).sum() / (ua ** 2).sum()))
        amp = float((ug * ua).sum() / (ua * ua).sum())
        print(lbm.STORE_NAMES[store], n, T, "stochastic rounding: u error %.3e, amplitude %.5f" % (err, amp))
        assert err <= bound and abs(amp - 1.0) <= bound


def test_cavity_grid_convergence_second_order():
    """Sec. III-C: Re 100 under diffusive scaling, grids 13^2..121^2 against an
    801^2 run; the relative global errors of the centre-line velocities and
    strain rates fall at about second order (the paper's fitted slopes: 2.11 /
    2.19 for u, 2.18 / 2.11 for v, 1.81 / 1.95 for dv/dy, 2.12 / 2.07 for
    du/dy + dv/dx on the vertical / horizontal centre lines).  The 801^2
    reference runs 16 M steps in FP32 (about 17 decay times of its slowest
    mode); the other grids run in FP64 to a steady state."""
    errs = X.cavity_convergence(sides=(13, 19, 25, 31, 37, 49, 61, 85, 97, 121), reference=801,
                                reference_store=lbm.F32, reference_steps=16_000_000)
    ns = sorted(errs)
    x = np.log(np.array(ns, dtype=float))
    for k in X.CONVERGENCE_QUANTITIES:
        slope = -np.polyfit(x, np.log([errs[n][k] for n in ns]), 1)[0]
        print(k, " ".join(f"{errs[n][k]:.3e}" for n in ns), f"slope {slope:.3f}")
        assert 1.8 < slope < 2.7, (k, slope)


TABLE_IV_GRIDS = (101, 201, 401)


@pytest.fixture(scope="module")
def stability_thresholds():
    """Max stable cell Re on the three grids of Table IV for the three models,
    bracketed to a few tenths of a percent (a blow-up within 20 convective
    times counts as unstable)."""
    out = {}
    for n in TABLE_IV_GRIDS:
        for model in (lbm.BGK, lbm.RAWMRT, lbm.CASCADED):
            th, un, _ = X.max_stable_cell_reynolds_refined(model, n)
            out[model, n] = (th, un)
            print(f"{n}^2 {lbm.MODEL_NAMES[model]}: stable up to {th:.2f}, unstable at {un}")
    return out


@pytest.mark.parametrize("n", TABLE_IV_GRIDS)
def test_stability_thresholds_of_table_IV_on_every_grid(stability_thresholds, n):
    """Sec. V, Table IV (14.14-14.25 / 59.40-62.34 / 148.50-199.50 for SRT / raw
    MRT / cascaded on 101^2..401^2): SRT's limit is nearly grid independent near
    14, raw MRT reaches several times SRT and the cascaded model about 2-3 times
    raw MRT on every grid."""
    srt = stability_thresholds[lbm.BGK, n][0]
    mrt = stability_thresholds[lbm.RAWMRT, n][0]
    casc = stability_thresholds[lbm.CASCADED, n][0]
    paper = P.PAPER["max_cell_reynolds"]
    k = paper["grid"].index(n)
    print(f"{n}^2: SRT {srt:.2f} ({paper['srt'][k]}), raw MRT {mrt:.2f} ({paper['raw_mrt'][k]}), "
          f"cascaded {casc:.2f} ({paper['cascaded'][k]})")
    assert abs(srt - paper["srt"][k]) <= 0.06 * paper["srt"][k]
    assert mrt >= 3.0 * srt
    assert casc >= 1.8 * mrt
