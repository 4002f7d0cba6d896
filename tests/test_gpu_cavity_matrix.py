"""The lid-driven cavity configuration on the CUDA path: Re 1000, 3200 and 5000
on a 257^2 grid, the cascaded, SRT-BGK and raw-moment MRT collisions side by
side, each in FP32 storage (run to max |du| < 1e-7 per 1000 steps) and in FP16
storage with both rounding modes (the same number of steps).  Context pins are
the paper's printed numbers (Sec. IV-C Tables I and II at 401^2, Sec. V Table
IV); the FP16 results are stated against the FP32 ones."""
import math

import pytest

from paper_1202_6351_gb300 import experiments as X
from paper_1202_6351_gb300 import lbm
from tests import _pins as P

pytestmark = pytest.mark.gpu

N = 257
RES = (1000.0, 3200.0, 5000.0)


@pytest.fixture(scope="module")
def matrix():
    import torch

    assert torch.cuda.is_available(), "GPU tests need a CUDA device"
    torch.cuda.set_device(0)

    def report(key, r):
        row = X.matrix_summary({key: r})
        print(row, flush=True)

    # SRT at Re 3200 (cell Re 12.5, near its limit of 14.1) keeps a slowly
    # decaying oscillation (max |du| per 1000 steps about 1e-6 at 3e6 steps and
    # 2e-7 at 2e7), so the matrix stops at 3e6 steps; the other cases are
    # steady by 1.4e6.
    return X.cavity_matrix(N, RES, max_steps=3_000_000, progress=report)


def _close(p, q, tol):
    return abs(p[0] - q[0]) < tol and abs(p[1] - q[1]) < tol


@pytest.mark.parametrize("re", RES)
def test_cascaded_and_raw_mrt_vortex_centres_match_table_I(matrix, re):
    """Table I: the primary vortex of the cascaded model at 401^2; here 257^2 in
    FP32 storage, steady state.  Raw MRT lands on the same centre (the paper:
    within 0.014 %)."""
    table = P.PAPER["primary_vortex"]
    px, py = table["cascaded"][table["re"].index(int(re))]
    casc = matrix[lbm.CASCADED, re]
    mrt = matrix[lbm.RAWMRT, re]
    assert casc["status"] == "steady" and mrt["status"] == "steady"
    c, m = casc["f32"]["centre"], mrt["f32"]["centre"]
    print(f"Re {re:.0f}: cascaded {c}, raw MRT {m}, paper ({px}, {py}); steps {casc['steps']}, {mrt['steps']}")
    assert _close(c, (px, py), 0.01)
    assert _close(m, c, 2e-3)


@pytest.mark.parametrize("re", RES)
def test_secondary_vortices_of_table_II(matrix, re):
    """Table II: the bottom corner vortices at every Re; the top-left one appears
    at Re 3200 and 5000 and not at Re 1000."""
    sec = P.PAPER["secondary_vortices"]["cascaded"][str(int(re))]
    for model in (lbm.CASCADED, lbm.RAWMRT):
        got = matrix[model, re]["f32"]["secondary"]
        print(lbm.MODEL_NAMES[model], re, got, sec)
        for region in ("bottom_left", "bottom_right"):
            assert got[region] is not None and _close(got[region], sec[region], 0.015), (region, got[region])
        if re >= 3200:
            assert got["top_left"] is not None and _close(got["top_left"], sec["top"], 0.015), got["top_left"]
        else:
            assert got["top_left"] is None


def test_srt_diverges_where_table_IV_says(matrix):
    """Table IV: SRT is stable up to a cell Reynolds number of about 14.1; at
    257^2 Re 5000 has U dx / nu = 19.5 and diverges, Re 1000 (3.9) reaches a
    steady state and Re 3200 (12.5) stays bounded, with a slowly decaying
    residual oscillation (max |du| per 1000 steps about 1e-6 after 3e6 steps,
    2e-7 after 2e7) and the vortex of the other two models.  The
    cascaded and raw-MRT models reach a steady state at all three."""
    assert matrix[lbm.BGK, 5000.0]["status"] == "diverged"
    assert matrix[lbm.BGK, 1000.0]["status"] == "steady"
    srt = matrix[lbm.BGK, 3200.0]
    assert srt["status"] in ("steady", "unsteady") and srt["f32"]["max_du"] < 5e-6
    assert _close(srt["f32"]["centre"], matrix[lbm.CASCADED, 3200.0]["f32"]["centre"], 2e-3)
    for model in (lbm.CASCADED, lbm.RAWMRT):
        for re in RES:
            assert matrix[model, re]["status"] == "steady"


def test_srt_divergence_is_reported_by_the_divergence_check():
    """The same SRT case run alone with lbm_set_check: lbm_step returns
    LBM_EDIVERGED and the lattice stays usable."""
    import numpy as np

    om = X.cavity_omega(N, 5000.0)
    with lbm.Lattice(N, N, (1.0, om, om, 1.0, 1.0, 1.0), edges=X.CAVITY_EDGES, wall_u=(0, 0, 0, 0.1),
                     model=lbm.BGK) as L:
        L.init()
        L.set_check(1000, 1e-3)
        with pytest.raises(lbm.LBMError) as ei:
            L.step(2_000_000)
        assert ei.value.code == lbm.LBM_EDIVERGED
        L.init()
        L.set_check(0, 1e-3)
        L.step(10)
        _, u = L.macros()
        assert np.isfinite(u).all()


# FP16 storage against FP32 on the steady cavity (stated bounds with margin over
# what was measured on one GB300: round to nearest 0.3-8 % in relative L2 and
# primary-vortex shifts up to 0.014; stochastic rounding 0.06-0.18 % and up to
# 0.004).  Round to nearest drops every per-step change below half an FP16
# spacing and settles on a visibly different flow; stochastic rounding keeps the
# steady flow to about 1e-3.
F16_BOUNDS = {"f16_nearest": (0.12, 0.025), "f16_stochastic": (3e-3, 6e-3)}


@pytest.mark.parametrize("re", RES)
def test_fp16_storage_against_fp32_on_the_steady_cavity(matrix, re):
    for model in (lbm.CASCADED, lbm.RAWMRT) + ((lbm.BGK,) if re < 3200 else ()):
        r = matrix[model, re]
        for name, (l2_bound, shift_bound) in F16_BOUNDS.items():
            e = r[name]
            print(f"{lbm.MODEL_NAMES[model]} Re {re:.0f} {name}: rel L2 vs FP32 {e['rel_l2_vs_f32']:.3e}, "
                  f"centre shift {e['centre_shift']:.2e}, max du per 1000 steps {e['max_du']:.2e}")
            assert e["rel_l2_vs_f32"] < l2_bound and e["centre_shift"] < shift_bound
            assert math.isfinite(e["max_du"])
        # stochastic rounding is the accurate 16-bit mode on this flow
        assert r["f16_stochastic"]["rel_l2_vs_f32"] < r["f16_nearest"]["rel_l2_vs_f32"]
