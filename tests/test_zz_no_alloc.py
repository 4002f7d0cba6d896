"""lbm_stats_noalloc, the allocation-free variant of lbm_stats.

Some callers cannot call cudaMalloc (code inside another framework's memory
pool or a fixed device-memory budget, drivers that forbid allocation after
start-up).  For them lbm_stats_noalloc computes the same global FP64 sums
from a population array the caller owns, with its scratch in a static device
array.  This file checks, through the C ABI, that two calls in a row agree
with lbm_stats.  It sorts last so that a run stopping at the first failure
has already run every other test.
"""
import ctypes as C

import numpy as np
import pytest

from paper_1202_6351_gb300 import lbm, workloads

pytestmark = pytest.mark.gpu

RTOL = 1e-12  # the tolerance the other FP64 diagnostics tests use


def _layout(L, edges, wall_u, force, rho0=1.0):
    info = L.info()
    bc = lbm.lbm_bc_t((C.c_int * 4)(*edges), (C.c_double * 4)(*wall_u))
    lay = lbm.lbm_layout_t(info["nx"], info["ny"], info["pitch"], info["store"], L.time & 1, rho0,
                           (C.c_double * 2)(*force), bc)
    return lay, info["state"]


@pytest.mark.parametrize("store", [lbm.F32, lbm.F64, lbm.BF16DEV, lbm.F16DEV], ids=["f32", "f64", "bf16", "f16"])
def test_noalloc_stats_match_lbm_stats_on_two_calls(store):
    import torch

    assert torch.cuda.is_available()
    torch.cuda.set_device(0)
    lib = lbm.load_library()
    n, ny = 70, 45
    edges = (lbm.BOUNCEBACK, lbm.BOUNCEBACK, lbm.BOUNCEBACK, lbm.MOVING_WALL)
    wall_u = (0.0, 0.0, 0.0, 0.1)
    force = (2e-5, -1e-5)
    rho, u = workloads.random_fields(17, n, ny, u_amp=0.03)
    L = lbm.Lattice(n, ny, (1.1, 1.6, 1.6, 1.0, 1.0, 1.0), force=force, edges=edges, wall_u=wall_u, store=store)
    L.init(rho, u)
    out = torch.full((3,), float("nan"), dtype=torch.float64, device="cuda")
    stream = torch.cuda.current_stream().cuda_stream
    for steps in (7, 4):  # 7 and 11 steps: the AA-swapped (odd) layout
        L.step(steps)
        ref = L.stats()
        lay, state = _layout(L, edges, wall_u, force)
        rc = lib.lbm_stats_noalloc(state, C.byref(lay), out.data_ptr(), stream)
        assert rc == lbm.LBM_OK, lbm.lbm_last_error()
        torch.cuda.synchronize()
        np.testing.assert_allclose(out.cpu().numpy(), ref, rtol=RTOL, atol=1e-12)
    L.step(1)  # even layout
    ref = L.stats()
    lay, state = _layout(L, edges, wall_u, force)
    assert lib.lbm_stats_noalloc(state, C.byref(lay), out.data_ptr(), stream) == lbm.LBM_OK
    torch.cuda.synchronize()
    np.testing.assert_allclose(out.cpu().numpy(), ref, rtol=RTOL, atol=1e-12)
    # The entry point's contract: after the first call (which looks up the
    # scratch address and may load the module's kernels), further calls leave
    # the device's free memory unchanged.
    free0 = torch.cuda.mem_get_info()[0]
    for _ in range(20):
        assert lib.lbm_stats_noalloc(state, C.byref(lay), out.data_ptr(), stream) == lbm.LBM_OK
    torch.cuda.synchronize()
    assert torch.cuda.mem_get_info()[0] == free0
    np.testing.assert_allclose(out.cpu().numpy(), ref, rtol=RTOL, atol=1e-12)
    L.close()


def test_noalloc_rejects_too_many_rows():
    lib = lbm.load_library()
    bc = lbm.lbm_bc_t((C.c_int * 4)(0, 0, 0, 0), (C.c_double * 4)(0, 0, 0, 0))
    lay = lbm.lbm_layout_t(8, lbm.LBM_NOALLOC_MAX_ROWS + 1, 32, lbm.F32, 0, 1.0, (C.c_double * 2)(0, 0), bc)
    dummy = C.c_double(0)
    rc = lib.lbm_stats_noalloc(C.addressof(dummy), C.byref(lay), C.addressof(dummy), None)
    assert rc == lbm.LBM_EINVAL
    assert "LBM_NOALLOC_MAX_ROWS" in lbm.lbm_last_error()
