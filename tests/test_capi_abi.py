"""The C ABI without a GPU: the library builds, loads, exports every symbol that
include/lbm.h and include/lbm3d.h declare, and its host-side argument checks
answer correctly.
No kernel is launched here."""
import ctypes as C
import os
import re

import pytest

from paper_1202_6351_gb300 import lbm

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def declared_functions():
    names = set()
    for hdr in os.listdir(os.path.join(ROOT, "include")):
        if not hdr.endswith(".h"):
            continue
        text = open(os.path.join(ROOT, "include", hdr)).read()
        text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
        for m in re.finditer(r"^[A-Za-z_][\w \*]*?\b(lbm3?_\w+)\s*\(", text, flags=re.M):
            names.add(m.group(1))
    return sorted(names)


def test_header_declares_the_boundary():
    names = declared_functions()
    for required in ("lbm_create", "lbm_step", "lbm_macros", "lbm_destroy"):
        assert required in names


def test_library_exports_every_declared_symbol():
    lib = lbm.load_library()
    missing = [n for n in declared_functions() if not hasattr(lib, n)]
    assert not missing, missing


def test_binding_covers_every_declared_symbol():
    assert set(declared_functions()) <= set(lbm.SIGNATURES)


def test_library_is_built_for_sm103a_only():
    from paper_1202_6351_gb300 import build as B

    assert B.ARCH == ["-gencode", "arch=compute_103a,code=sm_103a"]
    assert os.path.exists(lbm.library_path())


def test_bytes_per_update():
    assert [lbm.lbm_bytes_per_update(s) for s in (lbm.F64, lbm.F32, lbm.BF16DEV, lbm.F16DEV)] == [144, 72, 36, 36]
    assert lbm.lbm_bytes_per_update(99) == 0


BAD_CREATE = [
    dict(nx=0, ny=4),
    dict(nx=4, ny=-1),
    dict(nx=70000, ny=70000),
    dict(omegas=(1.0, 2.0, 1.0, 1.0, 1.0, 1.0)),
    dict(omegas=(0.0, 1.0, 1.0, 1.0, 1.0, 1.0)),
    dict(model=7),
    dict(store=9),
    dict(rho0=0.0),
    dict(edges=(lbm.PERIODIC, lbm.BOUNCEBACK, lbm.PERIODIC, lbm.PERIODIC)),
    dict(edges=(lbm.PERIODIC, lbm.PERIODIC, lbm.MOVING_WALL, lbm.PERIODIC)),
    dict(edges=(5, 5, 0, 0)),
    dict(force=(float("nan"), 0.0)),
    # size limits, one past each: ny <= 65535 (grid y dimension), and the row
    # pitch (nx rounded up to 32) times ny within 2^31 - 1 (32-bit plane offsets)
    dict(nx=8, ny=65536),
    dict(nx=2147483, ny=1000),
    dict(rho0=float("inf")),
    dict(edges=(lbm.PERIODIC, lbm.PERIODIC, lbm.BOUNCEBACK, lbm.MOVING_WALL), wall_u=(0, 0, 0, float("inf"))),
]


@pytest.mark.parametrize("kw", BAD_CREATE)
def test_create_rejects_bad_arguments_before_touching_the_device(kw):
    args = dict(nx=8, ny=8, omegas=(1.0,) * 6)
    args.update(kw)
    with pytest.raises(lbm.LBMError) as ei:
        lbm.lbm_create(**args)
    assert ei.value.code == lbm.LBM_EINVAL
    assert lbm.lbm_last_error()


def test_largest_lattice_passes_the_argument_checks():
    """32768 x 65535 (pitch 32768, 2^31 - 2^15 nodes per plane) is within every
    size limit, so without a GPU lbm_create gets as far as looking for a device."""
    import torch
    if torch.cuda.is_available():
        pytest.skip("would allocate the lattice")
    with pytest.raises(lbm.LBMError) as ei:
        lbm.lbm_create(32768, 65535, (1.0,) * 6, store=lbm.F16DEV)
    assert ei.value.code == lbm.LBM_ECUDA


def _noalloc_layout(nx=8, ny=8, pitch=32, store=lbm.F32, rho0=1.0, edges=(0, 0, 0, 0)):
    bc = lbm.lbm_bc_t((C.c_int * 4)(*edges), (C.c_double * 4)(0, 0, 0, 0))
    return lbm.lbm_layout_t(nx, ny, pitch, store, 0, rho0, (C.c_double * 2)(0, 0), bc)


BAD_NOALLOC = [
    dict(nx=0), dict(ny=0), dict(ny=lbm.LBM_NOALLOC_MAX_ROWS + 1), dict(pitch=7),
    dict(nx=131072, pitch=131072, ny=16384), dict(store=9), dict(rho0=0.0), dict(edges=(0, 0, 3, 0)),
    dict(edges=(0, 1, 0, 0)), dict(edges=(0, 0, 2, 0)),  # one edge of an opposite pair periodic, the other a wall
]


@pytest.mark.parametrize("kw", BAD_NOALLOC)
def test_noalloc_rejects_bad_layouts_before_touching_the_device(kw):
    """lbm_stats_noalloc checks the caller's layout before any CUDA call, so a
    rejected layout never reaches the (here dummy) buffers."""
    lib = lbm.load_library()
    dummy = C.c_double(0)
    lay = _noalloc_layout(**kw)
    rc = lib.lbm_stats_noalloc(C.addressof(dummy), C.byref(lay), C.addressof(dummy), None)
    assert rc == lbm.LBM_EINVAL
    assert lbm.lbm_last_error().startswith("lbm_stats_noalloc")
    for f, lp, out in ((None, C.byref(lay), C.addressof(dummy)), (C.addressof(dummy), None, C.addressof(dummy)),
                       (C.addressof(dummy), C.byref(_noalloc_layout()), None)):
        assert lib.lbm_stats_noalloc(f, lp, out, None) == lbm.LBM_EINVAL


def test_null_handles():
    lib = lbm.load_library()
    assert lib.lbm_destroy(None) == lbm.LBM_OK
    assert lib.lbm_step(None, 1) == lbm.LBM_EINVAL
    assert lib.lbm_macros(None, None, None) == lbm.LBM_EINVAL
    assert lib.lbm_time(None) == -1
    out = (C.c_double * 3)()
    assert lib.lbm_stats(None, out) == lbm.LBM_EINVAL


def test_null_handles_of_the_tuning_rounding_batch_and_adjoint_calls():
    """Every entry point answers a NULL handle with LBM_EINVAL before touching
    the device (here there is none: a CUDA call would give LBM_ECUDA)."""
    lib = lbm.load_library()
    ms = (C.c_float * 3)()
    assert lib.lbm_set_variant(None, 0) == lbm.LBM_EINVAL
    assert lib.lbm_set_rounding(None, lbm.ROUND_STOCHASTIC, 1) == lbm.LBM_EINVAL
    assert lib.lbm_tune(None, 4, ms) == lbm.LBM_EINVAL
    assert lib.lbm_set_graph_steps(None, 8) == lbm.LBM_EINVAL
    assert lib.lbm_set_check(None, 10, 1e-3) == lbm.LBM_EINVAL
    assert lib.lbm_adjoint_run(None, 10, 5, None, None, None, None, None, None, None) == lbm.LBM_EINVAL
    assert lib.lbm_batch_destroy(None) == lbm.LBM_OK
    assert lib.lbm_batch_step(None, 1) == lbm.LBM_EINVAL
    assert lib.lbm_batch_tune(None, 1, None) == lbm.LBM_EINVAL
    assert lib.lbm_batch_sync(None) == lbm.LBM_EINVAL
    assert lib.lbm_batch_set_graph_steps(None, 8) == lbm.LBM_EINVAL
    assert lib.lbm_batch_info(None, None, None) == lbm.LBM_EINVAL
    out = C.c_void_p()
    assert lib.lbm_batch_create(None, 0, C.byref(out)) == lbm.LBM_EINVAL
    assert lbm.lbm_last_error()



BAD_CREATE3 = [
    dict(nx=0), dict(nz=0), dict(nz=70000), dict(nx=2048, ny=2048, nz=1024),
    dict(omegas=(1.0, 2.0, 1.0, 1.0, 1.0, 1.0)), dict(store=7), dict(rho0=-1.0),
    dict(force=(float("nan"), 0.0, 0.0)),
]


@pytest.mark.parametrize("kw", BAD_CREATE3)
def test_d3q27_create_rejects_bad_arguments_before_touching_the_device(kw):
    lib = lbm.load_library()
    args = dict(nx=4, ny=4, nz=4, omegas=(1.0,) * 6, force=(0.0, 0.0, 0.0), store=lbm.F32, rho0=1.0)
    args.update(kw)
    h = C.c_void_p()
    rc = lib.lbm3_create(args["nx"], args["ny"], args["nz"], (C.c_double * 6)(*args["omegas"]),
                         (C.c_double * 3)(*args["force"]), args["store"], args["rho0"], C.byref(h))
    assert rc == lbm.LBM_EINVAL
    assert lbm.lbm_last_error().startswith("lbm3_create")


def test_d3q27_null_handles():
    lib = lbm.load_library()
    assert lib.lbm3_destroy(None) == lbm.LBM_OK
    assert lib.lbm3_step(None, 1) == lbm.LBM_EINVAL
    assert lib.lbm3_macros(None, None, None) == lbm.LBM_EINVAL
    assert lib.lbm3_time(None) == -1
    assert lib.lbm3_bytes_per_update(lbm.F32) == 216 and lib.lbm3_bytes_per_update(lbm.F64) == 432
    assert lib.lbm3_bytes_per_update(lbm.F16DEV) == 108 and lib.lbm3_bytes_per_update(lbm.BF16DEV) == 108
    assert lib.lbm3_bytes_per_update(7) == 0
