"""Python binding of the C ABI in include/lbm.h (ctypes; argument marshalling only).

Every function named ``lbm_*`` here calls the C function of the same name and
raises :class:`LBMError` on a non-zero status.  :class:`Lattice` bundles a
handle with numpy / torch conversions.  All computation happens in the CUDA
library; if it cannot be loaded this module raises instead of computing
anything itself.
"""
from __future__ import annotations

import ctypes as C
import os

import numpy as np

from . import build as _build

LBM_OK, LBM_EINVAL, LBM_ENOMEM, LBM_ECUDA, LBM_EDIVERGED = 0, 1, 2, 3, 4
PERIODIC, BOUNCEBACK, MOVING_WALL = 0, 1, 2
WEST, EAST, SOUTH, NORTH = 0, 1, 2, 3
CASCADED, BGK, RAWMRT = 0, 1, 2
F64, F32, BF16DEV, F16DEV = 0, 1, 2, 3
ROUND_NEAREST, ROUND_STOCHASTIC = 0, 1
NUM_VARIANTS = 4  # kernel variants 0..3 (lbm_set_variant)
STORE_NAMES = {F64: "f64", F32: "f32", BF16DEV: "bf16", F16DEV: "f16"}
MODEL_NAMES = {CASCADED: "cascaded", BGK: "bgk", RAWMRT: "rawmrt"}


class LBMError(RuntimeError):
    def __init__(self, code: int, message: str):
        super().__init__(f"[lbm status {code}] {message}")
        self.code = code


class lbm_bc_t(C.Structure):
    _fields_ = [("edge", C.c_int * 4), ("wall_u", C.c_double * 4)]


class lbm_layout_t(C.Structure):
    _fields_ = [("nx", C.c_int), ("ny", C.c_int), ("pitch", C.c_int), ("store", C.c_int), ("odd", C.c_int),
                ("rho0", C.c_double), ("force", C.c_double * 2), ("bc", lbm_bc_t)]


LBM_NOALLOC_MAX_ROWS = 16384

_lib = None
_vp, _dp, _i, _l, _d = C.c_void_p, C.POINTER(C.c_double), C.c_int, C.c_long, C.c_double

# name -> (restype, argtypes); mirrors include/lbm.h
SIGNATURES = {
    "lbm_create": (_i, [_i, _i, _dp, _dp, C.POINTER(lbm_bc_t), _i, _i, _d, C.POINTER(_vp)]),
    "lbm_destroy": (_i, [_vp]),
    "lbm_set_stream": (_i, [_vp, _vp]),
    "lbm_set_force": (_i, [_vp, _dp]),
    "lbm_set_omegas": (_i, [_vp, _dp]),
    "lbm_set_graph_steps": (_i, [_vp, _i]),
    "lbm_set_variant": (_i, [_vp, _i]),
    "lbm_set_rounding": (_i, [_vp, _i, C.c_ulonglong]),
    "lbm_tune": (_i, [_vp, _i, C.POINTER(C.c_float)]),
    "lbm_set_force_field": (_i, [_vp, _vp, _i]),
    "lbm_init": (_i, [_vp, _vp, _vp]),
    "lbm_init_device": (_i, [_vp, _vp, _vp]),
    "lbm_step": (_i, [_vp, _l]),
    "lbm_macros": (_i, [_vp, _vp, _vp]),
    "lbm_macros_device": (_i, [_vp, _vp, _vp]),
    "lbm_strain": (_i, [_vp, _vp]),
    "lbm_strain_device": (_i, [_vp, _vp]),
    "lbm_get_f": (_i, [_vp, _vp]),
    "lbm_set_f": (_i, [_vp, _vp]),
    "lbm_get_f_device": (_i, [_vp, _vp]),
    "lbm_set_f_device": (_i, [_vp, _vp]),
    "lbm_stats": (_i, [_vp, _dp]),
    "lbm_set_check": (_i, [_vp, _l, _d]),
    "lbm_time": (_l, [_vp]),
    "lbm_info": (_i, [_vp, C.POINTER(C.c_long), C.POINTER(C.c_size_t), C.POINTER(_vp)]),
    "lbm_bytes_per_update": (C.c_size_t, [_i]),
    "lbm_adjoint_run": (_i, [_vp, _l, _l, _vp, _vp, _vp, _dp, _vp, _vp, _dp]),
    "lbm_batch_create": (_i, [C.POINTER(_vp), _i, C.POINTER(_vp)]),
    "lbm_batch_destroy": (_i, [_vp]),
    "lbm_batch_tune": (_i, [_vp, _i, C.POINTER(C.c_float)]),
    "lbm_batch_step": (_i, [_vp, _l]),
    "lbm_batch_set_graph_steps": (_i, [_vp, _i]),
    "lbm_batch_sync": (_i, [_vp]),
    "lbm_batch_set_two_step": (_i, [_vp, _i]),
    "lbm_batch_info": (_i, [_vp, C.POINTER(C.c_int), C.POINTER(_vp)]),
    "lbm_stats_noalloc": (_i, [_vp, C.POINTER(lbm_layout_t), _vp, _vp]),
    "lbm_last_error": (C.c_char_p, []),
    # D3Q27 lattices (include/lbm3d.h)
    "lbm3_create": (_i, [_i, _i, _i, _dp, _dp, _i, _d, C.POINTER(_vp)]),
    "lbm3_destroy": (_i, [_vp]),
    "lbm3_set_stream": (_i, [_vp, _vp]),
    "lbm3_init": (_i, [_vp, _vp, _vp]),
    "lbm3_step": (_i, [_vp, _l]),
    "lbm3_macros": (_i, [_vp, _vp, _vp]),
    "lbm3_get_f": (_i, [_vp, _vp]),
    "lbm3_set_f": (_i, [_vp, _vp]),
    "lbm3_time": (_l, [_vp]),
    "lbm3_info": (_i, [_vp, C.POINTER(C.c_long), C.POINTER(C.c_size_t), C.POINTER(_vp)]),
    "lbm3_bytes_per_update": (C.c_size_t, [_i]),
}


def library_path() -> str:
    return _build.LIB


def load_library(build_if_missing: bool = True):
    """Load liblbm_gb300.so (building it first if asked and needed)."""
    global _lib
    if _lib is None:
        path = _build.build() if build_if_missing else _build.LIB
        if not os.path.exists(path):
            raise RuntimeError(f"CUDA library {path} is missing; run __graft_entry__.build()")
        lib = C.CDLL(path)
        for name, (res, args) in SIGNATURES.items():
            fn = getattr(lib, name)
            fn.restype = res
            fn.argtypes = args
        _lib = lib
    return _lib


def _check(rc: int):
    if rc != LBM_OK:
        raise LBMError(rc, load_library().lbm_last_error().decode())


def _darr(v, n):
    return (C.c_double * n)(*[float(x) for x in v])


def _host(a, shape):
    """float64 C-contiguous numpy view (copy if needed) and its address."""
    a = np.ascontiguousarray(np.asarray(a, dtype=np.float64)).reshape(shape)
    return a, a.ctypes.data


def _dev(t, shape):
    """Device address of a contiguous float64 CUDA tensor of the given shape."""
    import torch

    if not (isinstance(t, torch.Tensor) and t.is_cuda and t.dtype == torch.float64 and t.is_contiguous()):
        raise TypeError("expected a contiguous float64 CUDA tensor")
    if tuple(t.shape) != tuple(shape):
        raise ValueError(f"expected shape {shape}, got {tuple(t.shape)}")
    return t.data_ptr()


# ---------------------------------------------------------------- C-named wrappers

def lbm_create(nx, ny, omegas, force=(0.0, 0.0), edges=(PERIODIC,) * 4, wall_u=(0.0,) * 4,
               model=CASCADED, store=F32, rho0=1.0):
    lib = load_library()
    bc = lbm_bc_t((C.c_int * 4)(*[int(e) for e in edges]), _darr(wall_u, 4))
    h = C.c_void_p()
    _check(lib.lbm_create(int(nx), int(ny), _darr(omegas, 6), _darr(force, 2), C.byref(bc), int(model),
                          int(store), float(rho0), C.byref(h)))
    return h


def lbm_destroy(h):
    _check(load_library().lbm_destroy(h))


def lbm_set_stream(h, stream_ptr: int):
    _check(load_library().lbm_set_stream(h, C.c_void_p(stream_ptr)))


def lbm_set_force(h, force):
    _check(load_library().lbm_set_force(h, _darr(force, 2)))


def lbm_step(h, n: int):
    _check(load_library().lbm_step(h, int(n)))


def lbm_time(h) -> int:
    return int(load_library().lbm_time(h))


def lbm_stats(h):
    out = (C.c_double * 3)()
    _check(load_library().lbm_stats(h, out))
    return np.array(list(out))


def lbm_set_check(h, every: int, mass_rtol: float):
    _check(load_library().lbm_set_check(h, int(every), float(mass_rtol)))


def lbm_info(h):
    dims = (C.c_long * 7)()
    nbytes = C.c_size_t()
    state = C.c_void_p()
    _check(load_library().lbm_info(h, dims, C.byref(nbytes), C.byref(state)))
    return {"nx": dims[0], "ny": dims[1], "pitch": dims[2], "model": dims[3], "store": dims[4],
            "variant": dims[5], "block_x": dims[6], "bytes": nbytes.value, "state": state.value}


def lbm_bytes_per_update(store: int) -> int:
    return int(load_library().lbm_bytes_per_update(int(store)))


def lbm_last_error() -> str:
    return load_library().lbm_last_error().decode()


# ---------------------------------------------------------------- convenience object

class Lattice:
    """A lattice handle.  Host arrays are numpy float64 with the layouts of
    include/lbm.h; the *_device methods take / return float64 CUDA tensors."""

    def __init__(self, nx, ny, omegas, force=(0.0, 0.0), edges=(PERIODIC,) * 4, wall_u=(0.0,) * 4,
                 model=CASCADED, store=F32, rho0=1.0, stream=None):
        self.nx, self.ny, self.model, self.store = int(nx), int(ny), int(model), int(store)
        self.h = lbm_create(nx, ny, omegas, force, edges, wall_u, model, store, rho0)
        self.lib = load_library()
        if stream is not None:
            lbm_set_stream(self.h, stream)

    # lifetime
    def close(self):
        if self.h is not None:
            lbm_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.close()
        return False

    @property
    def shape(self):
        return (self.ny, self.nx)

    @property
    def time(self):
        return lbm_time(self.h)

    def set_stream(self, stream_ptr):
        lbm_set_stream(self.h, stream_ptr)

    def set_force(self, force):
        lbm_set_force(self.h, force)

    def set_omegas(self, omegas):
        _check(self.lib.lbm_set_omegas(self.h, _darr(omegas, 6)))

    def set_graph_steps(self, steps):
        _check(self.lib.lbm_set_graph_steps(self.h, int(steps)))
        return self

    def set_variant(self, variant):
        _check(self.lib.lbm_set_variant(self.h, int(variant)))
        return self

    def set_rounding(self, mode, seed=0):
        """ROUND_NEAREST or ROUND_STOCHASTIC (16-bit or FP32 storage) with a seed."""
        _check(self.lib.lbm_set_rounding(self.h, int(mode), int(seed) & (2 ** 64 - 1)))
        return self

    def tune(self, trial_steps=20):
        """Time the kernel variants and CTA shapes, keep the fastest; returns the
        best ms per step of variants 0..3 (0.0 where the storage has no such variant)."""
        ms = (C.c_float * NUM_VARIANTS)()
        _check(self.lib.lbm_tune(self.h, int(trial_steps), ms))
        return tuple(ms)

    def set_force_field(self, fxy):
        if fxy is None:
            _check(self.lib.lbm_set_force_field(self.h, None, 0))
            return
        try:
            import torch

            if isinstance(fxy, torch.Tensor):
                _check(self.lib.lbm_set_force_field(self.h, _dev(fxy, (2,) + self.shape), 1))
                return
        except ImportError:
            pass
        a, p = _host(fxy, (2,) + self.shape)
        _check(self.lib.lbm_set_force_field(self.h, p, 0))

    def init(self, rho=None, u=None):
        ra = ua = None
        rp = up = None
        if rho is not None:
            ra, rp = _host(rho, self.shape)
        if u is not None:
            ua, up = _host(u, (2,) + self.shape)
        _check(self.lib.lbm_init(self.h, rp, up))
        return self

    def init_device(self, rho=None, u=None):
        rp = _dev(rho, self.shape) if rho is not None else None
        up = _dev(u, (2,) + self.shape) if u is not None else None
        _check(self.lib.lbm_init_device(self.h, rp, up))
        return self

    def step(self, n=1):
        lbm_step(self.h, n)
        return self

    def macros(self):
        rho = np.empty(self.shape)
        u = np.empty((2,) + self.shape)
        _check(self.lib.lbm_macros(self.h, rho.ctypes.data, u.ctypes.data))
        return rho, u

    def macros_device(self, rho=None, u=None):
        import torch

        rho = torch.empty(self.shape, dtype=torch.float64, device="cuda") if rho is None else rho
        u = torch.empty((2,) + self.shape, dtype=torch.float64, device="cuda") if u is None else u
        _check(self.lib.lbm_macros_device(self.h, _dev(rho, self.shape), _dev(u, (2,) + self.shape)))
        return rho, u

    def strain(self):
        out = np.empty((3,) + self.shape)
        _check(self.lib.lbm_strain(self.h, out.ctypes.data))
        return out

    def get_f(self):
        f = np.empty((9,) + self.shape)
        _check(self.lib.lbm_get_f(self.h, f.ctypes.data))
        return f

    def set_f(self, f):
        a, p = _host(f, (9,) + self.shape)
        _check(self.lib.lbm_set_f(self.h, p))
        return self

    def get_f_device(self, out=None):
        import torch

        out = torch.empty((9,) + self.shape, dtype=torch.float64, device="cuda") if out is None else out
        _check(self.lib.lbm_get_f_device(self.h, _dev(out, (9,) + self.shape)))
        return out

    def set_f_device(self, f):
        _check(self.lib.lbm_set_f_device(self.h, _dev(f, (9,) + self.shape)))
        return self

    def stats(self):
        return lbm_stats(self.h)

    def set_check(self, every, mass_rtol=1e-6):
        lbm_set_check(self.h, every, mass_rtol)

    def info(self):
        return lbm_info(self.h)

    def adjoint_run(self, nsteps, every, u0, u_target, rho=None, want_u0=True, want_force=True):
        """lbm_adjoint_run with float64 CUDA tensors; returns (loss, grad_u0, grad_force, grad_omega[6])."""
        import torch

        shape2 = (2,) + self.shape
        gu = torch.empty(shape2, dtype=torch.float64, device="cuda") if want_u0 else None
        gf = torch.empty(shape2, dtype=torch.float64, device="cuda") if want_force else None
        loss = C.c_double()
        gom = (C.c_double * 6)()
        _check(self.lib.lbm_adjoint_run(
            self.h, int(nsteps), int(every), _dev(rho, self.shape) if rho is not None else None,
            _dev(u0, shape2), _dev(u_target, shape2), C.byref(loss),
            gu.data_ptr() if gu is not None else None, gf.data_ptr() if gf is not None else None, gom))
        return loss.value, gu, gf, np.array(list(gom))


class Batch:
    """Many lattices advanced together (lbm_batch_*): one launch per step over
    all their tiles, or one launch per two steps (set_two_step; the tuner may
    choose either)."""

    POLICIES = {0: "round_robin", 1: "chunked", 2: "dynamic", 3: "one_cta_per_tile", 4: "two_steps_per_launch"}
    ORDERS = {0: "largest_first", 1: "interleaved"}

    def __init__(self, lattices):
        self.lib = load_library()
        self.lattices = list(lattices)  # keep the handles alive
        arr = (C.c_void_p * len(self.lattices))(*[L.h.value if isinstance(L.h, C.c_void_p) else L.h
                                                   for L in self.lattices])
        self.b = C.c_void_p()
        _check(self.lib.lbm_batch_create(arr, len(self.lattices), C.byref(self.b)))

    def close(self):
        if self.b is not None:
            _check(self.lib.lbm_batch_destroy(self.b))
            self.b = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.close()
        return False

    def tune(self, trial_steps=5):
        ms = C.c_float()
        _check(self.lib.lbm_batch_tune(self.b, int(trial_steps), C.byref(ms)))
        return ms.value

    def step(self, n=1):
        _check(self.lib.lbm_batch_step(self.b, int(n)))
        return self

    def set_graph_steps(self, steps):
        _check(self.lib.lbm_batch_set_graph_steps(self.b, int(steps)))

    def set_two_step(self, on=True):
        """Two steps per launch for the whole batch (lbm_batch_set_two_step)."""
        _check(self.lib.lbm_batch_set_two_step(self.b, 1 if on else 0))
        return self

    def sync(self):
        _check(self.lib.lbm_batch_sync(self.b))

    def info(self):
        cfg = (C.c_int * 6)()
        st = C.c_void_p()
        _check(self.lib.lbm_batch_info(self.b, cfg, C.byref(st)))
        return {"tile": (cfg[0], cfg[1]), "policy": self.POLICIES[cfg[2]], "order": self.ORDERS[cfg[3]],
                "grid": cfg[4], "tiles": cfg[5], "stream": st.value or 0}


class Lattice3:
    """A periodic D3Q27 central-moment lattice (lbm3_* of include/lbm3d.h).
    omegas = (omega_bulk, omega_shear, omega_3, omega_4, omega_5, omega_6);
    store = F64, F32, BF16DEV or F16DEV; host arrays are numpy float64:
    rho [nz, ny, nx], u [3, nz, ny, nx], f [27, nz, ny, nx]."""

    def __init__(self, nx, ny, nz, omegas, force=(0.0, 0.0, 0.0), store=F32, rho0=1.0, stream=None):
        self.lib = load_library()
        self.shape = (int(nz), int(ny), int(nx))
        self.store = int(store)
        h = C.c_void_p()
        _check(self.lib.lbm3_create(int(nx), int(ny), int(nz), _darr(omegas, 6), _darr(force, 3), int(store),
                                    float(rho0), C.byref(h)))
        self.h = h
        if stream is not None:
            _check(self.lib.lbm3_set_stream(self.h, C.c_void_p(stream)))

    def close(self):
        if self.h is not None:
            _check(self.lib.lbm3_destroy(self.h))
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.close()
        return False

    @property
    def time(self):
        return int(self.lib.lbm3_time(self.h))

    def init(self, rho=None, u=None):
        rp = up = None
        if rho is not None:
            ra, rp = _host(rho, self.shape)
        if u is not None:
            ua, up = _host(u, (3,) + self.shape)
        _check(self.lib.lbm3_init(self.h, rp, up))
        return self

    def step(self, n=1):
        _check(self.lib.lbm3_step(self.h, int(n)))
        return self

    def macros(self):
        rho = np.empty(self.shape)
        u = np.empty((3,) + self.shape)
        _check(self.lib.lbm3_macros(self.h, rho.ctypes.data, u.ctypes.data))
        return rho, u

    def get_f(self):
        f = np.empty((27,) + self.shape)
        _check(self.lib.lbm3_get_f(self.h, f.ctypes.data))
        return f

    def set_f(self, f):
        a, p = _host(f, (27,) + self.shape)
        _check(self.lib.lbm3_set_f(self.h, p))
        return self

    def info(self):
        dims = (C.c_long * 5)()
        nbytes = C.c_size_t()
        state = C.c_void_p()
        _check(self.lib.lbm3_info(self.h, dims, C.byref(nbytes), C.byref(state)))
        return {"nx": dims[0], "ny": dims[1], "nz": dims[2], "pitch": dims[3], "store": dims[4],
                "bytes": nbytes.value, "state": state.value}
