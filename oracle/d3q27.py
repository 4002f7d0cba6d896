"""FP64 CPU oracle of the central-moment LBM on the D3Q27 lattice (ctypes
binding of lbm3d_oracle.c).

TEST INFRASTRUCTURE ONLY: only ``tests/``, ``__graft_entry__.smoke()`` and
``bench.py``'s CPU legs may import it; it shares no code with the CUDA path.
The paper defines the method for D2Q9 (Sec. II) and names 3-D lattices as
future work; lbm3d_oracle.h states how the method is carried to D3Q27.
Arrays are float64 with the layouts f[27, nz, ny, nx], u[3, nz, ny, nx].
"""
from __future__ import annotations

import ctypes as C
import math

import numpy as np

from . import build as _build

_lib = None


class _Lat3(C.Structure):
    _fields_ = [("nx", C.c_int), ("ny", C.c_int), ("nz", C.c_int), ("omega", C.c_double * 6),
                ("force", C.c_double * 3)]


def _load(path):
    L = C.CDLL(path)
    vp = C.c_void_p
    for name, argc in [("oracle3_velocities", 2), ("oracle3_central_moments", 3),
                       ("oracle3_from_central_moments", 3), ("oracle3_collide", 4), ("oracle3_source", 3),
                       ("oracle3_init", 4), ("oracle3_collide_all", 3), ("oracle3_stream_all", 3),
                       ("oracle3_macros", 4)]:
        fn = getattr(L, name)
        fn.argtypes = [vp] * argc
        fn.restype = None
    L.oracle3_macros_node.argtypes = [vp, vp, vp, vp]
    L.oracle3_macros_node.restype = None
    L.oracle3_equilibrium.argtypes = [C.c_double, vp, vp]
    L.oracle3_equilibrium.restype = None
    L.oracle3_run.argtypes = [vp, vp, vp, C.c_long]
    L.oracle3_run.restype = None
    return L


class substituted_library:
    """Context manager that routes this module's calls through another build
    of the D3Q27 oracle source (used to plant mistakes in tests)."""

    def __init__(self, path):
        self.path = path

    def __enter__(self):
        global _lib
        self.saved = _lib
        _lib = _load(self.path)
        return self

    def __exit__(self, *exc):
        global _lib
        _lib = self.saved
        return False


def lib():
    global _lib
    if _lib is None:
        _lib = _load(_build.build()["d3q27"])
    return _lib


def _p(a):
    return a.ctypes.data_as(C.c_void_p)


def _v(x, n):
    return np.ascontiguousarray(np.asarray(x, dtype=np.float64).reshape(n))


def velocities():
    """(e[27, 3] int, w[27]) in the oracle's direction order."""
    e = np.zeros((27, 3), dtype=np.int32)
    w = np.zeros(27)
    lib().oracle3_velocities(_p(e), _p(w))
    return e.astype(int), w


def collide_node(fb, force=(0.0, 0.0, 0.0), omegas=(1.0,) * 6):
    out = np.empty(27)
    lib().oracle3_collide(_p(_v(fb, 27)), _p(_v(force, 3)), _p(_v(omegas, 6)), _p(out))
    return out


def macros_node(fb, force=(0.0, 0.0, 0.0)):
    r = np.zeros(1)
    u = np.zeros(3)
    lib().oracle3_macros_node(_p(_v(fb, 27)), _p(_v(force, 3)), _p(r), _p(u))
    return float(r[0]), u


def equilibrium_node(rho, u):
    out = np.empty(27)
    lib().oracle3_equilibrium(float(rho), _p(_v(u, 3)), _p(out))
    return out


def source_node(u, force):
    out = np.empty(27)
    lib().oracle3_source(_p(_v(u, 3)), _p(_v(force, 3)), _p(out))
    return out


class Lattice3:
    """A periodic D3Q27 lattice advanced by the oracle; omegas = (omega_bulk,
    omega_shear, omega_3, omega_4, omega_5, omega_6)."""

    def __init__(self, nx, ny, nz, omegas, force=(0.0, 0.0, 0.0)):
        self.shape = (int(nz), int(ny), int(nx))
        self.s = _Lat3(int(nx), int(ny), int(nz), (C.c_double * 6)(*[float(o) for o in omegas]),
                       (C.c_double * 3)(*[float(v) for v in force]))
        self.f = np.zeros((27,) + self.shape)
        self._work = np.zeros_like(self.f)

    def init(self, rho=None, u=None):
        rho = np.ones(self.shape) if rho is None else rho
        u = np.zeros((3,) + self.shape) if u is None else u
        rho = np.ascontiguousarray(np.asarray(rho, dtype=np.float64).reshape(self.shape))
        u = np.ascontiguousarray(np.asarray(u, dtype=np.float64).reshape((3,) + self.shape))
        lib().oracle3_init(C.byref(self.s), _p(rho), _p(u), _p(self.f))
        return self

    def set_f(self, f):
        self.f[...] = np.asarray(f, dtype=np.float64).reshape(self.f.shape)
        return self

    def run(self, nsteps):
        lib().oracle3_run(C.byref(self.s), _p(self.f), _p(self._work), C.c_long(int(nsteps)))
        return self

    def collide(self):
        post = np.empty_like(self.f)
        lib().oracle3_collide_all(C.byref(self.s), _p(self.f), _p(post))
        return post

    def stream(self, post):
        post = np.ascontiguousarray(np.asarray(post, dtype=np.float64).reshape(self.f.shape))
        lib().oracle3_stream_all(C.byref(self.s), _p(post), _p(self.f))
        return self

    def macros(self):
        rho = np.empty(self.shape)
        u = np.empty((3,) + self.shape)
        lib().oracle3_macros(C.byref(self.s), _p(self.f), _p(rho), _p(u))
        return rho, u


def nu_from_omega(omega):
    """Shear viscosity (1/omega - 1/2) c_s^2, c_s^2 = 1/3."""
    return (1.0 / omega - 0.5) / 3.0


def shear_wave(n, u0, nu, t, k_index=1, axis_flow=0, axis_var=2, advect=(0.0, 0.0, 0.0)):
    """Decaying shear wave u_flow = u0 sin(k x_var) exp(-nu k^2 t) on an n^3
    periodic lattice (the exact linear solution; advected by a uniform
    velocity `advect` whose component along x_var shifts the phase).
    Returns u[3, n, n, n] (layout [3][z][y][x])."""
    k = 2.0 * math.pi * k_index / n
    c = np.arange(n, dtype=np.float64)
    Z, Y, X = np.meshgrid(c, c, c, indexing="ij")
    coord = (X, Y, Z)[axis_var] - advect[axis_var] * t
    u = np.zeros((3, n, n, n))
    for d in range(3):
        u[d] += advect[d]
    u[axis_flow] += u0 * np.sin(k * coord) * math.exp(-nu * k * k * t)
    return u
