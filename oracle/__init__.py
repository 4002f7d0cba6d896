"""FP64 CPU oracle of the cascaded central-moment LBM (D2Q9), Sec. II of the paper.

TEST INFRASTRUCTURE ONLY.  The CUDA library is checked against this package;
only ``tests/``, ``__graft_entry__.smoke()`` and ``bench.py``'s cpu_baseline /
reference leg may import it.  It shares no code with the CUDA path and never
loads the CUDA library.

The arithmetic lives in ``lbm_oracle.c`` (plain C, FP64, one node at a time,
collide-all then stream-all in push form).  This module only marshals numpy
arrays through ctypes, and adds the closed-form solutions the paper compares
against (Sec. III): the Poiseuille parabola and the decaying Taylor-Green
vortex.  Arrays are float64 (complex128 for the complex-step build) with the
layout f[9, ny, nx].
"""
from __future__ import annotations

import ctypes as C
import math

import numpy as np

from . import build as _build

CASCADED, BGK, RAWMRT = 0, 1, 2
PERIODIC, BOUNCEBACK, MOVING_WALL = 0, 1, 2
WEST, EAST, SOUTH, NORTH = 0, 1, 2, 3

_libs: dict = {}


def _fields(real):
    return [
        ("nx", C.c_int), ("ny", C.c_int), ("model", C.c_int), ("edge", C.c_int * 4),
        ("omega", real * 6), ("force", real * 2), ("wall_u", real * 4), ("rho_w", real),
        ("force_field", C.c_void_p),
    ]


class _Cplx(C.Structure):
    _fields_ = [("re", C.c_double), ("im", C.c_double)]


class _LatReal(C.Structure):
    _fields_ = _fields(C.c_double)


class _LatCplx(C.Structure):
    _fields_ = _fields(_Cplx)


def _load(path: str, kind: str):
    """Load one build of the oracle and declare its symbols."""
    lib = C.CDLL(path)
    sfx = "_cs" if kind == "complex" else ""
    vp = C.c_void_p
    for name, argc in [
        ("oracle_macros_node", 5), ("oracle_source", 3), ("oracle_collide_cascaded", 4),
        ("oracle_collide_bgk", 4), ("oracle_collide_rawmrt", 4),
        ("oracle_equilibrium_cascaded", 2), ("oracle_equilibrium_poly", 2),
        ("oracle_strain_node", 4), ("oracle_init", 4), ("oracle_collide_all", 3),
        ("oracle_stream_all", 3), ("oracle_macros", 4), ("oracle_strain", 3),
    ]:
        fn = getattr(lib, name + sfx)
        fn.argtypes = [vp] * argc
        fn.restype = None
    run = getattr(lib, "oracle_run" + sfx)
    run.argtypes = [vp, vp, vp, C.c_long]
    run.restype = None
    return lib


def _lib(kind: str = "real"):
    if kind not in _libs:
        _libs[kind] = _load(_build.build()[kind], kind)
    return _libs[kind]


class substituted_library:
    """Context manager that routes this module's real-valued calls through
    another build of the oracle source (used to plant mistakes in tests)."""

    def __init__(self, path: str):
        self.path = path

    def __enter__(self):
        self.saved = _libs.get("real")
        _libs["real"] = _load(self.path, "real")
        return self

    def __exit__(self, *exc):
        if self.saved is None:
            _libs.pop("real", None)
        else:
            _libs["real"] = self.saved
        return False


def _dtype(kind):
    return np.complex128 if kind == "complex" else np.float64


def _arr(x, kind, shape=None):
    a = np.ascontiguousarray(np.asarray(x, dtype=_dtype(kind)))
    if shape is not None:
        a = a.reshape(shape)
    return a


def _ptr(a):
    return a.ctypes.data_as(C.c_void_p) if a is not None else None


def _fn(kind, name):
    return getattr(_lib(kind), name + ("_cs" if kind == "complex" else ""))


def _kind_of(*xs):
    return "complex" if any(np.iscomplexobj(x) for x in xs if x is not None) else "real"


# --------------------------------------------------------------------------
# single-node functions


def collide_node(model, fb, force=(0.0, 0.0), omegas=(1.0,) * 6):
    """One node's post-collision populations (cascaded: Eq. 13-25)."""
    kind = _kind_of(fb, force, omegas)
    fb, F, om = _arr(fb, kind, (9,)), _arr(force, kind, (2,)), _arr(omegas, kind, (6,))
    out = np.empty(9, _dtype(kind))
    name = {CASCADED: "oracle_collide_cascaded", BGK: "oracle_collide_bgk",
            RAWMRT: "oracle_collide_rawmrt"}[model]
    _fn(kind, name)(_ptr(fb), _ptr(F), _ptr(om), _ptr(out))
    return out


def macros_node(fb, force=(0.0, 0.0)):
    """(rho, ux, uy) of Eq. (26)-(27)."""
    kind = _kind_of(fb, force)
    fb, F = _arr(fb, kind, (9,)), _arr(force, kind, (2,))
    r = np.empty(3, _dtype(kind))
    _fn(kind, "oracle_macros_node")(_ptr(fb), _ptr(F), _ptr(r[0:]), _ptr(r[1:]), _ptr(r[2:]))
    return r


def source_node(u, force):
    """S_0..S_8 of Eq. (14) with the m^s list before it."""
    kind = _kind_of(u, force)
    u, F = _arr(u, kind, (2,)), _arr(force, kind, (2,))
    S = np.empty(9, _dtype(kind))
    _fn(kind, "oracle_source")(_ptr(u), _ptr(F), _ptr(S))
    return S


def equilibrium_node(model, rho, ux, uy):
    """f_eq: central-moment matched (cascaded) or 2nd-order polynomial (siblings)."""
    kind = _kind_of(np.array([rho, ux, uy]))
    ru = _arr([rho, ux, uy], kind, (3,))
    out = np.empty(9, _dtype(kind))
    name = "oracle_equilibrium_cascaded" if model == CASCADED else "oracle_equilibrium_poly"
    _fn(kind, name)(_ptr(ru), _ptr(out))
    return out


def strain_node(fb, force=(0.0, 0.0), omegas=(1.0,) * 6):
    """(d_x j_x, d_y j_y, d_x j_y + d_y j_x) from non-equilibrium moments, Eq. (28)-(30)."""
    kind = _kind_of(fb, force, omegas)
    fb, F, om = _arr(fb, kind, (9,)), _arr(force, kind, (2,)), _arr(omegas, kind, (6,))
    out = np.empty(3, _dtype(kind))
    _fn(kind, "oracle_strain_node")(_ptr(fb), _ptr(F), _ptr(om), _ptr(out))
    return out


# --------------------------------------------------------------------------
# whole lattice


class Lattice:
    """A D2Q9 lattice advanced by the oracle.

    edges: (W, E, S, N) each PERIODIC / BOUNCEBACK / MOVING_WALL; wall_u the
    tangential wall speeds.  omegas = (omega_3..omega_8).  ``complex=True``
    runs the complex-step build (every parameter may then carry an imaginary
    perturbation).
    """

    def __init__(self, nx, ny, omegas, force=(0.0, 0.0), edges=(PERIODIC,) * 4,
                 wall_u=(0.0,) * 4, model=CASCADED, rho0=1.0, force_field=None,
                 complex=False):
        self.kind = "complex" if complex else "real"
        dt = _dtype(self.kind)
        self.nx, self.ny, self.model = int(nx), int(ny), int(model)
        self.omegas = np.asarray(omegas, dt).reshape(6)
        self.force = np.asarray(force, dt).reshape(2)
        self.edges = tuple(int(e) for e in edges)
        self.wall_u = np.asarray(wall_u, dt).reshape(4)
        self.rho0 = rho0
        self.force_field = (None if force_field is None
                            else _arr(force_field, self.kind, (2, self.ny, self.nx)))
        self.f = np.zeros((9, self.ny, self.nx), dt)
        self._work = np.zeros_like(self.f)

    def _struct(self):
        if self.kind == "complex":
            s = _LatCplx()
            conv = lambda v: _Cplx(complex(v).real, complex(v).imag)  # noqa: E731
        else:
            s = _LatReal()
            conv = float
        s.nx, s.ny, s.model = self.nx, self.ny, self.model
        for i in range(4):
            s.edge[i] = self.edges[i]
            s.wall_u[i] = conv(self.wall_u[i])
        for i in range(6):
            s.omega[i] = conv(self.omegas[i])
        s.force[0], s.force[1] = conv(self.force[0]), conv(self.force[1])
        s.rho_w = conv(self.rho0)
        s.force_field = (self.force_field.ctypes.data if self.force_field is not None else None)
        return s

    def init(self, rho=None, u=None):
        """Transformed equilibrium f_bar = f_eq(rho, u) - S/2 (Eq. 6, 12)."""
        shape = (self.ny, self.nx)
        rho = _arr(np.full(shape, self.rho0) if rho is None else rho, self.kind, shape)
        u = _arr(np.zeros((2,) + shape) if u is None else u, self.kind, (2,) + shape)
        s = self._struct()
        _fn(self.kind, "oracle_init")(C.byref(s), _ptr(rho), _ptr(u), _ptr(self.f))
        return self

    def set_f(self, f):
        self.f[...] = _arr(f, self.kind, self.f.shape)
        return self

    def run(self, nsteps):
        """nsteps of collide-all (Eq. 23) then stream-all (Eq. 24)."""
        s = self._struct()
        _fn(self.kind, "oracle_run")(C.byref(s), _ptr(self.f), _ptr(self._work), C.c_long(int(nsteps)))
        return self

    def collide(self):
        """Post-collision populations of the current state (no streaming)."""
        s = self._struct()
        post = np.empty_like(self.f)
        _fn(self.kind, "oracle_collide_all")(C.byref(s), _ptr(self.f), _ptr(post))
        return post

    def stream(self, post):
        s = self._struct()
        post = _arr(post, self.kind, self.f.shape)
        _fn(self.kind, "oracle_stream_all")(C.byref(s), _ptr(post), _ptr(self.f))
        return self

    def macros(self):
        """(rho[ny,nx], u[2,ny,nx]) of Eq. (26)-(27)."""
        rho = np.empty((self.ny, self.nx), _dtype(self.kind))
        u = np.empty((2, self.ny, self.nx), _dtype(self.kind))
        s = self._struct()
        _fn(self.kind, "oracle_macros")(C.byref(s), _ptr(self.f), _ptr(rho), _ptr(u))
        return rho, u

    def strain(self):
        """[3, ny, nx]: d_x j_x, d_y j_y, d_x j_y + d_y j_x (Eq. 28-30)."""
        out = np.empty((3, self.ny, self.nx), _dtype(self.kind))
        s = self._struct()
        _fn(self.kind, "oracle_strain")(C.byref(s), _ptr(self.f), _ptr(out))
        return out


# --------------------------------------------------------------------------
# closed-form solutions (Sec. III-A, III-B)


def omega_from_nu(nu):
    """Shear rate from nu = c_s^2 (1/omega - 1/2), c_s^2 = 1/3 (Sec. II)."""
    return 1.0 / (3.0 * nu + 0.5)


def nu_from_omega(omega):
    return (1.0 / omega - 0.5) / 3.0


def taylor_green(n, u0, nu, t, rho0=1.0, k=None):
    """Decaying Taylor-Green vortex, Eq. (35)-(40) of Sec. III-B, at integer
    node coordinates x_i = i, y_j = j on an n x n periodic lattice.
    Returns rho[n,n], u[2,n,n], strain S_xx[n,n]."""
    k = 2.0 * math.pi / n if k is None else k
    x = np.arange(n, dtype=np.float64)
    X, Y = np.meshgrid(x, x, indexing="xy")  # X[j, i] = i
    dec = math.exp(-2.0 * k * k * nu * t)
    ux = -u0 * np.cos(k * X) * np.sin(k * Y) * dec
    uy = u0 * np.sin(k * X) * np.cos(k * Y) * dec
    # p = c_s^2 rho; p0 = rho0/3; Eq. (37)/(40): p = p0 - u0^2/4 (cos 2kx + cos 2ky) e^{-4 k^2 nu t}
    p = rho0 / 3.0 - (u0 * u0 / 4.0) * (np.cos(2 * k * X) + np.cos(2 * k * Y)) * dec * dec
    rho = 3.0 * p
    sxx = k * u0 * np.sin(k * X) * np.sin(k * Y) * dec
    return rho, np.stack([ux, uy]), sxx


def taylor_green_decay_time(n, nu):
    """T = 1/(2 k^2 nu) with k = 2 pi / n (Sec. III-B)."""
    k = 2.0 * math.pi / n
    return 1.0 / (2.0 * k * k * nu)


def poiseuille_profile(ny, fx, nu):
    """Steady channel profile between half-way bounce-back walls at y = -1/2 and
    y = ny - 1/2: u(y) = u_max (1 - s^2/L^2) with L = ny/2 the half width and
    u_max = F L^2 / (2 nu) (Sec. III-A), s the distance from the centre line."""
    L = ny / 2.0
    y = np.arange(ny, dtype=np.float64) + 0.5  # distance from the south wall
    s = y - L
    return fx * L * L / (2.0 * nu) * (1.0 - s * s / (L * L))


def relative_error_paper(u_c, u_a):
    """Eq. (34): sum_i ||u_c,i - u_a,i|| / sum_i ||u_a,i|| (Euclidean norm per node)."""
    d = np.sqrt(((np.asarray(u_c) - np.asarray(u_a)) ** 2).sum(axis=0))
    a = np.sqrt((np.asarray(u_a) ** 2).sum(axis=0))
    return float(d.sum() / a.sum())


def relative_l2(u_c, u_ref):
    """sqrt(sum |u_c - u_ref|^2 / sum |u_ref|^2) over every node and component."""
    u_c, u_ref = np.asarray(u_c), np.asarray(u_ref)
    return float(np.sqrt(((u_c - u_ref) ** 2).sum() / (u_ref ** 2).sum()))
