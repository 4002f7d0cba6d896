"""Lid-driven cavity experiments of Sec. IV-V run on the CUDA path.

* :func:`cavity_steady` runs a lid-driven cavity to steady state (max |du| over
  1000 steps below a tolerance) and returns its velocity field.
* :func:`vortex_centre` locates the primary vortex (Sec. IV-C, Table I) from
  the stream function psi(x, y) = sum of u along y from the bottom wall.
* :func:`max_stable_cell_reynolds` finds, for one collision model and grid,
  the largest cell Reynolds number Re_c = U dx / nu at which the cavity stays
  bounded (Sec. V, Table IV), running many viscosities side by side in one
  batched launch per step.

All lattice work goes through the C ABI (:mod:`paper_1202_6351_gb300.lbm`);
this module only sets parameters and post-processes fields with numpy.
"""
from __future__ import annotations

import math

import numpy as np

from . import lbm

CAVITY_EDGES = (lbm.BOUNCEBACK, lbm.BOUNCEBACK, lbm.BOUNCEBACK, lbm.MOVING_WALL)


def cavity_omega(n, re, U=0.1):
    """Shear rate for a cavity of n nodes per side at Reynolds number re = U (n - 1)/nu."""
    nu = U * (n - 1) / re
    return 1.0 / (3.0 * nu + 0.5)


def cavity_steady(n, re, model=lbm.CASCADED, store=lbm.F32, U=0.1, tol=1e-7, check=1000, max_steps=2_000_000,
                  other_rate=1.0, fields=False):
    """Run from rest until max |u(t) - u(t - check)| < tol (per `check` steps).
    Returns (u[2, n, n], steps), or with fields=True (rho, u, strain[3, n, n], steps)
    where strain holds (d_x j_x, d_y j_y, d_x j_y + d_y j_x) from the
    non-equilibrium moments (Eq. 28-30)."""
    om = cavity_omega(n, re, U)
    rates = (other_rate, om, om, other_rate, other_rate, other_rate)
    with lbm.Lattice(n, n, rates, edges=CAVITY_EDGES, wall_u=(0, 0, 0, U), model=model, store=store) as L:
        L.init()
        L.set_check(check, 1e-3)
        prev = None
        steps = 0
        while steps < max_steps:
            L.step(check)
            steps += check
            rho, u = L.macros()
            if prev is not None and np.abs(u - prev).max() < tol:
                break
            prev = u
        if fields:
            return rho, u, L.strain(), steps
        return u, steps


# The five probe points of Sec. IV-C, Table III, in units of the cavity side L.
TABLE_III_POINTS = {"A": (0.25, 0.5), "B": (0.5, 0.25), "C": (0.5, 0.5), "D": (0.5, 0.75), "E": (0.75, 0.5)}


def strain_at_points(rho, u, strain):
    """dv/dy and du/dy + dv/dx at the Table III points by the two methods of
    Sec. IV-C: local non-equilibrium moments (strain / rho) and second-order
    central differences of the velocity.  Node i sits at (i + 1/2)/n; each point
    takes the nearest node.  Returns {point: (moments_dvdy, fd_dvdy, moments_shear, fd_shear)}."""
    n = u.shape[1]
    out = {}
    for name, (px, py) in TABLE_III_POINTS.items():
        i = int(round(px * n - 0.5))
        j = int(round(py * n - 0.5))
        dvdy_m = strain[1, j, i] / rho[j, i]
        shear_m = strain[2, j, i] / rho[j, i]
        dvdy_fd = 0.5 * (u[1, j + 1, i] - u[1, j - 1, i])
        shear_fd = 0.5 * (u[0, j + 1, i] - u[0, j - 1, i]) + 0.5 * (u[1, j, i + 1] - u[1, j, i - 1])
        out[name] = (float(dvdy_m), float(dvdy_fd), float(shear_m), float(shear_fd))
    return out


def stream_function(u):
    """psi[j, i] = sum_{k <= j} u_x[k, i] (unit spacing; psi = 0 below the bottom wall)."""
    return np.cumsum(u[0], axis=0)


def _parabola_vertex(fm, f0, fp):
    den = fm - 2.0 * f0 + fp
    return 0.0 if den == 0 else 0.5 * (fm - fp) / den


def vortex_centre(u):
    """Primary-vortex centre in units of the cavity side: the extremum of psi
    (clockwise vortex for a lid moving in +x: a minimum), refined by a parabola
    through the neighbours in each direction.  Node i sits at x = (i + 1/2)/n
    between half-way walls at 0 and 1."""
    psi = stream_function(u)
    n = psi.shape[0]
    j, i = np.unravel_index(np.argmin(psi), psi.shape)
    j, i = int(min(max(j, 1), n - 2)), int(min(max(i, 1), n - 2))
    di = _parabola_vertex(psi[j, i - 1], psi[j, i], psi[j, i + 1])
    dj = _parabola_vertex(psi[j - 1, i], psi[j, i], psi[j + 1, i])
    return ((i + di + 0.5) / n, (j + dj + 0.5) / n)


def max_stable_cell_reynolds(model, n, U=0.1, cell_res=None, convective_times=20.0, store=lbm.F32):
    """Largest Re_c = U / nu in `cell_res` (default: 48 values log-spaced in [4, 400])
    below which every candidate n x n cavity stays bounded for
    `convective_times` x n / U steps; all candidates run in one batch.

    Sec. V calls a run unstable when its error grows rapidly or exponentially;
    here a run is stable if every velocity stays finite and below the lattice
    sound speed c_s = 1/sqrt(3).  (Above some Re_c the cascaded and MRT runs keep
    a bounded hot spot of a few times U at the lid corners without blowing up;
    a bound of a few U would call those unstable.)
    Returns (threshold, list of (Re_c, stable, max |u|))."""
    if cell_res is None:
        cell_res = np.exp(np.linspace(math.log(4.0), math.log(400.0), 48))
    lattices = []
    for rc in cell_res:
        nu = U / rc
        om = 1.0 / (3.0 * nu + 0.5)
        L = lbm.Lattice(n, n, (1.0, om, om, 1.0, 1.0, 1.0), edges=CAVITY_EDGES, wall_u=(0, 0, 0, U), model=model,
                        store=store)
        L.init()
        lattices.append(L)
    steps = int(convective_times * n / U)
    steps += steps % 2
    with lbm.Batch(lattices) as B:
        B.step(steps)
        B.sync()
    result = []
    cs = 1.0 / math.sqrt(3.0)
    for rc, L in zip(cell_res, lattices):
        _, u = L.macros()
        umax = float(np.abs(u).max()) if np.isfinite(u).all() else float("inf")
        result.append((float(rc), umax < cs, umax))
        L.close()
    threshold = 0.0
    for rc, ok, _ in result:  # largest Re_c below which every candidate was stable
        if not ok:
            break
        threshold = rc
    return threshold, result
