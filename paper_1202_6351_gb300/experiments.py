"""Lid-driven cavity experiments of Sec. IV-V run on the CUDA path.

* :func:`cavity_steady` runs a lid-driven cavity to steady state (max |du| over
  1000 steps below a tolerance) and returns its velocity field.
* :func:`vortex_centre` locates the primary vortex (Sec. IV-C, Table I) from
  the stream function psi(x, y), the integral of u along y from the bottom wall.
* :func:`max_stable_cell_reynolds` finds, for one collision model and grid,
  the largest cell Reynolds number Re_c = U dx / nu at which the cavity stays
  stable (Sec. V, Table IV), running many viscosities side by side in one
  batched launch per step; :func:`max_stable_lid_velocity` does the same for
  the lid speed on a fixed coarse grid at fixed viscosity (Sec. V).
* :func:`secondary_vortex` locates the corner vortices of Table II and
  :func:`cavity_convergence` runs the grid-convergence study of Sec. III-C.
* :func:`cavity_matrix` runs the lid-driven cavity at several Reynolds numbers
  with the three collision models side by side, each in FP32 storage (to a
  steady state) and in FP16 storage with both rounding modes (for the same
  number of steps), one batched launch per model and step.

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
                  other_rate=1.0, fields=False, nu=None):
    """Run from rest until max |u(t) - u(t - check)| < tol (per `check` steps).
    The viscosity is nu = U (n - 1)/re unless `nu` is given.
    Returns (u[2, n, n], steps), or with fields=True (rho, u, strain[3, n, n], steps)
    where strain holds (d_x j_x, d_y j_y, d_x j_y + d_y j_x) from the
    non-equilibrium moments (Eq. 28-30)."""
    om = cavity_omega(n, re, U) if nu is None else 1.0 / (3.0 * nu + 0.5)
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
    """psi[j, i] = sum_{k < j} u_x[k, i] + u_x[j, i] / 2: the integral of u_x from
    the bottom wall (psi = 0 there, half a spacing below node row 0) up to the
    node itself, cell by cell with the midpoint rule (unit spacing)."""
    return np.cumsum(u[0], axis=0) - 0.5 * u[0]


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


def _stable(u):
    """A run is stable unless it blew up: every velocity finite and within the
    range D2Q9 populations can carry (|u_x|, |u_y| <= 1 needs no negative
    population).  Returns (stable, max |u|)."""
    if not np.isfinite(u).all():
        return False, float("inf")
    umax = float(np.abs(u).max())
    return umax <= 1.0, umax


def _cavity_sweep(model, n, cases, steps, store):
    """Run one n x n cavity per (nu, U) in `cases` side by side in one batched
    launch per step for `steps` steps; returns [(stable, max |u|)]."""
    lattices = []
    for nu, U in cases:
        om = 1.0 / (3.0 * nu + 0.5)
        L = lbm.Lattice(n, n, (1.0, om, om, 1.0, 1.0, 1.0), edges=CAVITY_EDGES, wall_u=(0, 0, 0, U), model=model,
                        store=store)
        L.init()
        lattices.append(L)
    steps += steps % 2
    with lbm.Batch(lattices) as B:
        B.step(steps)
        B.sync()
    out = []
    for L in lattices:
        _, u = L.macros()
        out.append(_stable(u))
        L.close()
    return out


def _threshold(values, flags):
    """Largest candidate below which every candidate (in increasing order) was stable."""
    threshold = 0.0
    for v, ok in zip(values, flags):
        if not ok:
            break
        threshold = v
    return threshold


def max_stable_cell_reynolds(model, n, U=0.1, cell_res=None, convective_times=20.0, store=lbm.F32):
    """Largest Re_c = U / nu in `cell_res` (default: 48 values log-spaced in [4, 400])
    below which every candidate n x n cavity stays stable for
    `convective_times` x n / U steps (Sec. V, Table IV: the lid speed is fixed
    and the viscosity lowered); all candidates run in one batch.

    Sec. V calls a run unstable when its error grows rapidly or becomes
    exponentially large; here a run is unstable when it blows up (a
    non-finite velocity, or one beyond what the lattice can carry).  Above
    some Re_c the cascaded runs keep a bounded hot spot near the lid corners
    with velocities close to the lattice sound speed without blowing up; they
    count as stable.
    Returns (threshold, list of (Re_c, stable, max |u|))."""
    if cell_res is None:
        cell_res = np.exp(np.linspace(math.log(4.0), math.log(400.0), 48))
    cell_res = [float(rc) for rc in cell_res]
    res = _cavity_sweep(model, n, [(U / rc, U) for rc in cell_res], int(convective_times * n / U), store)
    result = [(rc, ok, umax) for rc, (ok, umax) in zip(cell_res, res)]
    return _threshold(cell_res, [ok for _, ok, _ in result]), result


def max_stable_cell_reynolds_refined(model, n, U=0.1, lo=4.0, hi=400.0, first=16, per_round=8, rounds=3,
                                     convective_times=20.0, store=lbm.F32):
    """max_stable_cell_reynolds with the threshold bracketed ever more finely:
    `first` candidates log-spaced in [lo, hi], then `rounds` times `per_round`
    candidates log-spaced inside the bracket [last stable, first unstable] of
    the round before (all candidates of a round run in one batch).  After the
    default three rounds the bracket is about 1/512 of the first one in log
    space (a few tenths of a percent).  Returns (threshold, first unstable
    value, every (Re_c, stable, max |u|) tried)."""
    steps = int(convective_times * n / U)
    tried = []

    def run(values):
        res = _cavity_sweep(model, n, [(U / rc, U) for rc in values], steps, store)
        out = [(rc, ok, umax) for rc, (ok, umax) in zip(values, res)]
        tried.extend(out)
        return out

    values = [float(v) for v in np.exp(np.linspace(math.log(lo), math.log(hi), first))]
    res = run(values)
    stable, unstable = lo, None
    for rc, ok, _ in res:
        if not ok:
            unstable = rc
            break
        stable = rc
    if unstable is None:
        return stable, None, tried
    for _ in range(rounds):
        inner = [float(v) for v in np.exp(np.linspace(math.log(stable), math.log(unstable), per_round + 2))[1:-1]]
        for rc, ok, _ in run(inner):
            if not ok:
                unstable = rc
                break
            stable = rc
    return stable, unstable, tried


def max_stable_lid_velocity(model, nu, n=26, lid_u=None, steps=50_000, store=lbm.F32):
    """Sec. V's alternative test: on a fixed coarse n x n cavity (26 x 26) at a
    fixed viscosity, the largest lid speed in `lid_u` (default: 40 values
    log-spaced in [0.005, 0.8]) below which every candidate stays stable for
    `steps` steps (50,000).  Returns (threshold, list of (U, stable, max |u|))."""
    if lid_u is None:
        lid_u = np.exp(np.linspace(math.log(0.005), math.log(0.8), 40))
    lid_u = [float(U) for U in lid_u]
    res = _cavity_sweep(model, n, [(nu, U) for U in lid_u], steps, store)
    result = [(U, ok, umax) for U, (ok, umax) in zip(lid_u, res)]
    return _threshold(lid_u, [ok for _, ok, _ in result]), result


# Corner regions (in units of L) searched for the counter-rotating secondary
# vortices of Sec. IV-C, Table II.
SECONDARY_REGIONS = {"bottom_left": ((0.0, 0.35), (0.0, 0.35)), "bottom_right": ((0.65, 1.0), (0.0, 0.35)),
                     "top_left": ((0.0, 0.35), (0.65, 1.0))}


def secondary_vortex(u, region):
    """Centre of the secondary (counter-clockwise) vortex in a corner region:
    the maximum of psi there, refined by parabolas; None if psi has no interior
    maximum in the region (no such vortex)."""
    psi = stream_function(u)
    n = psi.shape[0]
    (x0, x1), (y0, y1) = SECONDARY_REGIONS[region]
    i0, i1 = max(1, int(x0 * n)), min(n - 2, int(x1 * n))
    j0, j1 = max(1, int(y0 * n)), min(n - 2, int(y1 * n))
    sub = psi[j0:j1 + 1, i0:i1 + 1]
    jj, ii = np.unravel_index(np.argmax(sub), sub.shape)
    j, i = j0 + int(jj), i0 + int(ii)
    if j in (j0, j1) or i in (i0, i1) or psi[j, i] <= 0.0:
        return None
    di = _parabola_vertex(-psi[j, i - 1], -psi[j, i], -psi[j, i + 1])
    dj = _parabola_vertex(-psi[j - 1, i], -psi[j, i], -psi[j + 1, i])
    return ((i + di + 0.5) / n, (j + dj + 0.5) / n)


def centreline_profiles(u):
    """u along the vertical centre line and v along the horizontal one (odd n:
    the centre lines pass through nodes), with their node positions in units of L."""
    n = u.shape[1]
    c = (n - 1) // 2
    pos = (np.arange(n) + 0.5) / n
    return pos, u[0][:, c], u[1][c, :]


# Centre-line quantities of the grid-convergence study (Sec. III-C, Figs. on the
# cavity): velocity components and the strain-rate components dv/dy and
# du/dy + dv/dx along the vertical (x = L/2) and horizontal (y = L/2) lines.
CONVERGENCE_QUANTITIES = ("u_vertical", "u_horizontal", "v_vertical", "v_horizontal", "dvdy_vertical",
                          "dvdy_horizontal", "shear_vertical", "shear_horizontal")


def _centre_lines(rho, u, strain, U, n):
    """The CONVERGENCE_QUANTITIES in units of U (velocities) and U / L (strain
    rates, from the non-equilibrium moments, Eq. 28-30, divided by rho)."""
    c = (n - 1) // 2
    dvdy = strain[1] / rho * (n / U)
    shear = strain[2] / rho * (n / U)
    ux, uy = u[0] / U, u[1] / U
    return {"u_vertical": ux[:, c], "u_horizontal": ux[c, :], "v_vertical": uy[:, c], "v_horizontal": uy[c, :],
            "dvdy_vertical": dvdy[:, c], "dvdy_horizontal": dvdy[c, :], "shear_vertical": shear[:, c],
            "shear_horizontal": shear[c, :]}


def cavity_convergence(sides=(13, 19, 25, 31, 37, 49), reference=121, re=100.0, u_coarsest=0.1, rel_tol=1e-6,
                       model=lbm.CASCADED, store=lbm.F64, reference_store=None, reference_steps=None):
    """Sec. III-C grid convergence at fixed Re under diffusive scaling (U ~ 1/n,
    nu fixed): relative global errors (Eq. 34, Euclidean norm) of the centre-line
    quantities CONVERGENCE_QUANTITIES against a finer run, linearly interpolated
    to the coarse nodes.  With half-way walls the side is L = n, so
    Re = U n / nu on every grid (a fixed n - 1 would shift Re by O(1/n)).

    Each grid runs until max |du| over 1000 steps is below
    rel_tol U (n0 / n)^2 (the slowest mode decays at a rate ~ nu / n^2, so this
    leaves the same residual on every grid); the reference may instead run a
    fixed `reference_steps` in `reference_store` (an FP32 801^2 run cannot
    resolve such small changes, and needs no checks).
    Returns {n: {quantity: error}}."""
    n0 = sides[0]
    nu = u_coarsest * n0 / re
    om = 1.0 / (3.0 * nu + 0.5)

    def run(n, st, steps=None):
        U = u_coarsest * n0 / n
        if steps is None:
            rho, u, strain, _ = cavity_steady(n, re, model=model, store=st, U=U, tol=rel_tol * U * (n0 / n) ** 2,
                                              max_steps=200_000_000, nu=nu, fields=True)
        else:
            with lbm.Lattice(n, n, (1.0, om, om, 1.0, 1.0, 1.0), edges=CAVITY_EDGES, wall_u=(0, 0, 0, U), model=model,
                             store=st) as L:
                L.init()
                L.step(steps + steps % 2)
                rho, u = L.macros()
                strain = L.strain()
        return (np.arange(n) + 0.5) / n, _centre_lines(rho, u, strain, U, n)

    pr, ref = run(reference, store if reference_store is None else reference_store, reference_steps)
    out = {}
    for n in sides:
        p, q = run(n, store)
        errs = {}
        for k in CONVERGENCE_QUANTITIES:
            qi = np.interp(p, pr, ref[k])
            errs[k] = float(np.sqrt(((q[k] - qi) ** 2).sum() / (qi ** 2).sum()))
        out[n] = errs
    return out


# ---------------------------------------------------------------------------
# The cavity configuration: Re x model x storage side by side


def _blown_up(u):
    return not np.isfinite(u).all() or float(np.abs(u).max()) > 1.0


def cavity_matrix(n, res=(1000.0, 3200.0, 5000.0), models=(lbm.CASCADED, lbm.BGK, lbm.RAWMRT), U=0.1, tol=1e-7,
                  check=1000, max_steps=20_000_000, f16=True, seed=2026, progress=None):
    """Lid-driven cavities of n x n nodes at each Reynolds number in `res`
    (nu = U (n - 1) / Re, other rates 1, from rest; Sec. IV-C, V) for each
    collision model, each in FP32 storage and, if `f16`, in FP16 storage with
    round to nearest and with stochastic rounding.  All lattices of one model
    advance together in one batched launch per two steps (lbm.Batch with two
    steps per launch); the batches of the models run on their own streams at
    the same time.

    A case (model, Re) runs until its FP32 lattice is steady (max |u(t) -
    u(t - check)| < tol) or blows up (a non-finite velocity or |u| > 1), or
    until max_steps.  Its FP16 lattices run the same number of steps and are
    compared with the FP32 field then (FP16 storage resolves velocities only to
    about 1e-5, so it has no steady state at tol; with stochastic rounding its
    field keeps a random jitter).

    Returns {(model, re): {"steps", "status" ("steady", "diverged" or
    "unsteady"), "f32": {...}, "f16_nearest": {...}, "f16_stochastic": {...}}};
    each storage entry holds the velocity field "u", its "max_du" over the last
    `check` steps and, when finite, the primary vortex "centre" and the
    secondary vortices of Table II; the FP16 entries also hold "rel_l2_vs_f32"
    (relative L2 difference of the velocity from the FP32 field) and
    "centre_shift" (distance of the primary vortex from the FP32 one)."""
    om_other = 1.0
    cases = {}
    for model in models:
        for re in res:
            om = cavity_omega(n, re, U)
            rates = (om_other, om, om, om_other, om_other, om_other)
            kinds = [("f32", lbm.F32, None)]
            if f16:
                kinds += [("f16_nearest", lbm.F16DEV, lbm.ROUND_NEAREST),
                          ("f16_stochastic", lbm.F16DEV, lbm.ROUND_STOCHASTIC)]
            lat = {}
            for name, st, rounding in kinds:
                L = lbm.Lattice(n, n, rates, edges=CAVITY_EDGES, wall_u=(0, 0, 0, U), model=model, store=st)
                if rounding == lbm.ROUND_STOCHASTIC:
                    L.set_rounding(rounding, seed)
                L.init()
                lat[name] = L
            cases[model, float(re)] = {"lattices": lat, "prev": {}, "result": None}

    def batches():
        out = []
        for model in models:
            ls = [L for (m, _), c in cases.items() if m == model and c["result"] is None for L in c["lattices"].values()]
            if ls:
                B = lbm.Batch(ls)
                if n >= 4:
                    B.set_two_step(True)  # two steps per launch; bit for bit the same states
                out.append(B)
        return out

    live = batches()
    steps = 0
    try:
        while live and steps < max_steps:
            for B in live:
                B.step(check)
            for B in live:
                B.sync()
            steps += check
            changed = False
            for key, c in cases.items():
                if c["result"] is not None:
                    continue
                fields = {name: L.macros()[1] for name, L in c["lattices"].items()}
                u32 = fields["f32"]
                du = {name: (float(np.abs(u - c["prev"][name]).max()) if name in c["prev"] else float("inf"))
                      for name, u in fields.items()}
                status = None
                if _blown_up(u32):
                    status = "diverged"
                elif du["f32"] < tol:
                    status = "steady"
                elif steps >= max_steps:
                    status = "unsteady"
                if status is not None:
                    c["result"] = _matrix_entry(status, steps, fields, du)
                    changed = True
                    if progress:
                        progress(key, c["result"])
                c["prev"] = fields
            if changed:
                for B in live:
                    B.close()
                live = batches()
    finally:
        for B in live:
            B.close()
        for c in cases.values():
            for L in c["lattices"].values():
                L.close()
    out = {}
    for key, c in cases.items():
        out[key] = c["result"] if c["result"] is not None else {"steps": steps, "status": "unsteady"}
    return out


def _matrix_entry(status, steps, fields, du):
    entry = {"steps": steps, "status": status}
    u32 = fields["f32"]
    c32 = None
    for name, u in fields.items():
        e = {"u": u, "max_du": du[name]}
        if not _blown_up(u):
            e["centre"] = vortex_centre(u)
            e["secondary"] = {r: secondary_vortex(u, r) for r in SECONDARY_REGIONS}
            if name == "f32":
                c32 = e["centre"]
            elif c32 is not None:
                e["rel_l2_vs_f32"] = float(np.sqrt(((u - u32) ** 2).sum() / (u32 ** 2).sum()))
                e["centre_shift"] = float(math.hypot(e["centre"][0] - c32[0], e["centre"][1] - c32[1]))
        entry[name] = e
    return entry


def matrix_summary(results):
    """The cavity matrix without velocity fields, keyed "model/Re" (JSON-ready)."""
    out = {}
    for (model, re), r in sorted(results.items()):
        row = {"steps": r["steps"], "status": r["status"]}
        for name in ("f32", "f16_nearest", "f16_stochastic"):
            if name in r:
                row[name] = {k: v for k, v in r[name].items() if k != "u"}
        out[f"{lbm.MODEL_NAMES[model]}/{int(re)}"] = row
    return out


def taylor_green_decay(n, store=lbm.F32, rounding=lbm.ROUND_NEAREST, omega=1.6, fractions=(0.25, 0.5, 1.0),
                       seed=2026, progress=None):
    """The Taylor-Green configuration (Sec. III-B) on n^2 (diffusive scaling
    U0 = 0.04 * 64 / n, shear omega, other rates 1) run to one decay time
    T = 1 / (2 nu k^2), with the relative L2 velocity error against the
    analytic decay and the fitted amplitude at the given fractions of T.
    Returns [(steps, error, amplitude, seconds)]."""
    import time

    from . import workloads

    nu = (1.0 / omega - 0.5) / 3.0
    u0 = workloads.diffusive_u0(n)
    T = workloads.taylor_green_decay_steps(n, nu)
    rho, u = workloads.taylor_green_init(n, u0)
    out = []
    t0 = time.time()
    with lbm.Lattice(n, n, (1.0, omega, omega, 1.0, 1.0, 1.0), store=store) as L:
        if rounding == lbm.ROUND_STOCHASTIC:
            L.set_rounding(rounding, seed)
        L.init(rho, u)
        done = 0
        for fr in fractions:
            target = int(round(fr * T))
            L.step(target - done)
            done = target
            _, ug = L.macros()
            ua = workloads.taylor_green_velocity(n, u0, nu, done)
            err = float(np.sqrt(((ug - ua) ** 2).sum() / (ua ** 2).sum()))
            amp = float((ug * ua).sum() / (ua * ua).sum())
            out.append((done, err, amp, time.time() - t0))
            if progress:
                progress(out[-1])
    return out


if __name__ == "__main__":
    import argparse
    import json
    import sys
    import time

    if len(sys.argv) > 1 and sys.argv[1] == "decay":
        ap = argparse.ArgumentParser(description="Taylor-Green to one decay time on the GPU.")
        ap.add_argument("decay")
        ap.add_argument("--n", type=int, default=4096)
        ap.add_argument("--store", choices=["f32", "f16", "bf16"], default="f32")
        ap.add_argument("--rounding", choices=["nearest", "stochastic"], default="nearest")
        args = ap.parse_args()
        st = {"f32": lbm.F32, "f16": lbm.F16DEV, "bf16": lbm.BF16DEV}[args.store]
        rd = lbm.ROUND_STOCHASTIC if args.rounding == "stochastic" else lbm.ROUND_NEAREST

        def show(r):
            print(json.dumps({"n": args.n, "store": args.store, "rounding": args.rounding, "steps": r[0],
                              "rel_l2_velocity_error": r[1], "amplitude": r[2], "seconds": round(r[3], 1)}),
                  flush=True)

        taylor_green_decay(args.n, st, rd, progress=show)
        sys.exit(0)

    ap = argparse.ArgumentParser(description="Run the lid-driven cavity matrix (three models, FP32 / FP16) on the GPU.")
    ap.add_argument("--n", type=int, default=257)
    ap.add_argument("--re", type=float, nargs="+", default=[1000.0, 3200.0, 5000.0])
    ap.add_argument("--models", nargs="+", default=["cascaded", "bgk", "rawmrt"])
    ap.add_argument("--max-steps", type=int, default=20_000_000)
    ap.add_argument("--no-f16", action="store_true")
    args = ap.parse_args()
    names = {v: k for k, v in lbm.MODEL_NAMES.items()}
    t0 = time.time()

    def report(key, r):
        print(json.dumps({"case": f"{lbm.MODEL_NAMES[key[0]]}/{int(key[1])}", "n": args.n,
                          "seconds": round(time.time() - t0, 1),
                          **matrix_summary({key: r})[f"{lbm.MODEL_NAMES[key[0]]}/{int(key[1])}"]}), flush=True)

    res = cavity_matrix(args.n, tuple(args.re), tuple(names[m] for m in args.models), max_steps=args.max_steps,
                        f16=not args.no_f16, progress=report)
    print(json.dumps({"n": args.n, "seconds": round(time.time() - t0, 1), "matrix": matrix_summary(res)}), flush=True)
