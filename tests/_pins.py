"""Independent checks shared by the oracle pin tests.

Everything here is written from the mathematics the paper fixes (definitions
of raw and central moments, the printed basis and tables under tests/golden/),
not from the oracle's code: moments are taken by direct summation over the
nine populations, never through the oracle's own moment formulas.
"""
from __future__ import annotations

import json
import os

import numpy as np

GOLDEN = os.path.join(os.path.dirname(os.path.abspath(__file__)), "golden")


def _table(name):
    rows = []
    with open(os.path.join(GOLDEN, name)) as fh:
        for line in fh:
            line = line.split("#", 1)[0].strip()
            if line:
                rows.append([float(v) for v in line.split()])
    return np.array(rows)


E = _table("lattice_vectors.txt")            # [2, 9]: e_ax, e_ay (Eq. 1)
EX, EY = E[0], E[1]
K = _table("k_matrix.txt")                   # [9, 9]: Eq. (3)
KERNEL_MOMENTS = _table("kernel_moments.txt")  # Eq. (16)
SOURCE_MATRIX = _table("source_matrix.txt")    # 36 * Eq. (14)
with open(os.path.join(GOLDEN, "paper_results.json")) as _fh:
    PAPER = json.load(_fh)

# the nine moment orders (m, n) in the paper's order 0, x, y, xx, yy, xy, xxy, xyy, xxyy
ORDERS = [(0, 0), (1, 0), (0, 1), (2, 0), (0, 2), (1, 1), (2, 1), (1, 2), (2, 2)]


def raw_moments(f):
    """sum_a e_ax^m e_ay^n f_a for the nine orders."""
    f = np.asarray(f)
    return np.array([(EX ** m * EY ** n * f).sum() for m, n in ORDERS])


def central_moments(f, ux, uy):
    """sum_a (e_ax - ux)^m (e_ay - uy)^n f_a for the nine orders (Sec. II definition)."""
    f = np.asarray(f)
    cx, cy = EX - ux, EY - uy
    return np.array([(cx ** m * cy ** n * f).sum() for m, n in ORDERS])


def central_matrix(ux, uy):
    """T(u): rows are (e_x - ux)^m (e_y - uy)^n, so T f = central moments."""
    cx, cy = EX - ux, EY - uy
    return np.array([cx ** m * cy ** n for m, n in ORDERS])


def relaxed_central(pre, rho, F, om):
    """Relaxation of central moments the cascaded scheme performs (Sec. II): the
    trace relaxes to 2 rho/3 at omega_3, the deviator to 0 at omega_4, xy to 0 at
    omega_5, xxy and xyy to 0 at omega_6, omega_7, xxyy to rho/9 at omega_8; mass
    is kept and the first central moments move from -F/2 to +F/2."""
    w3, w4, w5, w6, w7, w8 = om
    post = np.array(pre, dtype=float).copy()
    tr, dv = pre[3] + pre[4], pre[3] - pre[4]
    tr = (1 - w3) * tr + w3 * 2.0 * rho / 3.0
    dv = (1 - w4) * dv
    post[3], post[4] = 0.5 * (tr + dv), 0.5 * (tr - dv)
    post[5] = (1 - w5) * pre[5]
    post[6] = (1 - w6) * pre[6]
    post[7] = (1 - w7) * pre[7]
    post[8] = (1 - w8) * pre[8] + w8 * rho / 9.0
    post[1] = pre[1] + F[0]
    post[2] = pre[2] + F[1]
    return post


def weights():
    """Populations with central moments (1,0,0,1/3,1/3,0,0,0,1/9) at u = 0,
    solved from the monomial system (Eq. 10 with rho = 1)."""
    M = np.array([EX ** m * EY ** n for m, n in ORDERS])
    return np.linalg.solve(M, np.array([1, 0, 0, 1 / 3, 1 / 3, 0, 0, 0, 1 / 9]))


def stream_pull_reference(post, edges, wall_u, rho_w=1.0):
    """Streaming with periodic / bounce-back / moving-wall edges written in pull
    form with explicit loops: f_a(x) = post_a(x - e_a) if that node exists (after
    periodic wrap), else post_abar(x) plus the moving-wall term
    6 w_a rho_w (e_a . U_wall).  A source outside in y is decided by the S/N
    edge first; a source outside past both a S/N wall and a W/E wall (the
    corner point) takes no moving-wall term."""
    nine, ny, nx = post.shape
    w = weights()
    opp = [int(np.where((EX == -EX[a]) & (EY == -EY[a]))[0][0]) for a in range(9)]
    out = np.zeros_like(post)
    for y in range(ny):
        for x in range(nx):
            for a in range(9):
                sx, sy = x - int(EX[a]), y - int(EY[a])
                yw = 2 if sy < 0 else (3 if sy >= ny else -1)
                xw = 0 if sx < 0 else (1 if sx >= nx else -1)
                wall = -1
                if yw >= 0 and edges[yw] != 0:
                    wall = yw
                elif xw >= 0 and edges[xw] != 0:
                    wall = xw
                corner = yw >= 0 and edges[yw] != 0 and xw >= 0 and edges[xw] != 0
                if wall >= 0:
                    corr = 0.0
                    if edges[wall] == 2 and not corner:
                        U = (wall_u[wall], 0.0) if wall >= 2 else (0.0, wall_u[wall])
                        corr = 6.0 * w[a] * rho_w * (EX[a] * U[0] + EY[a] * U[1])
                    out[a, y, x] = post[opp[a], y, x] + corr
                else:
                    out[a, y, x] = post[a, sy % ny, sx % nx]
    return out
