"""Seeded synthetic inputs shared by the CUDA path's tests and bench and by the oracle.

This module holds no lattice Boltzmann arithmetic (no equilibrium, collision or
streaming): only initial macroscopic fields and random numbers.  Each generator
names the workload it builds and the passage of the paper it follows.
"""
from __future__ import annotations

import math

import numpy as np


def taylor_green_init(n: int, u0: float, rho0: float = 1.0):
    """Initial Taylor-Green fields on an n x n periodic lattice, Sec. III-B:
    u = -u0 cos(kx) sin(ky), v = u0 sin(kx) cos(ky), p = p0 [1 - u0^2/(4 c_s^2)
    (cos 2kx + cos 2ky)] with k = 2 pi / n, node coordinates x_i = i, y_j = j and
    p = rho / 3.  Returns rho[n, n] and u[2, n, n] (float64, row = y)."""
    k = 2.0 * math.pi / n
    x = np.arange(n, dtype=np.float64)
    X, Y = np.meshgrid(x, x, indexing="xy")
    ux = -u0 * np.cos(k * X) * np.sin(k * Y)
    uy = u0 * np.sin(k * X) * np.cos(k * Y)
    rho = rho0 * (1.0 - 0.75 * u0 * u0 * (np.cos(2 * k * X) + np.cos(2 * k * Y)))
    return rho, np.stack([ux, uy])


def taylor_green_velocity(n: int, u0: float, nu: float, t: float):
    """The analytic Taylor-Green velocity of Sec. III-B at time t on the n x n
    node grid of taylor_green_init: the initial field times exp(-2 nu k^2 t),
    k = 2 pi / n.  Returns u[2, n, n] (float64).  This is the decaying solution
    of the Navier-Stokes equations the lattice results are compared with, not
    lattice Boltzmann arithmetic."""
    _, u = taylor_green_init(n, u0)
    k = 2.0 * math.pi / n
    return u * math.exp(-2.0 * nu * k * k * t)


def taylor_green_decay_steps(n: int, nu: float) -> int:
    """One decay time T = 1 / (2 nu k^2), k = 2 pi / n (Sec. III-B), rounded to whole steps."""
    k = 2.0 * math.pi / n
    return int(round(1.0 / (2.0 * nu * k * k)))


def diffusive_u0(n: int, u_ref: float = 0.04, n_ref: int = 64) -> float:
    """Diffusive scaling of Sec. III (Ma/Kn constant): U0 = u_ref * n_ref / n."""
    return u_ref * n_ref / n


def random_fields(seed: int, nx: int, ny: int, u_amp: float = 0.05, rho_amp: float = 0.02):
    """Uncorrelated random (rho, u) fields for parity tests: rho = 1 + rho_amp*N(0,1),
    u = u_amp*N(0,1) per node and component."""
    rng = np.random.default_rng(seed)
    rho = 1.0 + rho_amp * rng.standard_normal((ny, nx))
    u = u_amp * rng.standard_normal((2, ny, nx))
    return rho, u


def random_noise(seed: int, shape, amp: float):
    """Multiplicative noise amp*N(0,1) used to push populations off equilibrium."""
    return amp * np.random.default_rng(seed).standard_normal(shape)


def random_force_field(seed: int, nx: int, ny: int, amp: float):
    """Per-node body force [2, ny, nx] with entries amp*N(0,1)."""
    return amp * np.random.default_rng(seed).standard_normal((2, ny, nx))


def fourier_modes_field(seed: int, n: int, modes: int = 16, amp: float = 0.02, kmax: int = 8):
    """Divergence-free random velocity field on an n x n periodic lattice made of
    `modes` Fourier modes of a stream function psi = sum_m A_m cos(2 pi (kx x + ky y)/n + phi_m),
    u = d psi/dy, v = -d psi/dx, integer wave vectors with 1 <= max(|kx|,|ky|) <= kmax and
    phases uniform in [0, 2 pi).  Each mode carries velocity amplitude `amp`; the sum is
    rescaled so that max |u| <= amp.  Returns u[2, n, n] (float64)."""
    rng = np.random.default_rng(seed)
    x = np.arange(n, dtype=np.float64)
    X, Y = np.meshgrid(x, x, indexing="xy")
    u = np.zeros((2, n, n))
    for _ in range(modes):
        while True:
            kx, ky = (int(v) for v in rng.integers(-kmax, kmax + 1, size=2))
            if 1 <= max(abs(kx), abs(ky)) <= kmax:
                break
        phi = rng.uniform(0.0, 2.0 * math.pi)
        kvec = 2.0 * math.pi * np.array([kx, ky]) / n
        knorm = float(np.hypot(*kvec))
        A = amp / knorm
        s = np.sin(kvec[0] * X + kvec[1] * Y + phi)
        u[0] += -A * kvec[1] * s
        u[1] += A * kvec[0] * s
    m = float(np.sqrt((u ** 2).sum(axis=0)).max())
    if m > amp:
        u *= amp / m
    return u


def batch_domains(seed: int = 20261202, count: int = 96, side_min: int = 64, side_max: int = 2048,
                  re_min: float = 100.0, re_max: float = 5000.0):
    """The batched ensemble: `count` independent square domains with sides drawn
    log-uniform in [side_min, side_max] (rounded), alternating lid-driven cavity
    (Re uniform in [re_min, re_max]) and Taylor-Green, storage alternating FP32 /
    FP16 deviations.  Returns a list of dicts (kind, side, re, store)."""
    rng = np.random.default_rng(seed)
    out = []
    for i in range(count):
        side = int(round(math.exp(rng.uniform(math.log(side_min), math.log(side_max)))))
        re = float(rng.uniform(re_min, re_max))
        out.append({
            "kind": "cavity" if i % 2 == 0 else "taylor_green",
            "side": side,
            "re": re,
            "store": "f32" if (i // 2) % 2 == 0 else "f16",
        })
    return out


def taylor_green_3d_init(n: int, u0: float, rho0: float = 1.0):
    """The three-dimensional Taylor-Green vortex on an n^3 periodic lattice:
    u = u0 sin(kx) cos(ky) cos(kz), v = -u0 cos(kx) sin(ky) cos(kz), w = 0,
    k = 2 pi / n, with the pressure of the incompressible solution,
    p = p0 + rho0 u0^2 / 16 (cos 2kx + cos 2ky)(cos 2kz + 2), and p = rho / 3.
    Returns rho[n, n, n] and u[3, n, n, n] (float64, axes z, y, x)."""
    k = 2.0 * math.pi / n
    c = np.arange(n, dtype=np.float64)
    Z, Y, X = np.meshgrid(c, c, c, indexing="ij")
    u = np.zeros((3, n, n, n))
    u[0] = u0 * np.sin(k * X) * np.cos(k * Y) * np.cos(k * Z)
    u[1] = -u0 * np.cos(k * X) * np.sin(k * Y) * np.cos(k * Z)
    rho = rho0 + 3.0 * rho0 * u0 * u0 / 16.0 * (np.cos(2 * k * X) + np.cos(2 * k * Y)) * (np.cos(2 * k * Z) + 2.0)
    return rho, u


def random_fields_3d(seed: int, nx: int, ny: int, nz: int, u_amp: float = 0.05, rho_amp: float = 0.02):
    """Uncorrelated random (rho, u) fields on an nx x ny x nz lattice (axes z, y, x)."""
    rng = np.random.default_rng(seed)
    rho = 1.0 + rho_amp * rng.standard_normal((nz, ny, nx))
    u = u_amp * rng.standard_normal((3, nz, ny, nx))
    return rho, u
