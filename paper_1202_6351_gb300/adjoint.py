"""Differentiable cascaded run: a torch.autograd.Function over lbm_adjoint_run.

``final_velocity_loss(u0, force, omega_shear, target, nsteps, every)`` returns
L = 1/2 sum |u(T) - target|^2 for a periodic cascaded lattice started at the
transformed equilibrium with velocity u0 (rho = rho0), driven by the per-node
body force ``force`` [2, ny, nx], with shear rate omega_4 = omega_5 =
``omega_shear`` and the other rates fixed.  Its backward pass returns the
gradients the CUDA adjoint computed in the same call (reverse streaming plus
the transposed collision, checkpoints every ``every`` steps, FP64
accumulation).  All tensors are float64 on the current CUDA device.
"""
from __future__ import annotations

import torch

from . import lbm


class FinalVelocityLoss(torch.autograd.Function):
    @staticmethod
    def forward(ctx, u0, force, omega_shear, target, nsteps, every, other_rates, store):
        ny, nx = u0.shape[1], u0.shape[2]
        w = float(omega_shear)
        rates = (other_rates[0], w, w, other_rates[1], other_rates[2], other_rates[3])
        stream = torch.cuda.current_stream().cuda_stream
        with lbm.Lattice(nx, ny, rates, model=lbm.CASCADED, store=store, stream=stream) as L:
            L.set_force_field(force.detach().contiguous())
            loss, gu, gf, gom = L.adjoint_run(nsteps, every, u0.detach().contiguous(), target.detach().contiguous())
        ctx.save_for_backward(gu, gf)
        # tied shear rate: omega_4 and omega_5 both follow omega_shear
        ctx.g_omega = float(gom[1] + gom[2])
        return torch.tensor(loss, dtype=torch.float64, device=u0.device)

    @staticmethod
    def backward(ctx, g):
        gu, gf = ctx.saved_tensors
        g_omega = torch.tensor(ctx.g_omega, dtype=torch.float64, device=g.device)
        return g * gu, g * gf, g * g_omega, None, None, None, None, None


def final_velocity_loss(u0, force, omega_shear, target, nsteps, every=100, other_rates=(1.0, 1.0, 1.0, 1.0),
                        store=lbm.F32):
    """other_rates = (omega_3, omega_6, omega_7, omega_8)."""
    if not torch.is_tensor(omega_shear):
        omega_shear = torch.tensor(float(omega_shear), dtype=torch.float64, device=u0.device)
    return FinalVelocityLoss.apply(u0, force, omega_shear, target, int(nsteps), int(every), tuple(other_rates),
                                   int(store))
