"""torch.autograd wrapper of the discrete adjoint.

``band_energy(uhat0, k_lo, k_hi, nsteps, ...)`` advances u_hat(0) by nsteps
fixed SSP-RK3 steps on the GPU and returns J = 1/2 sum_{k_lo <= |k| < k_hi}
|u_hat_k(T)|^2 over the full spectrum, evaluated by ns3d_band_energy; its
backward pass calls ns3d_grad_band_energy (the exact discrete adjoint,
checkpoint/recompute).  This module only marshals arguments: no step of the
observable or its gradient is computed here.

Gradient convention: for the D1 tensor of stored coefficients, PyTorch's
gradient of a real J is dJ/dRe z + i dJ/dIm z; the full-spectrum gradient g
of the adjoint enters with the multiplicity of each stored column (1 for
kz = 0 and N/2, 2 otherwise).
"""
from __future__ import annotations

import torch

from . import binding as B


def _weights(N: int, device):
    w = torch.full((N // 2 + 1,), 2.0, dtype=torch.float64, device=device)
    w[0] = 1.0
    w[-1] = 1.0
    return w


class BandEnergy(torch.autograd.Function):
    @staticmethod
    def forward(ctx, uhat0, plan, k_lo, k_hi, nsteps, checkpoint_every):
        plan.set_initial(0, uhat0.detach())
        plan.step(nsteps)
        J = plan.band_energy(0, k_lo, k_hi)
        plan.set_initial(0, uhat0.detach())          # the plan keeps u(0) for the backward
        ctx.plan, ctx.args = plan, (k_lo, k_hi, nsteps, checkpoint_every)
        return torch.tensor(J, dtype=torch.float64, device=uhat0.device)

    @staticmethod
    def backward(ctx, gJ):
        plan = ctx.plan
        k_lo, k_hi, nsteps, C = ctx.args
        g = plan.grad_band_energy(0, k_lo, k_hi, nsteps, C)
        w = _weights(plan.N[0], g.device).to(g.real.dtype)
        return (gJ.to(g.real.dtype) * w * g, None, None, None, None, None)


def band_energy(uhat0: torch.Tensor, k_lo: float, k_hi: float, nsteps: int, dt: float,
                dtype: int = B.NS3D_F64, checkpoint_every: int = 20, plan=None, **params):
    """J(u(T)) with an autograd backward through the discrete adjoint.  A
    one-member plan with fixed step dt is created unless one is given."""
    if plan is None:
        plan = B.Plan([uhat0.shape[-2]], dtype, dt_fixed=dt, **params)
    return BandEnergy.apply(uhat0, plan, k_lo, k_hi, nsteps, checkpoint_every)
