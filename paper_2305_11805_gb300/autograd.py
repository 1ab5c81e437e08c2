"""torch.autograd glue: energies and forces as a differentiable function of the network
parameters.

``PannaEnergyForces.apply(theta, pot, sysd)`` returns (E_cfg [C] FP64, F [N,3] FP32) from
the CUDA library; its backward maps upstream gradients (dL/dE_cfg, dL/dF) to dL/dtheta
with the library's hand-written reverse pass: the energy part is plain backpropagation
through the per-species networks, the force part is the double backward (descriptor JVP
along dL/dF, forward tangent through the networks, then the reverse pass), with the
descriptors recomputed instead of stored (Sec. II.A, on-the-fly descriptors).  Nothing
here computes anything itself: the arrays are only passed to the C ABI.
"""
from __future__ import annotations

import torch

from . import panna as P


class PannaEnergyForces(torch.autograd.Function):
    @staticmethod
    def forward(ctx, theta: torch.Tensor, pot: "P.Potential", sysd: "P.DeviceSystem"):
        if theta.dtype != torch.float32 or not theta.is_cuda:
            raise TypeError("theta must be a float32 CUDA tensor")
        theta_c = theta.detach().contiguous()
        E, _, F, _ = pot.energy_forces(sysd, theta_c, P.PANNA_MLP_FP32, virial=False, atom_energies=False)
        ctx.pot = pot
        ctx.sysd = sysd
        ctx.save_for_backward(theta_c)
        return E, F

    @staticmethod
    def backward(ctx, gE: torch.Tensor, gF: torch.Tensor):
        (theta,) = ctx.saved_tensors
        dE = None if gE is None else gE.detach().to(torch.float64).contiguous()
        dF = None if gF is None else gF.detach().to(torch.float32).contiguous()
        dtheta = ctx.pot.param_vjp(ctx.sysd, theta, dE, dF)
        return dtheta, None, None


def energy_forces(theta: torch.Tensor, pot: "P.Potential", sysd: "P.DeviceSystem"):
    """Differentiable (E_cfg, F) with respect to theta."""
    return PannaEnergyForces.apply(theta, pot, sysd)
