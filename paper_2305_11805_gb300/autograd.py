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


class PannaEnergy(torch.autograd.Function):
    """Per-configuration energies as a differentiable function of the atomic positions (and of
    the network parameters).  The forward pass is one panna_energy_forces call: descriptors,
    networks, and the descriptor adjoint, which turns g = dE/dG into the forces
    F = -dE/dx without materialising dG/dx (Sec. II).  The adjoint is linear in g, so the
    gradient of any loss L(E) with respect to the positions, dL/dx_i = (dL/dE_c) dE_c/dx_i =
    -(dL/dE_c) F_i for the configuration c of atom i, is the adjoint's output scaled per
    configuration; the parameter gradient is the library's reverse pass through the networks.
    First derivatives only (a loss on the forces goes through PannaEnergyForces instead)."""

    @staticmethod
    def forward(ctx, pos: torch.Tensor, theta: torch.Tensor, pot: "P.Potential", sysd: "P.DeviceSystem",
                prec: int):
        if pos.dtype != torch.float64 or not pos.is_cuda or pos.shape != (sysd.n_atoms, 3):
            raise TypeError("pos must be a float64 CUDA tensor of shape [n_atoms, 3]")
        if theta.dtype != torch.float32 or not theta.is_cuda:
            raise TypeError("theta must be a float32 CUDA tensor")
        pos_c = pos.detach().contiguous()
        theta_c = theta.detach().contiguous()
        s = P.DeviceSystem.from_tensors(sysd.atom_off, pos_c, sysd.species, sysd.cell, sysd.pbc, sysd.ghost)
        E, _, F, _ = pot.energy_forces(s, theta_c, prec, virial=False, atom_energies=False)
        cfg = torch.repeat_interleave(torch.arange(sysd.n_cfg, device=pos.device),
                                      torch.diff(sysd.atom_off))
        ctx.pot, ctx.sys = pot, s
        ctx.save_for_backward(theta_c, F, cfg)
        return E

    @staticmethod
    def backward(ctx, gE: torch.Tensor):
        theta, F, cfg = ctx.saved_tensors
        g = gE.detach().to(torch.float64)
        gpos = -(g[cfg].unsqueeze(1) * F.double()) if ctx.needs_input_grad[0] else None
        gth = ctx.pot.param_vjp(ctx.sys, theta, g.contiguous(), None) if ctx.needs_input_grad[1] else None
        return gpos, gth, None, None, None


def energy(pos: torch.Tensor, theta: torch.Tensor, pot: "P.Potential", sysd: "P.DeviceSystem",
           prec: int = P.PANNA_MLP_FP32):
    """Differentiable E_cfg with respect to the positions pos [n_atoms, 3] (FP64) and theta:
    -d(E.sum())/dpos are the forces.  sysd supplies the species, cells, periodic flags and
    configuration offsets; its own positions are not read."""
    return PannaEnergy.apply(pos, theta, pot, sysd, prec)
