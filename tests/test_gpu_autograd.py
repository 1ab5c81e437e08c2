"""The torch.autograd.Function around the C ABI: a loss written in torch over (E, F)
back-propagates to the network parameters through the hand-written double backward, and
matches the FP64 oracle's gradient of the same loss."""
import numpy as np
import pytest

from oracle import oracle as O
from paper_2305_11805_gb300 import panna as P
from paper_2305_11805_gb300 import workloads as W
from tests import gpu_common as H

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def torch_cuda():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2305_11805_gb300 import build
    build.build()
    return torch


def test_autograd_energy_force_loss_gradient(torch_cuda):
    torch = torch_cuda
    from paper_2305_11805_gb300.autograd import energy_forces
    wl = W.make("molecules16")
    pot = P.Potential(wl.desc, wl.archs)
    sysd = P.DeviceSystem(wl.system)
    th32 = wl.theta.astype(np.float32)
    theta = torch.tensor(th32, device="cuda", requires_grad=True)
    E_ref = torch.as_tensor(wl.e_ref, dtype=torch.float64, device="cuda")
    F_ref = torch.as_tensor(wl.f_ref, dtype=torch.float32, device="cuda")
    E, F = energy_forces(theta, pot, sysd)
    loss = ((E - E_ref) ** 2).mean() + wl.w_force * ((F.double() - F_ref.double()) ** 2).mean()
    loss.backward()
    ref = O.batch(wl.system, wl.desc, wl.archs, th32.astype(np.float64), e_ref=wl.e_ref,
                  f_ref=wl.f_ref.astype(np.float32).astype(np.float64), w_force=wl.w_force, param_grad=True)
    assert abs(loss.item() - ref["loss"]) <= 1e-5 * abs(ref["loss"])
    errs = H.layer_errors(wl.archs, theta.grad.cpu().numpy().astype(np.float64), ref["dtheta"])
    assert max(errs) <= H.TOL_DTHETA, errs


def test_autograd_energy_only_and_force_only(torch_cuda):
    torch = torch_cuda
    from paper_2305_11805_gb300.autograd import energy_forces
    wl = W.make("ragged8")
    pot = P.Potential(wl.desc, wl.archs)
    sysd = P.DeviceSystem(wl.system)
    theta = torch.tensor(wl.theta.astype(np.float32), device="cuda", requires_grad=True)
    E, F = energy_forces(theta, pot, sysd)
    E.sum().backward()
    gE = theta.grad.clone()
    theta.grad = None
    E, F = energy_forces(theta, pot, sysd)
    (F ** 2).sum().backward()
    gF = theta.grad.clone()
    theta.grad = None
    E, F = energy_forces(theta, pot, sysd)
    (E.sum() + (F ** 2).sum()).backward()
    assert torch.allclose(theta.grad, gE + gF, rtol=1e-5, atol=1e-6 * float(theta.grad.abs().max()))


@pytest.mark.parametrize("name", ["molecules16", "ragged8", "diamond64"])
def test_autograd_positions_give_forces(torch_cuda, name):
    """-dE/dx through the autograd Function (backward = the descriptor adjoint) against the
    FP64 oracle's forces, a per-configuration upstream gradient, and central differences of
    the GPU energies themselves."""
    torch = torch_cuda
    from paper_2305_11805_gb300.autograd import energy
    wl = W.make(name)
    pot = P.Potential(wl.desc, wl.archs)
    sysd = P.DeviceSystem(wl.system)
    th32 = wl.theta.astype(np.float32)
    theta = torch.tensor(th32, device="cuda", requires_grad=True)
    pos = sysd.pos.clone().requires_grad_(True)
    E = energy(pos, theta, pot, sysd)
    E.sum().backward()
    ref = O.batch(wl.system, wl.desc, wl.archs, th32.astype(np.float64))
    ferr, rms = H.force_error(-pos.grad.cpu().numpy(), ref["F"])
    assert ferr <= H.TOL_F_FP32, ferr
    # per-configuration weights: dL/dx_i = w_c dE_c/dx_i
    w = torch.linspace(0.5, 2.0, sysd.n_cfg, dtype=torch.float64, device="cuda")
    pos.grad = None
    theta.grad = None
    (w * energy(pos, theta, pot, sysd)).sum().backward()
    cfg = np.repeat(np.arange(sysd.n_cfg), np.diff(wl.system.atom_off))
    want = -ref["F"] * w.cpu().numpy()[cfg][:, None]
    assert H.force_error(pos.grad.cpu().numpy(), want)[0] <= H.TOL_F_FP32
    # the parameter gradient of sum_c w_c E_c equals the VJP with dE = w
    g2 = pot.param_vjp(sysd, theta.detach(), w, None)
    assert torch.allclose(theta.grad, g2, rtol=1e-5, atol=1e-6 * float(g2.abs().max()))
    # central differences of the GPU energy along a few coordinates, against the same central
    # differences of the oracle's energy (the step's truncation error cancels; what remains is
    # the FP32 rounding of the atomic energies, divided by the step), and the difference quotient
    # against the analytic force
    import dataclasses
    rng = np.random.default_rng(0)
    h = 1e-2
    th64 = th32.astype(np.float64)
    for _ in range(4):
        a, k = int(rng.integers(sysd.n_atoms)), int(rng.integers(3))
        c = int(cfg[a])
        p1, p2 = pos.detach().clone(), pos.detach().clone()
        p1[a, k] += h
        p2[a, k] -= h
        with torch.no_grad():
            d = (energy(p1, theta, pot, sysd)[c] - energy(p2, theta, pot, sysd)[c]).item() / (2 * h)
        q1, q2 = wl.system.pos.copy(), wl.system.pos.copy()
        q1[a, k] += h
        q2[a, k] -= h
        E1 = O.batch(dataclasses.replace(wl.system, pos=q1), wl.desc, wl.archs, th64)["E_cfg"][c]
        E2 = O.batch(dataclasses.replace(wl.system, pos=q2), wl.desc, wl.archs, th64)["E_cfg"][c]
        d_ref = (E1 - E2) / (2 * h)
        a0, a1 = int(wl.system.atom_off[c]), int(wl.system.atom_off[c + 1])
        e_scale = float(np.abs(ref["E_atom"][a0:a1]).sum())
        assert abs(d - d_ref) <= 1e-6 * e_scale / h + 1e-5 * rms, (a, k, d, d_ref)
        scale = max(rms, abs(ref["F"][a, k]))
        assert abs(d_ref + ref["F"][a, k]) <= 1e-2 * scale, (a, k, d_ref, ref["F"][a, k])
