"""GPU parity of the standard Behler-Parrinello angular term (the second descriptor form of
Sec. II.A) through the C ABI against the oracle: descriptors, energies and forces (FP32 and
BF16 networks), virials, the training gradient (descriptor adjoint and JVP of the BP term),
the allocation-free descriptor entry point, and the argument checks."""
import dataclasses

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


def _case(name):
    if name == "ragged_edges_bp":
        # an empty configuration, a lone atom and a dimer between periodic boxes, 3 species
        base = W.make("ragged8")
        return W.bp_variant(dataclasses.replace(base, system=H.ragged_with_edges()), 1.0, 0.1)
    return W.make(name)


CASES = ["molecules16_bp", "water512_bp", "ragged_edges_bp"]


@pytest.mark.parametrize("name", CASES)
def test_bp_descriptors_match_oracle(torch_cuda, name):
    wl = _case(name)
    pot = P.Potential(wl.desc, wl.archs)
    G = pot.descriptors(P.DeviceSystem(wl.system)).cpu().numpy().astype(np.float64)
    ref = O.batch(wl.system, wl.desc, wl.archs, wl.theta, want_G=True)["G"]
    err = H.descriptor_error(G, ref, wl.desc)
    print("%s: D=%d, BP descriptors %.3g of the block maximum" % (name, wl.desc.D, err))
    assert err <= H.TOL_G


@pytest.mark.parametrize("name", CASES)
@pytest.mark.parametrize("prec", [P.PANNA_MLP_FP32, P.PANNA_MLP_BF16])
def test_bp_energy_forces_match_oracle(torch_cuda, name, prec):
    torch = torch_cuda
    wl = _case(name)
    if prec == P.PANNA_MLP_BF16 and wl.desc.D % 8:
        pytest.skip("BF16 networks need D % 8 == 0")
    pot = P.Potential(wl.desc, wl.archs)
    th32 = wl.theta.astype(np.float32)
    E, Ea, F, V = pot.energy_forces(P.DeviceSystem(wl.system), torch.as_tensor(th32, device="cuda"), prec)
    ref = O.batch(wl.system, wl.desc, wl.archs, th32.astype(np.float64))
    tol = H.TOL_F_FP32 if prec == P.PANNA_MLP_FP32 else H.TOL_F_BF16
    ferr = H.force_error(F.cpu().numpy().astype(np.float64), ref["F"])[0]
    escale = np.abs(ref["E_atom"]).sum()
    eerr = float(np.abs(E.cpu().numpy() - ref["E_cfg"]).max() / escale)
    verr = float(np.abs(V.cpu().numpy() - ref["virial"]).max() / max(np.abs(ref["virial"]).max(), 1e-30))
    print("%s prec %d: forces %.3g, energies %.3g, virial %.3g" % (name, prec, ferr, eerr, verr))
    assert ferr <= tol and eerr <= (H.TOL_E if prec == P.PANNA_MLP_FP32 else tol) and verr <= 10 * tol


@pytest.mark.parametrize("name", ["molecules16_bp", "water512_bp"])
def test_bp_training_gradient_matches_oracle(torch_cuda, name):
    torch = torch_cuda
    wl = _case(name)
    pot = P.Potential(wl.desc, wl.archs)
    th64 = wl.theta.astype(np.float32).astype(np.float64)
    base = O.batch(wl.system, wl.desc, wl.archs, th64)
    rng = np.random.default_rng(2)
    # labels off by O(1) per atom (as the other training tests): the energy residual of a
    # 512-atom box then dwarfs the FP32 rounding of its 512-term sum
    n = np.diff(wl.system.atom_off)
    e_ref = base["E_cfg"] + rng.normal(0.0, 0.2, size=wl.system.n_cfg) * n
    f_ref = (base["F"] + rng.normal(0.0, 0.3, size=base["F"].shape)).astype(np.float32).astype(np.float64)
    loss, g, E, F = pot.loss_grad(P.DeviceSystem(wl.system), torch.as_tensor(th64.astype(np.float32), device="cuda"),
                                  torch.as_tensor(e_ref, device="cuda"),
                                  torch.as_tensor(f_ref.astype(np.float32), device="cuda"), 0.5)
    ref = O.batch(wl.system, wl.desc, wl.archs, th64, e_ref=e_ref, f_ref=f_ref, w_force=0.5, param_grad=True)
    lerr = abs(loss.item() - ref["loss"]) / abs(ref["loss"])
    errs = H.layer_errors(wl.archs, g.cpu().numpy().astype(np.float64), ref["dtheta"])
    print("%s training step: loss %.3g, dtheta worst layer %.3g" % (name, lerr, max(errs)))
    assert lerr <= 1e-5 and max(errs) <= H.TOL_DTHETA


def test_bp_static_entry_point_and_store_rejection(torch_cuda):
    torch = torch_cuda
    wl = W.make("molecules16_bp")
    pot = P.Potential(wl.desc, wl.archs)
    sysd = P.DeviceSystem(wl.system)
    G1 = pot.descriptors(sysd)
    G2 = torch.empty_like(G1)
    P.panna_descriptors_static(wl.desc, sysd, G2)
    torch.cuda.synchronize()
    assert (G1 - G2).abs().max().item() <= 1e-6 * G1.abs().max().item()
    with pytest.raises(P.PannaError) as ei:
        P.panna_store_plan(pot.ctx, sysd)
    assert ei.value.status == P.PANNA_ERR_UNSUPPORTED


def test_bp_parameter_checks(torch_cuda):
    wl = W.make("molecules16_bp")
    for bad in (dict(bp_zeta=np.array([1.0, 0.5, 4.0, 4.0])), dict(bp_eta=np.array([-1.0, 0.1])),
                dict(bp_lambda=np.array([1.0, np.nan, 1.0, -1.0]))):
        d = dataclasses.replace(wl.desc, **bad)
        with pytest.raises(P.PannaError) as ei:
            P.Potential(d, wl.archs)
        assert ei.value.status == P.PANNA_ERR_INVALID_ARG
