"""GPU parity of the multi-rank building blocks through the C ABI: ghost atoms (the halo
of a slab decomposition) against the oracle's ghost mask, ranks emulated one after the
other on one GPU (independent launches; the exchange is done on the host) against the
whole configuration, and data-parallel training shards with the global loss normalisers.
"""
import dataclasses

import numpy as np
import pytest

from oracle import oracle as O
from paper_2305_11805_gb300 import domain as Dm
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


def _triclinic(system):
    shear = np.array([[1.0, 0.0, 0.0], [0.15, 1.0, 0.0], [0.1, -0.2, 1.0]])
    return dataclasses.replace(system, pos=system.pos @ shear,
                               cell=(system.cell.reshape(3, 3) @ shear).reshape(1, 9))


CASES = [("fcc256", True, 3), ("water512", False, 2)]


def _case(name, tri, world):
    wl = W.make(name)
    if tri:
        wl.system = _triclinic(wl.system)
    return wl, Dm.SlabPlan(wl.system, wl.desc.rc, world)


@pytest.mark.parametrize("name,tri,world", CASES)
@pytest.mark.parametrize("prec", [P.PANNA_MLP_FP32, P.PANNA_MLP_BF16])
def test_ghost_atoms_match_oracle_mask(torch_cuda, name, tri, world, prec):
    torch = torch_cuda
    wl, plan = _case(name, tri, world)
    pot = P.Potential(wl.desc, wl.archs)
    th32 = wl.theta.astype(np.float32)
    theta = torch.as_tensor(th32, device="cuda")
    tol = H.TOL_F_FP32 if prec == P.PANNA_MLP_FP32 else H.TOL_F_BF16
    # force scale: RMS of the physical force field (ghost rows hold partial sums only)
    whole = O.batch(wl.system, wl.desc, wl.archs, th32.astype(np.float64))
    rms = float(np.sqrt((whole["F"] ** 2).mean()))
    for d in plan.domains:
        sysd = P.DeviceSystem(d.system, ghost=d.ghost)
        E, Ea, F, V = pot.energy_forces(sysd, theta, prec)
        ref = O.batch(d.system, wl.desc, wl.archs, th32.astype(np.float64), ghost=d.ghost)
        Ea = Ea.cpu().numpy()
        assert not np.any(Ea[d.n_owned:]), "ghost atoms have no energy"
        escale = np.abs(ref["E_atom"]).sum()
        assert abs(E.item() - ref["E_cfg"][0]) <= 10 * tol * escale
        ferr = float(np.abs(F.cpu().numpy().astype(np.float64) - ref["F"]).max()) / rms
        verr = float(np.abs(V.cpu().numpy() - ref["virial"]).max() / np.abs(ref["virial"]).max())
        print("%s rank %d/%d prec %d: %d owned + %d ghosts, forces %.3g, virial %.3g" % (
            name, d.rank, world, prec, d.n_owned, d.ghost_src.size, ferr, verr))
        assert ferr <= tol and verr <= 10 * tol


@pytest.mark.parametrize("name,tri,world", CASES)
def test_ghost_descriptors_and_neighbours(torch_cuda, name, tri, world):
    torch = torch_cuda
    wl, plan = _case(name, tri, world)
    pot = P.Potential(wl.desc, wl.archs)
    d = plan.domains[-1]
    sysd = P.DeviceSystem(d.system, ghost=d.ghost)
    G = pot.descriptors(sysd).cpu().numpy().astype(np.float64)
    ref = O.batch(d.system, wl.desc, wl.archs, wl.theta, want_G=True, ghost=d.ghost)
    assert not np.any(G[d.n_owned:]), "ghost rows are zero"
    assert H.descriptor_error(G[:d.n_owned], ref["G"][:d.n_owned], wl.desc) <= 1e-5
    off, j, sh = pot.neighbors(sysd)
    off = off.cpu().numpy()
    assert np.all(np.diff(off)[d.n_owned:] == 0), "ghosts have empty neighbour lists"
    ii, jj, ss = O.neighbor_list(d.system, wl.desc.rc)
    keep = ii < d.n_owned
    want = H.sorted_pairs(ii[keep], jj[keep], ss[keep])
    got = H.sorted_pairs(np.repeat(np.arange(d.system.n_atoms), np.diff(off)), j.cpu().numpy(), sh.cpu().numpy())
    np.testing.assert_array_equal(got, want)


@pytest.mark.parametrize("name,tri,world", CASES)
def test_emulated_ranks_match_whole_configuration(torch_cuda, name, tri, world):
    torch = torch_cuda
    wl, plan = _case(name, tri, world)
    pot = P.Potential(wl.desc, wl.archs)
    th32 = wl.theta.astype(np.float32)
    theta = torch.as_tensor(th32, device="cuda")
    Fl, E, V = [], 0.0, 0.0
    for d in plan.domains:
        e, _, f, v = pot.energy_forces(P.DeviceSystem(d.system, ghost=d.ghost), theta)
        Fl.append(f.cpu().numpy().astype(np.float64))
        E += e.item()
        V = V + v.cpu().numpy()
    F = plan.gather_forces(Fl)
    ref = O.batch(wl.system, wl.desc, wl.archs, th32.astype(np.float64))
    Ew, _, Fw, Vw = pot.energy_forces(P.DeviceSystem(wl.system), theta)
    ferr = H.force_error(F, ref["F"])[0]
    fw = H.force_error(F, Fw.cpu().numpy().astype(np.float64))[0]
    escale = np.abs(ref["E_atom"]).sum()
    print("%s over %d ranks: forces vs oracle %.3g, vs one-GPU whole box %.3g, dE %.3g" % (
        name, world, ferr, fw, abs(E - ref["E_cfg"][0]) / escale))
    assert ferr <= H.TOL_F_FP32 and fw <= H.TOL_F_FP32
    assert abs(E - ref["E_cfg"][0]) <= H.TOL_E * escale and abs(E - Ew.item()) <= H.TOL_E * escale
    assert np.abs(V - ref["virial"]).max() <= 10 * H.TOL_F_FP32 * np.abs(ref["virial"]).max()


def test_param_vjp_with_ghosts_adds_up_to_oracle(torch_cuda):
    # The oracle's loss gradient with E_ref = E - dE C / 2, F_ref = F - dF 3N / (2 w) has
    # seeds (dE, dF), so it is the vector-Jacobian product for any chosen (dE, dF).
    torch = torch_cuda
    wl, plan = _case("fcc256", True, 3)
    th32 = wl.theta.astype(np.float32)
    th64 = th32.astype(np.float64)
    rng = np.random.default_rng(5)
    N = wl.system.n_atoms
    full = O.batch(wl.system, wl.desc, wl.archs, th64)
    dE = np.array([0.7])
    dF = rng.normal(size=(N, 3)).astype(np.float32).astype(np.float64) * 0.01
    w = 0.5
    ref = O.batch(wl.system, wl.desc, wl.archs, th64, e_ref=full["E_cfg"] - dE / 2.0,
                  f_ref=full["F"] - dF * 3 * N / (2 * w), w_force=w, param_grad=True)
    pot = P.Potential(wl.desc, wl.archs)
    theta = torch.as_tensor(th32, device="cuda")
    g = 0.0
    for d in plan.domains:
        rows = np.concatenate([d.owned, d.ghost_src])
        g = g + pot.param_vjp(P.DeviceSystem(d.system, ghost=d.ghost), theta,
                              torch.as_tensor(dE, device="cuda"),
                              torch.as_tensor(dF[rows].astype(np.float32), device="cuda")).cpu().numpy()
    errs = H.layer_errors(wl.archs, np.asarray(g, np.float64), ref["dtheta"])
    print("vjp over 3 ranks with ghosts: worst layer %.3g" % max(errs))
    assert max(errs) <= H.TOL_DTHETA


def test_sharded_training_with_global_normalisers(torch_cuda):
    torch = torch_cuda
    wl = W.make("molecules1024")
    s = wl.system
    th32 = wl.theta.astype(np.float32)
    theta = torch.as_tensor(th32, device="cuda")
    pot = P.Potential(wl.desc, wl.archs)
    world = 4
    b = Dm.shard_bounds(Dm.estimated_costs(s, wl.desc.rc), world)
    P.panna_set_loss_normalization(pot.ctx, s.n_cfg, s.n_atoms)
    loss, g = 0.0, 0.0
    for r in range(world):
        cfgs = list(range(b[r], b[r + 1]))
        a0, a1 = s.atom_off[b[r]], s.atom_off[b[r + 1]]
        l, gr, _, _ = pot.loss_grad(P.DeviceSystem(s.subset(cfgs)), theta,
                                    torch.as_tensor(wl.e_ref[cfgs], device="cuda"),
                                    torch.as_tensor(wl.f_ref[a0:a1], dtype=torch.float32, device="cuda"),
                                    wl.w_force)
        loss += l.item()
        g = g + gr.cpu().numpy().astype(np.float64)
    P.panna_set_loss_normalization(pot.ctx, 0, 0)
    ref = O.batch(s, wl.desc, wl.archs, th32.astype(np.float64), e_ref=wl.e_ref,
                  f_ref=wl.f_ref.astype(np.float32).astype(np.float64), w_force=wl.w_force, param_grad=True)
    errs = H.layer_errors(wl.archs, g, ref["dtheta"])
    lerr = abs(loss - ref["loss"]) / ref["loss"]
    print("molecules1024 in %d shards %s: loss %.3g, dtheta worst layer %.3g" % (world, np.diff(b).tolist(), lerr,
                                                                             max(errs)))
    assert lerr <= 1e-5 and max(errs) <= H.TOL_DTHETA


def test_normaliser_arguments_and_ghost_training_rejected(torch_cuda):
    torch = torch_cuda
    wl, plan = _case("fcc256", False, 2)
    pot = P.Potential(wl.desc, wl.archs)
    for bad in ((0, 5), (3, 0), (-1, -1)):
        with pytest.raises(P.PannaError) as ei:
            P.panna_set_loss_normalization(pot.ctx, *bad)
        assert ei.value.status == P.PANNA_ERR_INVALID_ARG
    d = plan.domains[0]
    sysd = P.DeviceSystem(d.system, ghost=d.ghost)
    theta = torch.as_tensor(wl.theta.astype(np.float32), device="cuda")
    with pytest.raises(P.PannaError) as ei:
        pot.loss_grad(sysd, theta, torch.zeros(1, dtype=torch.float64, device="cuda"),
                      torch.zeros((d.system.n_atoms, 3), dtype=torch.float32, device="cuda"), 0.1)
    assert ei.value.status == P.PANNA_ERR_UNSUPPORTED
