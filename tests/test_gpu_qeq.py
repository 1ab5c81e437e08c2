"""GPU parity of the charge-equilibration path (Sec. II.B) through the C ABI against the
oracle: energies, atomic energies, charges and forces of NaCl clusters with a +1 total charge,
per-configuration total charges, edge cases (an empty configuration, a lone atom, a dimer)
and the argument checks."""
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


def _pot(wl):
    pot = P.Potential(wl.desc, wl.archs)
    P.panna_set_qeq(pot.ctx, wl.qeq["sigma"], wl.qeq["chi0"], wl.qeq["hard0"])
    return pot


def _compare(torch, wl, charge):
    pot = _pot(wl)
    sysd = P.DeviceSystem(wl.system)
    th32 = wl.theta.astype(np.float32)
    Q = None if charge is None else torch.as_tensor(charge, dtype=torch.float64, device="cuda")
    E, Ea, q, F = pot.qeq_energy_forces(sysd, torch.as_tensor(th32, device="cuda"), Q)
    ref = O.qeq_batch(wl.system, wl.desc, wl.archs, th32.astype(np.float64), wl.qeq, charge)
    escale = max(np.abs(ref["E_atom"]).sum(), 1e-30)
    errs = dict(
        E=float(np.abs(E.cpu().numpy() - ref["E_cfg"]).max() / escale),
        E_atom=float(np.abs(Ea.cpu().numpy() - ref["E_atom"]).max() / max(np.abs(ref["E_atom"]).max(), 1e-30)),
        q=float(np.abs(q.cpu().numpy() - ref["q"]).max()),
        F=H.force_error(F.cpu().numpy().astype(np.float64), ref["F"])[0])
    return errs, (E, Ea, q, F), ref


def test_qeq_clusters_match_oracle(torch_cuda):
    wl = W.make("nacl64")
    errs, out, ref = _compare(torch_cuda, wl, wl.charge)
    q = out[2].cpu().numpy()
    sums = np.add.reduceat(q, wl.system.atom_off[:-1])
    print("nacl64 (%d atoms): %s; total charges %.3g..%.3g" % (wl.system.n_atoms, errs, sums.min(), sums.max()))
    assert np.abs(sums - 1.0).max() <= 1e-9
    assert errs["E"] <= H.TOL_E and errs["E_atom"] <= 1e-5 and errs["q"] <= 1e-5 and errs["F"] <= H.TOL_F_FP32


def test_qeq_total_charges_and_neutral_default(torch_cuda):
    wl = W.make("nacl64")
    charge = np.array([(-1.0) ** c * (c % 3) for c in range(wl.system.n_cfg)])
    errs, out, _ = _compare(torch_cuda, wl, charge)
    print("per-configuration charges: %s" % errs)
    assert errs["E"] <= H.TOL_E and errs["q"] <= 1e-5 and errs["F"] <= H.TOL_F_FP32
    errs0, out0, _ = _compare(torch_cuda, wl, None)
    print("neutral: %s" % errs0)
    assert errs0["E"] <= H.TOL_E and errs0["q"] <= 1e-5 and errs0["F"] <= H.TOL_F_FP32
    sums = np.add.reduceat(out0[2].cpu().numpy(), wl.system.atom_off[:-1])
    assert np.abs(sums).max() <= 1e-9


def _with_edges(wl):
    s = wl.system
    parts = [(s.pos[:17], s.species[:17]), (np.zeros((0, 3)), np.zeros(0, np.int32)),
             (np.array([[1.0, 2.0, 3.0]]), np.array([1], np.int32)),
             (np.array([[0.0, 0.0, 0.0], [2.6, 0.3, -0.2]]), np.array([0, 1], np.int32)),
             (s.pos[17:33], s.species[17:33])]
    off = np.concatenate([[0], np.cumsum([len(p[1]) for p in parts])]).astype(np.int64)
    C = len(parts)
    wl.system = W.System(off, np.concatenate([p[0] for p in parts]), np.concatenate([p[1] for p in parts]),
                         np.zeros((C, 9)), np.zeros((C, 3), np.uint8), 2)
    return wl, np.array([1.0, 0.0, 0.5, 0.0, 1.0])


def test_qeq_edge_cases(torch_cuda):
    wl, charge = _with_edges(W.make("nacl2"))
    errs, out, ref = _compare(torch_cuda, wl, charge)
    q = out[2].cpu().numpy()
    print("empty / lone atom / dimer between clusters: %s; lone-atom charge %.6f" % (errs, q[17]))
    assert abs(q[17] - 0.5) <= 1e-12 and out[0][1].item() == 0.0
    assert errs["E"] <= H.TOL_E and errs["q"] <= 1e-5 and errs["F"] <= H.TOL_F_FP32


def test_qeq_repeat_calls_agree(torch_cuda):
    torch = torch_cuda
    wl = W.make("nacl64")
    pot = _pot(wl)
    sysd = P.DeviceSystem(wl.system)
    theta = torch.as_tensor(wl.theta.astype(np.float32), device="cuda")
    Q = torch.as_tensor(wl.charge, device="cuda")
    a = pot.qeq_energy_forces(sysd, theta, Q)
    b = pot.qeq_energy_forces(sysd, theta, Q)
    # (the flattened descriptor kernels sum in shared memory: equal up to rounding)
    assert (a[2] - b[2]).abs().max().item() <= 1e-6 and (a[1] - b[1]).abs().max().item() <= 1e-6 * a[1].abs().max().item()
    assert (a[3] - b[3]).abs().max().item() <= 1e-6 * a[3].abs().max().item()


def test_qeq_arguments(torch_cuda):
    torch = torch_cuda
    wl = W.make("nacl2")
    theta = torch.as_tensor(wl.theta.astype(np.float32), device="cuda")
    pot = P.Potential(wl.desc, wl.archs)
    sysd = P.DeviceSystem(wl.system)
    E = torch.empty(2, dtype=torch.float64, device="cuda")
    F = torch.empty((wl.system.n_atoms, 3), dtype=torch.float32, device="cuda")
    # constants not set yet
    with pytest.raises(P.PannaError) as ei:
        P.panna_qeq_energy_forces(pot.ctx, sysd, theta, None, E, None, None, F)
    assert ei.value.status == P.PANNA_ERR_INVALID_ARG
    with pytest.raises(P.PannaError) as ei:
        P.panna_set_qeq(pot.ctx, [0.0, 1.0], [1.0, 1.0], [1.0, 1.0])
    assert ei.value.status == P.PANNA_ERR_INVALID_ARG
    P.panna_set_qeq(pot.ctx, wl.qeq["sigma"], wl.qeq["chi0"], wl.qeq["hard0"])
    # 3-output networks do not serve the energy-only calls
    with pytest.raises(P.PannaError) as ei:
        pot.energy_forces(sysd, theta)
    assert ei.value.status == P.PANNA_ERR_UNSUPPORTED
    # periodic configurations and oversized ones are rejected
    s = wl.system
    per = P.DeviceSystem(W.System(s.atom_off, s.pos, s.species, np.tile((np.eye(3) * 30.0).reshape(1, 9), (2, 1)),
                                  np.ones((2, 3), np.uint8), 2))
    with pytest.raises(P.PannaError) as ei:
        P.panna_qeq_energy_forces(pot.ctx, per, theta, None, E, None, None, F)
    assert ei.value.status == P.PANNA_ERR_UNSUPPORTED
    rng = np.random.default_rng(0)
    big = W.System(np.array([0, 130], np.int64), rng.uniform(0, 30, (130, 3)), rng.integers(0, 2, 130).astype(np.int32),
                   np.zeros((1, 9)), np.zeros((1, 3), np.uint8), 2)
    Fb = torch.empty((130, 3), dtype=torch.float32, device="cuda")
    with pytest.raises(P.PannaError) as ei:
        P.panna_qeq_energy_forces(pot.ctx, P.DeviceSystem(big), theta, None, E[:1], None, None, Fb)
    assert ei.value.status == P.PANNA_ERR_UNSUPPORTED
    # a context with single-output networks has no charge equilibration
    one = W.make("molecules16")
    pot1 = P.Potential(one.desc, one.archs)
    with pytest.raises(P.PannaError) as ei:
        P.panna_set_qeq(pot1.ctx, [1.0] * 4, [1.0] * 4, [1.0] * 4)
    assert ei.value.status == P.PANNA_ERR_INVALID_ARG


@pytest.mark.parametrize("with_charges", [False, True])
def test_qeq_training_gradient_matches_oracle(torch_cuda, with_charges):
    torch = torch_cuda
    wl = W.make("nacl64")
    s = wl.system
    th32 = wl.theta.astype(np.float32)
    th64 = th32.astype(np.float64)
    base = O.qeq_batch(s, wl.desc, wl.archs, th64, wl.qeq, wl.charge)
    rng = np.random.default_rng(4)
    e_ref = base["E_cfg"] + rng.normal(0, 0.3, s.n_cfg) * np.diff(s.atom_off)
    f_ref = (base["F"] + rng.normal(0, 0.2, base["F"].shape)).astype(np.float32).astype(np.float64)
    q_ref = base["q"] + rng.normal(0, 0.05, s.n_atoms) if with_charges else None
    w_force, w_q = 0.7, 0.3
    ref = O.qeq_loss_grad(s, wl.desc, wl.archs, th64, wl.qeq, wl.charge, e_ref, f_ref, w_force, q_ref, w_q)
    pot = _pot(wl)
    dev = lambda a, dt=torch.float64: None if a is None else torch.as_tensor(a, dtype=dt, device="cuda")
    loss = torch.empty(1, dtype=torch.float64, device="cuda")
    g = torch.empty(pot.P, dtype=torch.float32, device="cuda")
    E = torch.empty(s.n_cfg, dtype=torch.float64, device="cuda")
    q = torch.empty(s.n_atoms, dtype=torch.float64, device="cuda")
    F = torch.empty((s.n_atoms, 3), dtype=torch.float32, device="cuda")
    P.panna_qeq_loss_grad(pot.ctx, P.DeviceSystem(s), torch.as_tensor(th32, device="cuda"), dev(wl.charge), dev(e_ref),
                          dev(f_ref, torch.float32), w_force, dev(q_ref), w_q, loss, g, E, q, F)
    lerr = abs(loss.item() - ref["loss"]) / abs(ref["loss"])
    errs = H.layer_errors(wl.archs, g.cpu().numpy().astype(np.float64), ref["dtheta"])
    ferr = H.force_error(F.cpu().numpy().astype(np.float64), ref["F"])[0]
    qerr = float(np.abs(q.cpu().numpy() - ref["q"]).max())
    print("qeq training step (charges %s): loss %.3g, dtheta worst layer %.3g, forces %.3g, charges %.3g" % (
        with_charges, lerr, max(errs), ferr, qerr))
    assert lerr <= 1e-5 and max(errs) <= H.TOL_DTHETA and ferr <= H.TOL_F_FP32 and qerr <= 1e-5


def test_qeq_nacl4096_sampled_clusters(torch_cuda):
    """The benchmark's batch (4096 clusters) in one call; the clusters are independent, so the
    oracle redoes a sample of them one by one."""
    torch = torch_cuda
    wl = W.make("nacl4096")
    s = wl.system
    pot = _pot(wl)
    th32 = wl.theta.astype(np.float32)
    E, Ea, q, F = pot.qeq_energy_forces(P.DeviceSystem(s), torch.as_tensor(th32, device="cuda"),
                                        torch.as_tensor(wl.charge, device="cuda"))
    E, q, F = E.cpu().numpy(), q.cpu().numpy(), F.cpu().numpy().astype(np.float64)
    rng = np.random.default_rng(9)
    cfgs = sorted(rng.choice(s.n_cfg, 24, replace=False).tolist())
    sub = s.subset(cfgs)
    ref = O.qeq_batch(sub, wl.desc, wl.archs, th32.astype(np.float64), wl.qeq, wl.charge[cfgs])
    rows = np.concatenate([np.arange(s.atom_off[c], s.atom_off[c + 1]) for c in cfgs])
    eerr = float(np.abs(E[cfgs] - ref["E_cfg"]).max() / np.abs(ref["E_atom"]).sum())
    qerr = float(np.abs(q[rows] - ref["q"]).max())
    ferr = float(np.abs(F[rows] - ref["F"]).max() / np.sqrt((F ** 2).mean()))
    sums = np.add.reduceat(q, s.atom_off[:-1])
    print("nacl4096 (%d atoms), 24 sampled clusters: energies %.3g, charges %.3g, forces %.3g; "
          "total charges within %.3g of +1" % (s.n_atoms, eerr, qerr, ferr, np.abs(sums - 1).max()))
    assert eerr <= H.TOL_E and qerr <= 1e-5 and ferr <= H.TOL_F_FP32 and np.abs(sums - 1).max() <= 1e-9
