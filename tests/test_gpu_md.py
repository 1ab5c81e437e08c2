"""GPU parity of the Langevin dynamics loop (panna_md_run) with the oracle's BAOAB
trajectory, neighbour-list reuse against a search every step, batched replicas, and energy
conservation of the deterministic limit."""
import math

import numpy as np
import pytest

from oracle import oracle as O
from paper_2305_11805_gb300 import panna as P
from paper_2305_11805_gb300 import workloads as W

pytestmark = pytest.mark.gpu

ACC = 9.648533212e-3
KB = 8.617333262e-5
MASS = [12.011]


@pytest.fixture(scope="module")
def torch_cuda():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2305_11805_gb300 import build
    build.build()
    return torch


def _start(wl, T, seed=5):
    rng = np.random.default_rng(seed)
    v = rng.normal(0.0, math.sqrt(KB * T * ACC / MASS[0]), size=(wl.system.n_atoms, 3))
    for c in range(wl.system.n_cfg):
        a0, a1 = wl.system.atom_off[c], wl.system.atom_off[c + 1]
        v[a0:a1] -= v[a0:a1].mean(0)
    return v


def _run(torch, wl, v0, n_steps, dt, T, gam, skin, seed=11, prec=P.PANNA_MLP_FP32):
    pot = P.Potential(wl.desc, wl.archs)
    sysd = P.DeviceSystem(wl.system)
    theta = torch.as_tensor(wl.theta.astype(np.float32), device="cuda")
    vel = torch.as_tensor(v0, dtype=torch.float64, device="cuda").contiguous()
    F = torch.zeros((wl.system.n_atoms, 3), dtype=torch.float32, device="cuda")
    E = torch.zeros(wl.system.n_cfg, dtype=torch.float64, device="cuda")
    Et = torch.zeros((max(n_steps, 1), wl.system.n_cfg), dtype=torch.float64, device="cuda")
    nb = P.panna_md_run(pot.ctx, sysd, vel, theta, prec, dt, T, gam, skin, MASS, seed, 0, n_steps, F, False, E, Et)
    torch.cuda.synchronize()
    return dict(pos=sysd.pos.cpu().numpy(), vel=vel.cpu().numpy(), F=F.cpu().numpy().astype(np.float64),
                E=E.cpu().numpy(), E_traj=Et.cpu().numpy()[:n_steps], builds=nb)


def test_langevin_trajectory_matches_oracle(torch_cuda):
    wl = W.make("carbon16")
    v0 = _start(wl, 300.0)
    th32 = wl.theta.astype(np.float32).astype(np.float64)
    n, dt, T, gam = 20, 0.5, 300.0, 0.02
    got = _run(torch_cuda, wl, v0, n, dt, T, gam, skin=0.5)
    ref = O.md_baoab(wl.system, wl.desc, wl.archs, th32, v0, MASS, dt, T, gam, 11, 0, n)
    dx = np.abs(got["pos"] - ref["pos"]).max()
    dv = np.abs(got["vel"] - ref["vel"]).max() / np.sqrt((ref["vel"] ** 2).mean())
    dF = np.abs(got["F"] - ref["F"]).max() / np.sqrt((ref["F"] ** 2).mean())
    dE = np.abs(got["E_traj"] - ref["E_traj"]).max() / np.abs(ref["E_traj"]).max()
    print("carbon16, %d BAOAB steps: max|dx| %.3g A, max|dv|/rms %.3g, forces %.3g, energies %.3g, searches %d"
          % (n, dx, dv, dF, dE, got["builds"]))
    assert dx <= 1e-5 and dv <= 1e-4 and dF <= 2e-5 and dE <= 1e-5
    assert got["builds"] <= 2


def test_verlet_reuse_matches_search_every_step(torch_cuda):
    wl = W.make("carbon16")
    v0 = _start(wl, 300.0)
    n = 50
    a = _run(torch_cuda, wl, v0, n, 0.5, 300.0, 0.02, skin=1.0)
    b = _run(torch_cuda, wl, v0, n, 0.5, 300.0, 0.02, skin=0.0)
    print("skin 1.0: %d searches, skin 0: %d searches, max|dx| %.3g" % (
        a["builds"], b["builds"], np.abs(a["pos"] - b["pos"]).max()))
    assert b["builds"] == n + 1 and a["builds"] < n // 5
    assert np.abs(a["pos"] - b["pos"]).max() <= 1e-6
    assert np.abs(a["E_traj"] - b["E_traj"]).max() <= 1e-6 * np.abs(b["E_traj"]).max()


def test_batched_replicas_follow_their_own_trajectories(torch_cuda):
    wl = W.make("carbon16x64")
    v0 = _start(wl, 300.0)
    th32 = wl.theta.astype(np.float32).astype(np.float64)
    n = 4
    got = _run(torch_cuda, wl, v0, n, 0.5, 300.0, 0.02, skin=0.5)
    ref = O.md_baoab(wl.system, wl.desc, wl.archs, th32, v0, MASS, 0.5, 300.0, 0.02, 11, 0, n)
    dx = np.abs(got["pos"] - ref["pos"]).max()
    dE = np.abs(got["E_traj"] - ref["E_traj"]).max() / np.abs(ref["E_traj"]).max()
    print("64 replicas x 16 atoms, %d steps: max|dx| %.3g, energies %.3g" % (n, dx, dE))
    assert dx <= 1e-5 and dE <= 1e-5
    # replicas start from different displacements and draw different noise
    e = got["E_traj"][-1]
    assert len(np.unique(np.round(e, 9))) == len(e)


def test_deterministic_limit_conserves_energy(torch_cuda):
    wl = W.make("carbon16")
    v0 = _start(wl, 600.0)
    n, dt = 200, 0.25
    got = _run(torch_cuda, wl, v0, n, dt, 0.0, 0.0, skin=0.5)
    ekin0 = 0.5 * MASS[0] * (v0 ** 2).sum() / ACC
    e0 = O.batch(wl.system, wl.desc, wl.archs, wl.theta.astype(np.float32).astype(np.float64))["E_cfg"].sum() + ekin0
    ekin = 0.5 * MASS[0] * (got["vel"] ** 2).sum() / ACC
    drift = abs(got["E"].sum() + ekin - e0)
    print("velocity Verlet, %d steps of %.2f fs: |E_tot - E_0| %.3g eV (E_kin0 %.3g eV), searches %d" % (
        n, dt, drift, ekin0, got["builds"]))
    assert drift <= 2e-3 * ekin0


def test_dynamics_arguments(torch_cuda):
    torch = torch_cuda
    wl = W.make("carbon16")
    pot = P.Potential(wl.desc, wl.archs)
    sysd = P.DeviceSystem(wl.system)
    theta = torch.as_tensor(wl.theta.astype(np.float32), device="cuda")
    vel = torch.zeros((16, 3), dtype=torch.float64, device="cuda")
    F = torch.zeros((16, 3), dtype=torch.float32, device="cuda")
    E = torch.zeros(1, dtype=torch.float64, device="cuda")
    for dt, T, gam, skin, mass in ((0.0, 300.0, 0.01, 0.5, MASS), (0.5, -1.0, 0.01, 0.5, MASS),
                                   (0.5, 300.0, 0.01, -0.1, MASS), (0.5, 300.0, 0.01, 0.5, [0.0])):
        with pytest.raises(P.PannaError) as ei:
            P.panna_md_run(pot.ctx, sysd, vel, theta, 0, dt, T, gam, skin, mass, 1, 0, 1, F, False, E)
        assert ei.value.status == P.PANNA_ERR_INVALID_ARG
    ghost = P.DeviceSystem(wl.system, ghost=np.zeros(16, np.uint8))
    with pytest.raises(P.PannaError) as ei:
        P.panna_md_run(pot.ctx, ghost, vel, theta, 0, 0.5, 300.0, 0.01, 0.5, MASS, 1, 0, 1, F, False, E)
    assert ei.value.status == P.PANNA_ERR_UNSUPPORTED
