"""Parity at the full sizes of the paper-shaped workloads, in the call the benchmark times.

Large configurations are checked on sampled atoms that the oracle computes one by one
(neighbour list bit for bit, descriptor, atomic energy, force), and through properties
that hold at any size (sum of forces, agreement of the BF16 and FP32 network paths).
The 1024-molecule training step is small enough for the oracle to redo in full.
"""
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


def _sampled_check(torch, wl, cfg, samples, prec, ftol, pot=None, sysd=None, out=None):
    s = wl.system
    pot = pot or P.Potential(wl.desc, wl.archs)
    sysd = sysd or P.DeviceSystem(s)
    theta = torch.as_tensor(wl.theta.astype(np.float32), device="cuda")
    if out is None:
        out = pot.energy_forces(sysd, theta, prec)
    E, Ea, F, V = out
    a0 = int(s.atom_off[cfg])
    ref = O.sampled(s, cfg, wl.desc, wl.archs, wl.theta.astype(np.float32).astype(np.float64), samples)
    Fg = F[a0 + np.asarray(samples)].cpu().numpy().astype(np.float64)
    Eg = Ea[a0 + np.asarray(samples)].cpu().numpy().astype(np.float64)
    rms = float(np.sqrt((F.double() ** 2).mean().item()))
    ferr = float(np.abs(Fg - ref["F"]).max() / rms)
    eerr = float(np.abs(Eg - ref["E"]).max() / np.abs(ref["E"]).max())
    return ferr, eerr, ref, out


def _neighbors_of(pot, sysd):
    off, j, sh = pot.neighbors(sysd)
    return off.cpu().numpy(), j.cpu().numpy(), sh.cpu().numpy()


def test_water32k_bf16_and_fp32(torch_cuda):
    torch = torch_cuda
    wl = W.make("water32k")
    pot = P.Potential(wl.desc, wl.archs)
    sysd = P.DeviceSystem(wl.system)
    rng = np.random.default_rng(0)
    smp = sorted(rng.choice(wl.system.n_atoms, 24, replace=False).tolist())
    ferr, eerr, ref, out16 = _sampled_check(torch, wl, 0, smp, P.PANNA_MLP_BF16, H.TOL_F_BF16, pot, sysd)
    theta = torch.as_tensor(wl.theta.astype(np.float32), device="cuda")
    out32 = pot.energy_forces(sysd, theta, P.PANNA_MLP_FP32)
    ferr32, eerr32, _, _ = _sampled_check(torch, wl, 0, smp, P.PANNA_MLP_FP32, H.TOL_F_FP32, pot, sysd, out32)
    rms = float(np.sqrt((out32[2].double() ** 2).mean().item()))
    d16 = float((out16[2] - out32[2]).abs().max().item()) / rms
    print("water32k: BF16 sampled max|dF|/rms %.3g, E %.3g; FP32 %.3g, E %.3g; BF16 vs FP32 all atoms %.3g" % (
        ferr, eerr, ferr32, eerr32, d16))
    assert ferr <= H.TOL_F_BF16 and ferr32 <= H.TOL_F_FP32 and d16 <= H.TOL_F_BF16
    assert eerr <= H.TOL_F_BF16 and eerr32 <= 10 * H.TOL_E
    # neighbour lists of the sampled atoms, bit for bit
    off, j, sh = _neighbors_of(pot, sysd)
    for q, m in enumerate(smp):
        n = int(ref["nnb"][q])
        got = H.sorted_pairs(np.full(off[m + 1] - off[m], m), j[off[m]:off[m + 1]], sh[off[m]:off[m + 1]])
        want = H.sorted_pairs(np.full(n, m), ref["nb_j"][q, :n].astype(np.int64), ref["nb_shift"][q, :n])
        np.testing.assert_array_equal(got, want)


def test_fcc1m_bf16(torch_cuda):
    torch = torch_cuda
    wl = W.make("fcc1m")
    pot = P.Potential(wl.desc, wl.archs)
    sysd = P.DeviceSystem(wl.system)
    rng = np.random.default_rng(1)
    smp = sorted(rng.choice(wl.system.n_atoms, 24, replace=False).tolist())
    ferr, eerr, ref, out = _sampled_check(torch, wl, 0, smp, P.PANNA_MLP_BF16, H.TOL_F_BF16, pot, sysd)
    F = out[2].double()
    rms = float(np.sqrt((F ** 2).mean().item()))
    fsum = float(F.sum(0).abs().max().item()) / (rms * np.sqrt(wl.system.n_atoms))
    # descriptors of the sampled atoms (plain FP32 angular form in this mode -> compare the
    # allocating descriptor entry point, extended precision)
    G = pot.descriptors(sysd)[torch.as_tensor(smp, device="cuda")].cpu().numpy().astype(np.float64)
    gerr = H.descriptor_error(G, ref["G"], wl.desc)
    print("fcc1m: BF16 sampled max|dF|/rms %.3g, atom E %.3g, |sum F|/(rms sqrt N) %.3g, G %.3g" % (
        ferr, eerr, fsum, gerr))
    assert ferr <= H.TOL_F_BF16 and eerr <= H.TOL_F_BF16
    assert fsum <= 1e-3
    assert gerr <= 1e-5
    off, j, sh = _neighbors_of(pot, sysd)
    for q, m in enumerate(smp):
        n = int(ref["nnb"][q])
        got = H.sorted_pairs(np.full(off[m + 1] - off[m], m), j[off[m]:off[m + 1]], sh[off[m]:off[m + 1]])
        want = H.sorted_pairs(np.full(n, m), ref["nb_j"][q, :n].astype(np.int64), ref["nb_shift"][q, :n])
        np.testing.assert_array_equal(got, want)


def test_ragged4096_bf16(torch_cuda):
    torch = torch_cuda
    wl = W.make("ragged4096")
    s = wl.system
    pot = P.Potential(wl.desc, wl.archs)
    sysd = P.DeviceSystem(s)
    theta = torch.as_tensor(wl.theta.astype(np.float32), device="cuda")
    out = pot.energy_forces(sysd, theta, P.PANNA_MLP_BF16)
    E = out[0].cpu().numpy()
    sizes = np.diff(s.atom_off)
    rng = np.random.default_rng(2)
    # whole configurations: the smallest ones (several periodic images per neighbour) in full
    small = np.argsort(sizes)[:4].tolist()
    sub = s.subset(small)
    full = O.batch(sub, wl.desc, wl.archs, wl.theta.astype(np.float32).astype(np.float64))
    eerr = float(np.abs(E[small] - full["E_cfg"]).max() / np.abs(full["E_atom"]).sum())
    Fsub = np.concatenate([out[2][int(s.atom_off[c]):int(s.atom_off[c + 1])].cpu().numpy() for c in small])
    fsmall = H.force_error(Fsub.astype(np.float64), full["F"])[0]
    # sampled atoms in a few large configurations
    worst = 0.0
    for c in rng.choice(np.nonzero(sizes > 1000)[0], 3, replace=False).tolist():
        smp = sorted(rng.choice(int(sizes[c]), 6, replace=False).tolist())
        ferr, aerr, _, _ = _sampled_check(torch, wl, c, smp, P.PANNA_MLP_BF16, H.TOL_F_BF16, pot, sysd, out)
        worst = max(worst, ferr, aerr)
    print("ragged4096 (%d atoms): small configs dE %.3g dF %.3g; sampled atoms worst %.3g" % (
        s.n_atoms, eerr, fsmall, worst))
    assert eerr <= H.TOL_F_BF16 and fsmall <= H.TOL_F_BF16 and worst <= H.TOL_F_BF16


def test_molecules1024_training_step(torch_cuda):
    torch = torch_cuda
    wl = W.make("molecules1024")
    pot = P.Potential(wl.desc, wl.archs)
    sysd = P.DeviceSystem(wl.system)
    th32 = wl.theta.astype(np.float32)
    loss, g, E, F = pot.loss_grad(sysd, torch.as_tensor(th32, device="cuda"),
                                  torch.as_tensor(wl.e_ref, device="cuda"),
                                  torch.as_tensor(wl.f_ref, dtype=torch.float32, device="cuda"), wl.w_force)
    ref = O.batch(wl.system, wl.desc, wl.archs, th32.astype(np.float64), e_ref=wl.e_ref,
                  f_ref=wl.f_ref.astype(np.float32).astype(np.float64), w_force=wl.w_force, param_grad=True)
    lerr = abs(loss.item() - ref["loss"]) / abs(ref["loss"])
    errs = H.layer_errors(wl.archs, g.cpu().numpy().astype(np.float64), ref["dtheta"])
    ferr = H.force_error(F.cpu().numpy().astype(np.float64), ref["F"])[0]
    eerr = float(np.abs(E.cpu().numpy() - ref["E_cfg"]).max() / np.abs(ref["E_atom"]).sum())
    print("molecules1024: loss %.3g, dtheta worst layer %.3g, forces %.3g, energies %.3g" % (
        lerr, max(errs), ferr, eerr))
    assert lerr <= 1e-5 and max(errs) <= H.TOL_DTHETA
    assert ferr <= H.TOL_F_FP32 and eerr <= H.TOL_E
