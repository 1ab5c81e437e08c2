"""Pins of the oracle's charge-equilibration layer (Sec. II.B) against facts fixed by the
mathematics: the C oracle's pinned networks (column by column), the two-atom closed form,
the constraint and stationarity conditions, the point-charge limit of the Gaussian
interaction, central differences of the kernel and of the total energy (forces), and
rotation / permutation invariance."""
import math

import numpy as np
import pytest

from oracle import oracle as O
from paper_2305_11805_gb300 import workloads as W


def test_mlp_rows_columns_match_single_output_oracle():
    wl = W.make("nacl2")
    arch = wl.archs[1]
    off = W.param_offsets(wl.archs)
    th = wl.theta[off[1]:off[2]]
    rng = np.random.default_rng(0)
    X = rng.normal(size=(5, arch.widths[0]))
    out = O.mlp_rows(arch, th, X)
    last = sum(arch.widths[l + 1] * arch.widths[l] + arch.widths[l + 1] for l in range(arch.n_layers - 1))
    h = arch.widths[-2]
    one = W.MLPArch(arch.widths[:-1] + (1,), arch.acts)
    for k in range(3):
        thk = np.concatenate([th[:last], th[last + k * h:last + (k + 1) * h], th[last + 3 * h + k:last + 3 * h + k + 1]])
        seeds = np.zeros((5, 3))
        seeds[:, k] = 1.0
        _, g = O.mlp_rows(arch, th, X, seeds)
        for r in range(5):
            E, gr, _ = O.mlp(one, thk, X[r])
            assert abs(out[r, k] - E) < 1e-12 * max(1.0, abs(E))
            np.testing.assert_allclose(g[r], gr, rtol=1e-11, atol=1e-13)


def test_two_atoms_closed_form():
    pos = np.array([[0.0, 0.0, 0.0], [2.3, 0.4, -0.1]])
    sig, chi, J, Q = np.array([1.0, 1.3]), np.array([2.0, 7.5]), np.array([5.0, 9.0]), 0.4
    q, lam, K = O.qeq_solve(pos, sig, chi, J, Q)
    a11, a22, a12 = J[0] + K[0, 0], J[1] + K[1, 1], K[0, 1]
    q1 = (chi[1] - chi[0] + (a22 - a12) * Q) / (a11 + a22 - 2 * a12)
    assert abs(q[0] - q1) < 1e-12 and abs(q[1] - (Q - q1)) < 1e-12
    r = np.linalg.norm(pos[1] - pos[0])
    g = math.sqrt(2 * (1.0 + 1.3 ** 2))
    assert abs(K[0, 1] - O.KE_EV_A * math.erf(r / g) / r) < 1e-12
    assert abs(K[1, 1] - O.KE_EV_A / (1.3 * math.sqrt(math.pi))) < 1e-12


def test_constraint_stationarity_and_minimum():
    rng = np.random.default_rng(1)
    n = 7
    pos = rng.normal(size=(n, 3)) * 2.5
    sig = rng.uniform(0.8, 1.4, n)
    chi = rng.uniform(2.0, 8.0, n)
    J = rng.uniform(4.0, 10.0, n)
    q, lam, K = O.qeq_solve(pos, sig, chi, J, -1.0)
    assert abs(q.sum() + 1.0) < 1e-12
    grad = (np.diag(J) + K) @ q + chi
    np.testing.assert_allclose(grad, -lam * np.ones(n), atol=1e-10)

    def energy(qq):
        return chi @ qq + 0.5 * qq @ ((np.diag(J) + K) @ qq)
    e0 = energy(q)
    for _ in range(5):
        d = rng.normal(size=n)
        d -= d.mean()
        assert energy(q + 0.01 * d) > e0


def test_point_charge_limit_and_kernel_derivative():
    for r in (0.7, 2.0, 5.5):
        K, dK = O.qeq_kernel(r, 1e-4, 1e-4)
        assert abs(K - O.KE_EV_A / r) < 1e-12 * O.KE_EV_A / r
        assert abs(dK + O.KE_EV_A / r ** 2) < 1e-10 * O.KE_EV_A / r ** 2
        h = 1e-6
        fd = (O.qeq_kernel(r + h, 0.9, 1.3)[0] - O.qeq_kernel(r - h, 0.9, 1.3)[0]) / (2 * h)
        assert abs(fd - O.qeq_kernel(r, 0.9, 1.3)[1]) < 1e-7 * abs(fd)
    # short range: the Gaussian pair interaction stays finite, tending to 2 ke / (sqrt(pi) g)
    g = math.sqrt(2 * (0.9 ** 2 + 1.3 ** 2))
    assert abs(O.qeq_kernel(1e-6, 0.9, 1.3)[0] - 2 * O.KE_EV_A / (math.sqrt(math.pi) * g)) < 1e-6


def _energy(wl, pos):
    s = wl.system
    sysm = W.System(s.atom_off, pos, s.species, s.cell, s.pbc, s.n_species)
    return O.qeq_batch(sysm, wl.desc, wl.archs, wl.theta, wl.qeq, wl.charge)["E_cfg"].sum()


def test_forces_are_minus_energy_differences():
    wl = W.make("nacl2")
    ref = O.qeq_batch(wl.system, wl.desc, wl.archs, wl.theta, wl.qeq, wl.charge)
    np.testing.assert_allclose(ref["q"][:17].sum(), 1.0, atol=1e-12)
    h = 1e-5
    scale = np.abs(ref["F"]).max()
    for m in (0, 5, 20, 32):
        for c in range(3):
            p, n = wl.system.pos.copy(), wl.system.pos.copy()
            p[m, c] += h
            n[m, c] -= h
            fd = -(_energy(wl, p) - _energy(wl, n)) / (2 * h)
            assert abs(fd - ref["F"][m, c]) < 1e-6 * scale, (m, c, fd, ref["F"][m, c])


def test_rotation_and_permutation_invariance():
    wl = W.make("nacl2")
    s = wl.system
    ref = O.qeq_batch(s, wl.desc, wl.archs, wl.theta, wl.qeq, wl.charge)
    q_rot, _ = np.linalg.qr(np.random.default_rng(3).normal(size=(3, 3)))
    perm = np.concatenate([np.random.default_rng(4).permutation(17), 17 + np.arange(16)])
    pos = (s.pos @ q_rot.T)[perm]
    sysm = W.System(s.atom_off, pos, s.species[perm], s.cell, s.pbc, s.n_species)
    out = O.qeq_batch(sysm, wl.desc, wl.archs, wl.theta, wl.qeq, wl.charge)
    np.testing.assert_allclose(out["E_cfg"], ref["E_cfg"], rtol=1e-11)
    np.testing.assert_allclose(out["q"], ref["q"][perm], atol=1e-11)
    np.testing.assert_allclose(out["F"], (ref["F"] @ q_rot.T)[perm], atol=1e-10 * np.abs(ref["F"]).max())


def test_mlp_rows_train_matches_single_output_oracle():
    wl = W.make("nacl2")
    arch = wl.archs[0]
    off = W.param_offsets(wl.archs)
    th = wl.theta[off[0]:off[1]]
    rng = np.random.default_rng(5)
    X, Xd = rng.normal(size=(3, arch.widths[0])), rng.normal(size=(3, arch.widths[0]))
    last = sum(arch.widths[l + 1] * arch.widths[l] + arch.widths[l + 1] for l in range(arch.n_layers - 1))
    h = arch.widths[-2]
    one = W.MLPArch(arch.widths[:-1] + (1,), arch.acts)
    for k in range(3):
        seeds, tseeds = np.zeros((3, 3)), np.zeros((3, 3))
        seeds[:, k], tseeds[:, k] = 0.7, -1.3
        _, _, dth = O.mlp_rows_train(arch, th, X, Xd, seeds, tseeds)
        want = np.zeros(len(th))
        for r in range(3):
            thk = np.concatenate([th[:last], th[last + k * h:last + (k + 1) * h],
                                  th[last + 3 * h + k:last + 3 * h + k + 1]])
            _, _, d1 = O.mlp(one, thk, X[r], Xd[r], 0.7, -1.3, param_grad=True)
            want[:last] += d1[:last]
            want[last + k * h:last + (k + 1) * h] += d1[last:last + h]
            want[last + 3 * h + k] += d1[last + h]
        np.testing.assert_allclose(dth, want, rtol=1e-10, atol=1e-12 * np.abs(want).max())


def test_qeq_loss_gradient_central_differences():
    """Energy, force and charge terms together; the charges' response (the second solve) is a
    sizeable part of the gradient, so dropping it fails the comparison."""
    wl = W.make("nacl2")
    s = wl.system
    base = O.qeq_batch(s, wl.desc, wl.archs, wl.theta, wl.qeq, wl.charge)
    rng = np.random.default_rng(0)
    e_ref = base["E_cfg"] + rng.normal(0, 0.5, 2)
    f_ref = base["F"] + rng.normal(0, 0.2, base["F"].shape)
    q_ref = base["q"] + rng.normal(0, 0.05, s.n_atoms)
    args = (wl.qeq, wl.charge, e_ref, f_ref, 0.7, q_ref, 0.3)
    r = O.qeq_loss_grad(s, wl.desc, wl.archs, wl.theta, *args)
    off = W.param_offsets(wl.archs)
    arch = wl.archs[0]
    last = sum(arch.widths[l + 1] * arch.widths[l] + arch.widths[l + 1] for l in range(arch.n_layers - 1))
    picks = list(rng.choice(len(wl.theta), 10, replace=False))
    # the chi and J output rows of species 0 and 1 (where the charge response enters)
    picks += [off[0] + last + 15 + 3, off[0] + last + 30 + 4, off[1] + last + 15 + 1, off[1] + last + 30 + 7]
    h = 1e-6
    scale = np.abs(r["dtheta"]).max()
    for k in picks:
        tp, tm = wl.theta.copy(), wl.theta.copy()
        tp[k] += h
        tm[k] -= h
        fd = (O.qeq_loss_grad(s, wl.desc, wl.archs, tp, *args)["loss"] -
              O.qeq_loss_grad(s, wl.desc, wl.archs, tm, *args)["loss"]) / (2 * h)
        assert abs(fd - r["dtheta"][k]) <= 1e-6 * scale + 1e-5 * abs(fd), (k, fd, r["dtheta"][k])
    assert np.abs(r["mu"]).max() > 1e-3


def test_qeq_loss_without_labels_terms():
    """With labels equal to the predictions, only the charge term remains (and vanishes with it)."""
    wl = W.make("nacl2")
    s = wl.system
    base = O.qeq_batch(s, wl.desc, wl.archs, wl.theta, wl.qeq, wl.charge)
    r = O.qeq_loss_grad(s, wl.desc, wl.archs, wl.theta, wl.qeq, wl.charge, base["E_cfg"], base["F"], 0.5,
                        base["q"], 0.4)
    assert r["loss"] < 1e-20 and np.abs(r["dtheta"]).max() < 1e-10


def test_nacl_workload_shapes():
    """The clusters are those of the paper's NaCl experiment: Na9Cl8+ and Na8Cl8+ alternating,
    each with a total charge of +1, rock-salt distances (nearest neighbours near a/2)."""
    wl = W.make("nacl64")
    s = wl.system
    assert s.n_cfg == 64 and wl.desc.D == 45 and wl.archs[0].widths == (45, 15, 15, 3)
    for c in range(s.n_cfg):
        sp = s.species[s.atom_off[c]:s.atom_off[c + 1]]
        na, cl = int((sp == 0).sum()), int((sp == 1).sum())
        assert (na, cl) == ((9, 8) if c % 2 == 0 else (8, 8))
        x = s.pos[s.atom_off[c]:s.atom_off[c + 1]]
        d = np.linalg.norm(x[:, None] - x[None], axis=-1)[np.triu_indices(len(x), 1)]
        assert 2.2 < d.min() and abs(np.sort(d)[0:10].mean() - 2.82) < 0.3
    np.testing.assert_array_equal(wl.charge, np.ones(s.n_cfg))
    assert not s.pbc.any()
