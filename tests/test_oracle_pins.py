"""Pins of the FP64 oracle against facts fixed by the paper and by mathematics.

Each test checks the oracle against something other than itself: sizes printed in the
paper, crystallographic shell counts, closed forms of dimers / trimers / undisplaced
lattices, independent brute force, symmetry (invariance), library routines (numpy) and
central finite differences.  A plausible slip anywhere in the oracle (a dropped term,
a wrong sign or index, a transposed operand, a wrong block offset) fails one of them.
"""
import itertools
import math
import os

import numpy as np
import pytest

from oracle import oracle as O
from paper_2305_11805_gb300 import workloads as W

GOLD = os.path.join(os.path.dirname(__file__), "golden")


def _desc(S=1, rc=4.6, n_rad=8, n_theta=4, n_ang=3, eta_r=4.0, eta_a=3.0, zeta=6.0, eps=1e-6):
    return W.descriptor_params(S, rc, n_rad, n_theta, n_ang, eta_rad=eta_r, eta_ang=eta_a,
                               zeta=zeta, eps_theta=eps)


def _fc(r, rc):
    return 0.5 * (1.0 + math.cos(math.pi * r / rc)) if r < rc else 0.0


def _sys(pos, species, cell=None, pbc=(0, 0, 0), S=1):
    pos = np.asarray(pos, np.float64).reshape(-1, 3)
    n = len(pos)
    cell = np.zeros(9) if cell is None else np.asarray(cell, np.float64).reshape(9)
    return W.System(np.array([0, n], np.int64), pos, np.asarray(species, np.int32),
                    cell.reshape(1, 9), np.asarray(pbc, np.uint8).reshape(1, 3), S)


# ------------------------------------------------------------------ layout / sizes

def test_descriptor_sizes_printed_in_paper():
    rows = [l.split() for l in open(os.path.join(GOLD, "descriptor_sizes.txt"))
            if l.strip() and not l.startswith("#")]
    assert len(rows) == 4
    for r in rows:
        S, nr, nt, na, D = map(int, r[:5])
        d = W.descriptor_params(S, 5.0, nr, nt, na)
        assert O.descriptor_size(d) == D, r


# ------------------------------------------------------------------ cutoff + radial

def test_cutoff_function_properties():
    # smooth cosine cutoff: 1 at r=0, 1/2 at rc/2, 0 with zero slope at rc, 0 beyond.
    d = _desc(rc=4.0, n_rad=1)
    d.rs_rad = np.array([0.0])
    d.eta_rad = 0.0  # Gaussian factor 1: G = f_c(r)
    for r, want in [(1e-9, 1.0), (2.0, 0.5), (4.0 - 1e-9, 0.0), (4.5, 0.0)]:
        G = O.center(d, [[r, 0, 0]], [0], jacobian=False)
        assert abs(G[0] - want) < 1e-8
    G1 = O.center(d, [[3.999, 0, 0]], [0], jacobian=False)[0]
    G2 = O.center(d, [[3.998, 0, 0]], [0], jacobian=False)[0]
    assert G1 < 1e-5 and G2 < 1e-4 and abs((G1 - G2) / 1e-3) < 1e-2  # slope -> 0


@pytest.mark.parametrize("r", [0.7, 1.9, 2.5, 4.1, 4.59])
def test_dimer_radial_closed_form(r):
    # Two species; centre species 0, neighbour species 1: only radial block 1 is filled,
    # with exp(-eta (r - Rs_n)^2) f_c(r); every angular entry is zero (no pair).
    d = _desc(S=2, rc=4.6, n_rad=16, eta_r=16.0)
    sysm = _sys([[0, 0, 0], [0.3 * r, -0.4 * r, math.sqrt(0.75) * r]], [0, 1], S=2)
    out = O.batch(sysm, d, [W._mlp(d.D, (4,))] * 2, np.zeros(2 * W._mlp(d.D, (4,)).n_params),
                  want_G=True)
    G0 = out["G"][0]
    want = np.zeros(d.D)
    for n, rs in enumerate(d.rs_rad):
        want[16 + n] = math.exp(-16.0 * (r - rs) ** 2) * _fc(r, 4.6)
    np.testing.assert_allclose(G0, want, rtol=1e-13, atol=1e-15)
    # the other atom sees species 0 in radial block 0
    np.testing.assert_allclose(out["G"][1][:16], want[16:32], rtol=1e-13, atol=1e-15)


def test_undisplaced_fcc_radial_shell_sum():
    # FCC, a = 4.05: shells of 12 at a/sqrt2, 6 at a, 24 at a*sqrt(3/2) inside rc=5.0
    a, rc = 4.05, 5.0
    pos = W.FCC_BASIS * a
    d = _desc(rc=rc, n_rad=12, eta_r=2.0)
    sysm = _sys(pos, [0] * 4, np.eye(3) * a, (1, 1, 1))
    G = O.batch(sysm, d, [W._mlp(d.D, (2,))], np.zeros(W._mlp(d.D, (2,)).n_params),
                want_G=True)["G"]
    shells = [(12, a / math.sqrt(2)), (6, a), (24, a * math.sqrt(1.5))]
    want = [sum(c * math.exp(-2.0 * (r - rs) ** 2) * _fc(r, rc) for c, r in shells)
            for rs in d.rs_rad]
    for i in range(4):
        np.testing.assert_allclose(G[i, :12], want, rtol=1e-12)


# ------------------------------------------------------------------ angular

def _trimer(r1, r2, theta, phi=0.3):
    e1 = np.array([math.cos(phi), math.sin(phi), 0.0])
    e2 = np.array([-math.sin(phi), math.cos(phi), 0.0])
    return [[0, 0, 0], list(r1 * e1), list(r2 * (math.cos(theta) * e1 + math.sin(theta) * e2))]


@pytest.mark.parametrize("theta", [0.4, 1.3, math.pi / 2, 2.2, 3.0])
def test_trimer_angular_closed_form_eps0(theta):
    # eps = 0: the angular factor is exactly (1 + cos(theta - theta_m)) with theta the
    # geometric angle; species (centre 0, neighbours 1 and 2 of a 3-species system) put
    # the single pair term in block {1,2}.
    S, rc, r1, r2, zeta = 3, 4.6, 1.7, 2.9, 6.0
    d = _desc(S=S, rc=rc, n_rad=4, n_theta=5, n_ang=3, eta_a=3.0, zeta=zeta, eps=0.0)
    pos = _trimer(r1, r2, theta)
    G = O.center(d, np.array(pos[1:]), [1, 2], jacobian=False)
    block = 1 * 3 - 0 + (2 - 1)   # upper-triangle index of {1,2} for S=3 -> 4
    assert block == 4
    off = S * 4 + block * 5 * 3
    fcp = _fc(r1, rc) * _fc(r2, rc)
    want = np.zeros(d.D)
    for m, tm in enumerate(d.theta_s):
        for n, rs in enumerate(d.rs_ang):
            want[off + m * 3 + n] = (2.0 ** (1 - zeta) * (1 + math.cos(theta - tm)) ** zeta
                                     * math.exp(-3.0 * ((r1 + r2) / 2 - rs) ** 2) * fcp)
    for n, rs in enumerate(d.rs_rad):
        want[1 * 4 + n] = math.exp(-4.0 * (r1 - rs) ** 2) * _fc(r1, rc)
        want[2 * 4 + n] = math.exp(-4.0 * (r2 - rs) ** 2) * _fc(r2, rc)
    np.testing.assert_allclose(G, want, rtol=1e-12, atol=1e-300)


def test_trimer_special_angles():
    # theta = pi (opposite neighbours): at theta_m = pi the factor 2^(1-zeta)(1+1)^zeta = 2;
    # at theta_m = 0 it is 0.  theta = pi/2 with theta_m = pi/2 also gives 2.
    d = _desc(S=1, rc=5.0, n_rad=2, n_theta=3, n_ang=1, eta_a=0.0, zeta=8.0, eps=0.0)
    d.rs_ang = np.array([0.0])
    r = 2.0
    for theta, m_peak, m_zero in [(math.pi, 2, 0), (math.pi / 2, 1, None)]:
        pos = _trimer(r, r, theta)
        G = O.center(d, np.array(pos[1:]), [0, 0], jacobian=False)
        ang = G[2:]
        assert abs(ang[m_peak] - 2.0 * _fc(r, 5.0) ** 2) < 1e-12
        if m_zero is not None:
            assert abs(ang[m_zero]) < 1e-15


def test_trimer_eps_reading():
    # eps > 0 replaces sin(theta) by sqrt(sin^2 theta + eps) in cos(theta - theta_m).
    eps, theta, zeta = 1e-3, 1.1, 4.0
    d = _desc(S=1, rc=5.0, n_rad=1, n_theta=4, n_ang=1, eta_a=0.0, zeta=zeta, eps=eps)
    d.rs_ang = np.array([0.0])
    pos = _trimer(1.5, 2.5, theta)
    G = O.center(d, np.array(pos[1:]), [0, 0], jacobian=False)[1:]
    f = _fc(1.5, 5.0) * _fc(2.5, 5.0)
    for m, tm in enumerate(d.theta_s):
        c = math.cos(theta) * math.cos(tm) + math.sqrt(math.sin(theta) ** 2 + eps) * math.sin(tm)
        assert abs(G[m] - 2 ** (1 - zeta) * (1 + c) ** zeta * f) < 1e-13


def test_angular_pairs_counted_once_and_images_distinct():
    # A single atom in a small periodic cube: its neighbours are its own images (6 at
    # L, 12 at L*sqrt2); every unordered pair of distinct image entries contributes once,
    # which a brute-force enumeration in numpy reproduces.
    L, rc = 3.0, 4.5
    d = _desc(S=1, rc=rc, n_rad=2, n_theta=3, n_ang=2, eta_a=0.5, zeta=2.0, eps=0.0)
    sysm = _sys([[0.1, 0.2, 0.3]], [0], np.eye(3) * L, (1, 1, 1))
    G = O.batch(sysm, d, [W._mlp(d.D, (2,))], np.zeros(W._mlp(d.D, (2,)).n_params),
                want_G=True)["G"][0]
    vecs = [np.array(n) * L for n in itertools.product(range(-2, 3), repeat=3)
            if 0 < np.linalg.norm(np.array(n) * L) < rc]
    assert len(vecs) == 6 + 12
    want = np.zeros(d.D)
    for a, b in itertools.combinations(vecs, 2):
        ra, rb = np.linalg.norm(a), np.linalg.norm(b)
        th = math.acos(np.clip(a @ b / (ra * rb), -1, 1))
        for m, tm in enumerate(d.theta_s):
            for n, rs in enumerate(d.rs_ang):
                want[2 + m * 2 + n] += (0.5 * (1 + math.cos(th - tm)) ** 2
                                        * math.exp(-0.5 * ((ra + rb) / 2 - rs) ** 2)
                                        * _fc(ra, rc) * _fc(rb, rc))
    np.testing.assert_allclose(G[2:], want[2:], rtol=1e-11, atol=1e-14)


# ------------------------------------------------------------------ neighbour lists

def _count_lattice(n_basis_pos, cell, rc):
    """independent brute force in numpy: neighbour entries of atom 0 in a periodic cell"""
    cnt = 0
    for n in itertools.product(range(-4, 5), repeat=3):
        sh = np.array(n) @ cell
        for p in n_basis_pos:
            r = np.linalg.norm(p + sh - n_basis_pos[0])
            if 0 < r < rc:
                cnt += 1
    return cnt


def test_shell_counts_fcc_diamond():
    a = 4.05
    sysm = _sys(W.FCC_BASIS * a, [0] * 4, np.eye(3) * a, (1, 1, 1))
    i, j, s = O.neighbor_list(sysm, 5.0)
    assert np.all(np.bincount(i) == 42)  # 12 + 6 + 24
    a = 5.43
    sysm = _sys(W.DIAMOND_BASIS * a, [0] * 8, np.eye(3) * a, (1, 1, 1))
    i, j, s = O.neighbor_list(sysm, 4.6)
    assert np.all(np.bincount(i) == 28)  # 4 + 12 + 12
    # single atom in a cube of side 2 with rc 4.5: integer vectors with 0 < |n|^2 < 5.0625
    sysm = _sys([[0.5, 0.5, 0.5]], [0], np.eye(3) * 2.0, (1, 1, 1))
    i, j, s = O.neighbor_list(sysm, 4.5)
    assert len(i) == 6 + 12 + 8 + 6 + 24
    assert _count_lattice(np.array([[0.5, 0.5, 0.5]]), np.eye(3) * 2.0, 4.5) == len(i)


def _rel_vectors(sysm, rc):
    i, j, s = O.neighbor_list(sysm, rc)
    cell = sysm.cell[0].reshape(3, 3)
    rv = sysm.pos[j] + s @ cell - sysm.pos[i]
    return i, j, s, rv


def test_neighbors_vs_numpy_brute_force_triclinic():
    rng = np.random.default_rng(3)
    cell = np.array([[5.0, 0.0, 0.0], [1.7, 4.6, 0.0], [-0.9, 1.1, 5.3]])
    frac = rng.uniform(0, 1, (9, 3))
    pos = frac @ cell
    rc = 4.7
    sysm = _sys(pos, [0] * 9, cell, (1, 1, 1))
    i, j, s, rv = _rel_vectors(sysm, rc)
    got = sorted(zip(i.tolist(), j.tolist(), map(tuple, s.tolist())))
    want = []
    for ii in range(9):
        for jj in range(9):
            for n in itertools.product(range(-4, 5), repeat=3):
                if ii == jj and n == (0, 0, 0):
                    continue
                r = np.linalg.norm(pos[jj] + np.array(n) @ cell - pos[ii])
                if r < rc:
                    want.append((ii, jj, n))
    assert got == sorted(want)


def test_neighbors_equivalent_cell_and_unwrapped_positions():
    # Same lattice spanned by a sheared basis, atoms moved by lattice vectors: the
    # multiset of relative vectors per atom is unchanged.
    rng = np.random.default_rng(5)
    cell = np.eye(3) * 7.0
    pos = rng.uniform(0, 7.0, (12, 3))
    rc = 5.2
    sysm = _sys(pos, [0] * 12, cell, (1, 1, 1))
    i, _, _, rv = _rel_vectors(sysm, rc)
    cell2 = np.array([cell[0], cell[1] + cell[0], cell[2] - 2 * cell[1]])
    pos2 = pos + rng.integers(-3, 4, (12, 3)) @ cell
    sysm2 = _sys(pos2, [0] * 12, cell2, (1, 1, 1))
    i2, _, _, rv2 = _rel_vectors(sysm2, rc)
    for a in range(12):
        A = np.round(rv[i == a], 9)
        B = np.round(rv2[i2 == a], 9)
        assert sorted(map(tuple, A.tolist())) == sorted(map(tuple, B.tolist()))


def test_neighbors_non_periodic_brute_force():
    rng = np.random.default_rng(7)
    pos = rng.uniform(-4, 4, (15, 3))
    sysm = _sys(pos, [0] * 15)
    i, j, s = O.neighbor_list(sysm, 3.5)
    want = [(a, b) for a in range(15) for b in range(15)
            if a != b and np.linalg.norm(pos[a] - pos[b]) < 3.5]
    assert list(zip(i.tolist(), j.tolist())) == want
    assert not np.any(s)


# ------------------------------------------------------------------ invariance

def _small_periodic(seed=0):
    wl = W.make("ragged8", seed)
    return wl, wl.system.subset([0])


def test_invariance_rotation_translation_permutation():
    wl, sysm = _small_periodic()
    base = O.batch(sysm, wl.desc, wl.archs, wl.theta, want_G=True)
    rng = np.random.default_rng(11)
    q, _ = np.linalg.qr(rng.normal(size=(3, 3)))
    if np.linalg.det(q) < 0:
        q[:, 0] *= -1
    rot = W.System(sysm.atom_off, sysm.pos @ q.T + np.array([0.3, -1.2, 2.5]), sysm.species,
                   (sysm.cell.reshape(3, 3) @ q.T).reshape(1, 9), sysm.pbc, sysm.n_species)
    out = O.batch(rot, wl.desc, wl.archs, wl.theta, want_G=True)
    np.testing.assert_allclose(out["G"], base["G"], rtol=1e-10, atol=1e-12)
    np.testing.assert_allclose(out["E_cfg"], base["E_cfg"], rtol=1e-12)
    np.testing.assert_allclose(out["F"], base["F"] @ q.T, atol=1e-10 * np.abs(base["F"]).max())
    perm = rng.permutation(sysm.n_atoms)
    per = W.System(sysm.atom_off, sysm.pos[perm], sysm.species[perm], sysm.cell, sysm.pbc,
                   sysm.n_species)
    out = O.batch(per, wl.desc, wl.archs, wl.theta, want_G=True)
    np.testing.assert_allclose(out["G"], base["G"][perm], rtol=1e-12, atol=1e-13)
    np.testing.assert_allclose(out["F"], base["F"][perm], atol=1e-12 * np.abs(base["F"]).max())
    np.testing.assert_allclose(out["E_cfg"], base["E_cfg"], rtol=1e-12)


# ------------------------------------------------------------------ network (Eq. 1)

def test_mlp_matches_numpy_chain():
    rng = np.random.default_rng(1)
    arch = W.MLPArch((7, 5, 4, 1), (W.ACT_GAUSSIAN, W.ACT_TANH, W.ACT_LINEAR))
    th = rng.normal(size=arch.n_params)
    x = rng.normal(size=7)
    E, g, _ = O.mlp(arch, th, x)
    W1 = th[:35].reshape(5, 7); b1 = th[35:40]
    W2 = th[40:60].reshape(4, 5); b2 = th[60:64]
    W3 = th[64:68].reshape(1, 4); b3 = th[68:69]
    h1 = np.exp(-(W1 @ x + b1) ** 2)
    h2 = np.tanh(W2 @ h1 + b2)
    assert abs(E - float((W3 @ h2 + b3)[0])) < 1e-13
    # ReLU path
    arch2 = W.MLPArch((7, 5, 1), (W.ACT_RELU, W.ACT_LINEAR))
    th2 = rng.normal(size=arch2.n_params)
    E2, _, _ = O.mlp(arch2, th2, x)
    h = np.maximum(th2[:35].reshape(5, 7) @ x + th2[35:40], 0)
    assert abs(E2 - float(th2[40:45] @ h + th2[45])) < 1e-13


def test_mlp_single_unit_closed_form():
    arch = W.MLPArch((1, 1, 1), (W.ACT_GAUSSIAN, W.ACT_LINEAR))
    w1, b1, w2, b2 = 0.7, -0.2, 1.3, 0.4
    x = 0.9
    E, g, _ = O.mlp(arch, np.array([w1, b1, w2, b2]), np.array([x]))
    z = w1 * x + b1
    assert abs(E - (w2 * math.exp(-z * z) + b2)) < 1e-15
    assert abs(g[0] - w2 * (-2 * z) * math.exp(-z * z) * w1) < 1e-15


def test_mlp_input_and_param_gradients_fd():
    rng = np.random.default_rng(2)
    arch = W.MLPArch((6, 5, 3, 1), (W.ACT_GAUSSIAN, W.ACT_TANH, W.ACT_LINEAR))
    th = rng.normal(size=arch.n_params) * 0.7
    x = rng.normal(size=6)
    xd = rng.normal(size=6)
    E, g, _ = O.mlp(arch, th, x)
    h = 1e-6
    gfd = np.array([(O.mlp(arch, th, x + h * e)[0] - O.mlp(arch, th, x - h * e)[0]) / (2 * h)
                    for e in np.eye(6)])
    np.testing.assert_allclose(g, gfd, rtol=1e-7, atol=1e-9)
    alpha, beta = 0.8, -1.3
    _, _, dth = O.mlp(arch, th, x, xd, alpha, beta, param_grad=True)

    def phi(t):
        e, gg, _ = O.mlp(arch, t, x)
        return alpha * e + beta * gg @ xd
    fd = np.array([(phi(th + h * e) - phi(th - h * e)) / (2 * h) for e in np.eye(len(th))])
    np.testing.assert_allclose(dth, fd, rtol=1e-6, atol=1e-8)


# ------------------------------------------------------------------ derivatives

def test_descriptor_jacobian_fd():
    rng = np.random.default_rng(4)
    d = _desc(S=2, rc=4.0, n_rad=5, n_theta=4, n_ang=3, eta_r=3.0, eta_a=2.0, zeta=6.0, eps=1e-6)
    rv = rng.normal(size=(6, 3)) * 1.4
    sp = np.array([0, 1, 1, 0, 1, 0], np.int32)
    G, J = O.center(d, rv, sp)
    h = 1e-6
    for e in range(6):
        for c in range(3):
            dr = np.zeros_like(rv); dr[e, c] = h
            fd = (O.center(d, rv + dr, sp, jacobian=False) - O.center(d, rv - dr, sp, jacobian=False)) / (2 * h)
            np.testing.assert_allclose(J[:, e, c], fd, rtol=1e-6, atol=1e-9)


def _energy(sysm, wl):
    return O.batch(sysm, wl.desc, wl.archs, wl.theta)["E_cfg"].sum()


@pytest.mark.parametrize("name", ["diamond64", "ragged8"])
def test_forces_central_differences(name):
    wl = W.make(name)
    sysm = wl.system.subset([0]) if wl.system.n_cfg > 1 else wl.system
    out = O.batch(sysm, wl.desc, wl.archs, wl.theta)
    F = out["F"]
    assert np.sqrt((F ** 2).mean()) > 0.05
    np.testing.assert_allclose(F.sum(0), 0.0, atol=1e-10 * np.abs(F).max())
    h = 1e-5
    rng = np.random.default_rng(0)
    for m in rng.choice(sysm.n_atoms, 3, replace=False):
        for c in range(3):
            p = sysm.pos.copy(); p[m, c] += h
            ep = _energy(W.System(sysm.atom_off, p, sysm.species, sysm.cell, sysm.pbc, sysm.n_species), wl)
            p[m, c] -= 2 * h
            em = _energy(W.System(sysm.atom_off, p, sysm.species, sysm.cell, sysm.pbc, sysm.n_species), wl)
            assert abs(-(ep - em) / (2 * h) - F[m, c]) < 1e-6 * np.abs(F).max()


def test_virial_strain_fd():
    wl, sysm = _small_periodic(1)
    out = O.batch(sysm, wl.desc, wl.archs, wl.theta)
    Wv = out["virial"][0]
    np.testing.assert_allclose(Wv, Wv.T, atol=1e-10 * np.abs(Wv).max())
    h = 1e-6
    cell = sysm.cell.reshape(3, 3)
    for a in range(3):
        for b in range(3):
            eps = np.zeros((3, 3)); eps[a, b] = h
            vals = []
            for sgn in (1, -1):
                Fm = np.eye(3) + sgn * eps
                s2 = W.System(sysm.atom_off, sysm.pos @ Fm.T, sysm.species,
                              (cell @ Fm.T).reshape(1, 9), sysm.pbc, sysm.n_species)
                vals.append(_energy(s2, wl))
            assert abs(-(vals[0] - vals[1]) / (2 * h) - Wv[a, b]) < 1e-6 * np.abs(Wv).max()


def test_loss_parameter_gradient_fd():
    # Full energy + force loss of a small training batch; gradient vs central FD of the
    # oracle loss on a random subset of parameters of every layer and species.
    wl = W.make("molecules16")
    sysm = wl.system.subset([0, 1, 2])
    d = W.descriptor_params(4, 5.2, 6, 3, 2)
    archs = [W._mlp(d.D, (5, 3)) for _ in range(4)]
    rng = np.random.default_rng(9)
    theta = W.init_weights(rng, d, archs, 2.0, 2.0)
    e_ref = rng.normal(size=3)
    f_ref = rng.normal(size=(sysm.n_atoms, 3))
    out = O.batch(sysm, d, archs, theta, e_ref=e_ref, f_ref=f_ref, w_force=0.1, param_grad=True)
    g = out["dtheta"]
    assert np.abs(g).max() > 1e-3
    h = 1e-6
    present = set(sysm.species.tolist())
    off = W.param_offsets(archs)
    idx = []
    for s in present:
        idx += list(rng.choice(np.arange(off[s], off[s + 1]), 12, replace=False))
    for k in idx:
        tp = theta.copy(); tp[k] += h
        tm = theta.copy(); tm[k] -= h
        lp = O.batch(sysm, d, archs, tp, e_ref=e_ref, f_ref=f_ref, w_force=0.1)["loss"]
        lm = O.batch(sysm, d, archs, tm, e_ref=e_ref, f_ref=f_ref, w_force=0.1)["loss"]
        assert abs((lp - lm) / (2 * h) - g[k]) < 1e-6 * max(1.0, abs(g[k])) + 1e-7 * np.abs(g).max(), k
    # species absent from the batch get exactly zero gradient
    for s in set(range(4)) - present:
        assert not np.any(g[off[s]:off[s + 1]])


def test_ghost_mask_partial_sum_and_forces_fd():
    # Atoms flagged ghost are neighbours only (the halo of a spatial decomposition): the
    # energy is the sum of the OTHER atoms' energies of the unmasked evaluation, the forces
    # are minus its derivative on every atom, ghosts included (central differences), and
    # they still sum to zero (the partial sum is translation invariant).
    wl, sysm = _small_periodic(1)
    full = O.batch(sysm, wl.desc, wl.archs, wl.theta)
    rng = np.random.default_rng(4)
    ghost = (rng.random(sysm.n_atoms) < 0.4).astype(np.uint8)
    assert 0 < ghost.sum() < sysm.n_atoms
    out = O.batch(sysm, wl.desc, wl.archs, wl.theta, ghost=ghost)
    assert not np.any(out["E_atom"][ghost == 1])
    np.testing.assert_allclose(out["E_atom"][ghost == 0], full["E_atom"][ghost == 0], rtol=1e-13)
    assert abs(out["E_cfg"][0] - full["E_atom"][ghost == 0].sum()) < 1e-10 * np.abs(full["E_atom"]).sum()
    F = out["F"]
    np.testing.assert_allclose(F.sum(0), 0.0, atol=1e-10 * np.abs(F).max())
    h = 1e-5
    for m in [int(np.nonzero(ghost)[0][0]), int(np.nonzero(ghost == 0)[0][0])]:
        for c in range(3):
            vals = []
            for sgn in (1, -1):
                p = sysm.pos.copy(); p[m, c] += sgn * h
                s2 = W.System(sysm.atom_off, p, sysm.species, sysm.cell, sysm.pbc, sysm.n_species)
                vals.append(O.batch(s2, wl.desc, wl.archs, wl.theta, ghost=ghost)["E_cfg"].sum())
            assert abs(-(vals[0] - vals[1]) / (2 * h) - F[m, c]) < 1e-6 * np.abs(F).max(), (m, c)


def test_loss_normalisers_closed_form_and_fd():
    # A shard of a larger batch normalises its loss terms by the global counts (C', N'):
    # L = sum_c (E_c - E_ref)^2 / C' + w sum (F - F_ref)^2 / (3 N'), recomputed here from the
    # returned energies and forces, and dL/dtheta against central differences of that loss.
    wl = W.make("molecules16")
    sysm = wl.system.subset([3, 4])
    d = W.descriptor_params(4, 5.2, 6, 3, 2)
    archs = [W._mlp(d.D, (5, 3)) for _ in range(4)]
    rng = np.random.default_rng(12)
    theta = W.init_weights(rng, d, archs, 2.0, 2.0)
    e_ref = rng.normal(size=2)
    f_ref = rng.normal(size=(sysm.n_atoms, 3))
    norm = (7, 5 * sysm.n_atoms + 3)
    out = O.batch(sysm, d, archs, theta, e_ref=e_ref, f_ref=f_ref, w_force=0.3, param_grad=True, norm=norm)
    want = ((out["E_cfg"] - e_ref) ** 2).sum() / norm[0] + 0.3 * ((out["F"] - f_ref) ** 2).sum() / (3 * norm[1])
    assert abs(out["loss"] - want) < 1e-12 * want
    g = out["dtheta"]
    h = 1e-6
    off = W.param_offsets(archs)
    idx = []
    for s in set(sysm.species.tolist()):
        idx += list(rng.choice(np.arange(off[s], off[s + 1]), 6, replace=False))
    for k in idx:
        tp = theta.copy(); tp[k] += h
        tm = theta.copy(); tm[k] -= h
        lp = O.batch(sysm, d, archs, tp, e_ref=e_ref, f_ref=f_ref, w_force=0.3, norm=norm)["loss"]
        lm = O.batch(sysm, d, archs, tm, e_ref=e_ref, f_ref=f_ref, w_force=0.3, norm=norm)["loss"]
        assert abs((lp - lm) / (2 * h) - g[k]) < 1e-6 * max(1.0, abs(g[k])) + 1e-7 * np.abs(g).max(), k


def test_sampled_matches_batch():
    wl = W.make("fcc256")
    full = O.batch(wl.system, wl.desc, wl.archs, wl.theta, want_G=True)
    smp = [0, 17, 255]
    s = O.sampled(wl.system, 0, wl.desc, wl.archs, wl.theta, smp)
    np.testing.assert_allclose(s["G"], full["G"][smp], rtol=1e-12, atol=1e-14)
    np.testing.assert_allclose(s["E"], full["E_atom"][smp], rtol=1e-12)
    np.testing.assert_allclose(s["F"], full["F"][smp], atol=1e-11)
    i, j, sh = O.neighbor_list(wl.system, wl.desc.rc)
    for q, m in enumerate(smp):
        sel = i == m
        assert s["nnb"][q] == sel.sum()
        np.testing.assert_array_equal(s["nb_j"][q, :sel.sum()], j[sel])
        np.testing.assert_array_equal(s["nb_shift"][q, :sel.sum()], sh[sel])
