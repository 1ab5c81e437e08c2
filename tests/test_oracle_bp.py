"""Pins of the oracle's standard Behler-Parrinello angular term (the second descriptor form
Sec. II.A names): the trimer closed form, the cutoff on the third side, the Jacobian against
central differences (integer and non-integer zeta, both signs of lambda), and forces against
energy differences on a batch with the BP descriptor."""
import math

import numpy as np
import pytest

from oracle import oracle as O
from paper_2305_11805_gb300 import workloads as W


def _bp_desc(S=2, rc=4.5, lambdas=(1.0, -1.0, 0.5), zetas=(1.0, 2.0, 3.7), etas=(0.01, 0.2)):
    base = W.descriptor_params(S, rc, 5, 3, 2, eta_rad=2.0)
    import dataclasses
    return dataclasses.replace(base, angular="bp", bp_lambda=np.array(lambdas), bp_zeta=np.array(zetas),
                               bp_eta=np.array(etas))


def _fc(r, rc):
    return 0.5 * (1.0 + math.cos(math.pi * r / rc)) if r < rc else 0.0


@pytest.mark.parametrize("theta", [0.4, 1.3, 2.0, 2.9])
def test_trimer_closed_form(theta):
    d = _bp_desc()
    r1, r2 = 1.7, 2.2
    rv = np.array([[r1, 0.0, 0.0], [r2 * math.cos(theta), r2 * math.sin(theta), 0.0]])
    G = O.center(d, rv, [0, 1], jacobian=False)
    S, nr, NT, NA = 2, d.n_rad, d.n_theta, d.n_ang_r
    r12 = math.sqrt(r1 * r1 + r2 * r2 - 2 * r1 * r2 * math.cos(theta))
    F3 = _fc(r1, d.rc) * _fc(r2, d.rc) * _fc(r12, d.rc)
    blk = S * nr + 1 * NT * NA            # block {0, 1}
    for m in range(NT):
        lam, z = d.bp_lambda[m], d.bp_zeta[m]
        A = 2.0 ** (1 - z) * max(1 + lam * math.cos(theta), 0.0) ** z
        for n in range(NA):
            want = A * math.exp(-d.bp_eta[n] * (r1 * r1 + r2 * r2 + r12 * r12)) * F3
            assert abs(G[blk + m * NA + n] - want) < 1e-13 * max(1.0, abs(want))
    # the same-species blocks stay empty for a mixed pair
    assert not np.any(G[S * nr:S * nr + NT * NA]) and not np.any(G[S * nr + 2 * NT * NA:])


def test_third_side_beyond_cutoff_drops_the_pair():
    d = _bp_desc(rc=4.0)
    rv = np.array([[3.0, 0.0, 0.0], [-3.0, 0.2, 0.0]])   # r_jk ~ 6 > rc
    G = O.center(d, rv, [0, 0], jacobian=False)
    assert not np.any(G[2 * d.n_rad:])
    assert np.any(G[:2 * d.n_rad])


def test_bp_jacobian_central_differences():
    rng = np.random.default_rng(6)
    d = _bp_desc()
    rv = rng.normal(size=(6, 3)) * 1.3
    sp = np.array([0, 1, 1, 0, 1, 0], np.int32)
    G, J = O.center(d, rv, sp)
    assert np.any(G[2 * d.n_rad:])
    h = 1e-6
    for e in range(6):
        for c in range(3):
            dr = np.zeros_like(rv)
            dr[e, c] = h
            fd = (O.center(d, rv + dr, sp, jacobian=False) - O.center(d, rv - dr, sp, jacobian=False)) / (2 * h)
            np.testing.assert_allclose(J[:, e, c], fd, rtol=1e-6, atol=1e-9)


def test_bp_batch_forces_are_minus_energy_differences():
    wl = W.make("molecules16_bp")
    wl.system = wl.system.subset([0, 1, 2])
    s = wl.system
    ref = O.batch(s, wl.desc, wl.archs, wl.theta)
    h = 1e-5
    scale = np.abs(ref["F"]).max()
    for m in (0, 7, 20):
        for c in range(3):
            p, n = s.pos.copy(), s.pos.copy()
            p[m, c] += h
            n[m, c] -= h
            ep = O.batch(W.System(s.atom_off, p, s.species, s.cell, s.pbc, s.n_species), wl.desc, wl.archs,
                         wl.theta)["E_cfg"].sum()
            en = O.batch(W.System(s.atom_off, n, s.species, s.cell, s.pbc, s.n_species), wl.desc, wl.archs,
                         wl.theta)["E_cfg"].sum()
            assert abs(-(ep - en) / (2 * h) - ref["F"][m, c]) < 1e-6 * scale


def test_bp_sizes_and_workloads():
    for name in ("molecules16_bp", "water512_bp"):
        wl = W.make(name)
        S = wl.desc.n_species
        assert wl.desc.D == S * wl.desc.n_rad + S * (S + 1) // 2 * 4 * 2 == O.descriptor_size(wl.desc)
        assert wl.archs[0].widths[0] == wl.desc.D
