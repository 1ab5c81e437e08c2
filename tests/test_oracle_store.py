"""Pins of the oracle's per-entry descriptor Jacobians (the quantity a precomputed-descriptor
store keeps, Sec. II.A) against central differences of the whole batch's descriptors and
against the oracle's pinned forces and virial.

dG_i/dx_m = sum over entries e of i with j(e) = m of J_e  -  [i = m] sum over entries of i of J_e
(a periodic self-image of i moves with i, so it enters both sums and cancels).
"""
import numpy as np
import pytest

from oracle import oracle as O
from paper_2305_11805_gb300 import workloads as W
from tests import gpu_common as H


def _predicted_dG(jac, n_atoms, m, c):
    D = jac["J"].shape[1]
    out = np.zeros((n_atoms, D))
    np.add.at(out, jac["i"][jac["j"] == m], jac["J"][jac["j"] == m, :, c])
    own = jac["i"] == m
    out[m] -= jac["J"][own, :, c].sum(0)
    return out


CASES = ["molecules16_head", "carbon16", "tiny_cell", "triclinic"]


def _case(name):
    if name == "molecules16_head":
        wl = W.make("molecules16")
        wl.system = wl.system.subset([0, 1])
        return wl
    if name == "tiny_cell":
        return H.workload_with_system("diamond64", H.tiny_cell_system())
    if name == "triclinic":
        wl = W.make("molecules16")
        s = H.triclinic_system()
        wl.system = W.System(s.atom_off, s.pos, s.species, s.cell, s.pbc, wl.system.n_species)
        return wl
    return W.make(name)


@pytest.mark.parametrize("name", CASES)
def test_entry_jacobians_match_position_differences(name):
    wl = _case(name)
    s = wl.system
    jac = O.jacobians(s, wl.desc)
    assert len(jac["i"]) > 0
    rng = np.random.default_rng(1)
    h = 1e-6
    for m in rng.choice(s.n_atoms, min(3, s.n_atoms), replace=False):
        for c in range(3):
            plus, minus = s.pos.copy(), s.pos.copy()
            plus[m, c] += h
            minus[m, c] -= h
            Gp = O.batch(W.System(s.atom_off, plus, s.species, s.cell, s.pbc, s.n_species), wl.desc, wl.archs,
                         wl.theta, want_G=True)["G"]
            Gm = O.batch(W.System(s.atom_off, minus, s.species, s.cell, s.pbc, s.n_species), wl.desc, wl.archs,
                         wl.theta, want_G=True)["G"]
            fd = (Gp - Gm) / (2 * h)
            want = _predicted_dG(jac, s.n_atoms, m, c)
            # (a lone atom among its own images has dG/dx = 0: scale by the entries' size)
            scale = max(np.abs(want).max(), np.abs(jac["J"][:, :, c]).max())
            assert np.abs(fd - want).max() <= 2e-6 * scale, (name, m, c)


def test_entry_jacobians_contract_to_forces_and_virial():
    wl = W.make("molecules16")
    s = wl.system
    ref = O.batch(s, wl.desc, wl.archs, wl.theta, want_G=True)
    jac = O.jacobians(s, wl.desc)
    off = W.param_offsets(wl.archs)
    g = np.zeros_like(ref["G"])
    for a in range(s.n_atoms):
        sp = int(s.species[a])
        _, g[a], _ = O.mlp(wl.archs[sp], wl.theta[off[sp]:off[sp + 1]], ref["G"][a])
    q = np.einsum("ed,edc->ec", g[jac["i"]], jac["J"])
    F = np.zeros((s.n_atoms, 3))
    np.add.at(F, jac["i"], q)
    np.add.at(F, jac["j"], -q)
    np.testing.assert_allclose(F, ref["F"], rtol=0, atol=1e-10 * np.abs(ref["F"]).max())
    cfg = np.searchsorted(s.atom_off, jac["i"], side="right") - 1
    V = np.zeros((s.n_cfg, 3, 3))
    np.add.at(V, cfg, -np.einsum("ea,eb->eab", q, jac["r"]))
    np.testing.assert_allclose(V, ref["virial"], rtol=0, atol=1e-10 * np.abs(ref["virial"]).max())


def test_entry_jacobian_sparsity_follows_species_blocks():
    """Columns outside the neighbour's radial block and the angular blocks containing its
    species are zero: what a compact store may leave out."""
    wl = W.make("molecules16")
    wl.system = wl.system.subset([0, 1, 2])
    d = wl.desc
    jac = O.jacobians(wl.system, d)
    S, nr, A = d.n_species, d.n_rad, d.n_theta * d.n_ang_r
    blocks = [(a, b) for a in range(S) for b in range(a, S)]
    sj = wl.system.species[jac["j"]]
    for sp in range(S):
        keep = np.zeros(d.D, bool)
        keep[sp * nr:(sp + 1) * nr] = True
        for k, (a, b) in enumerate(blocks):
            if sp in (a, b):
                keep[S * nr + k * A:S * nr + (k + 1) * A] = True
        sel = sj == sp
        if sel.any():
            assert not np.any(jac["J"][sel][:, ~keep, :])
            assert np.any(jac["J"][sel][:, keep, :])
