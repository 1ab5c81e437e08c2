"""GPU parity of the precomputed-descriptor path (Sec. II.A: descriptors and their derivatives
computed once, stored, reused) through the C ABI: every section of a store against the
oracle (descriptor rows, maps, entries, per-entry Jacobians expanded from the documented
compact layout), and energies, forces, virials and the training gradient evaluated from a
store against the oracle and against the on-the-fly path."""
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
    if name == "ragged_edges":
        return H.workload_with_system("ragged8", H.ragged_with_edges())
    if name == "tiny_cell":
        return H.workload_with_system("diamond64", H.tiny_cell_system())
    if name == "triclinic":
        wl = W.make("molecules16")
        s = H.triclinic_system()
        wl.system = W.System(s.atom_off, s.pos, s.species, s.cell, s.pbc, wl.system.n_species)
        return wl
    return W.make(name)


def _dense_columns(desc, sj):
    """Descriptor column of every compact Jacobian column for neighbour species sj (-1 = padding),
    written from the store format's definition."""
    S, nr, A = desc.n_species, desc.n_rad, desc.n_theta * desc.n_ang_r
    Rp, Ap = 4 * ((nr + 3) // 4), 4 * ((A + 3) // 4)
    blk = {}
    k = 0
    for a in range(S):
        for b in range(a, S):
            blk[(a, b)] = k
            k += 1
    cols = np.full(Rp + S * Ap, -1, np.int64)
    cols[:nr] = sj * nr + np.arange(nr)
    for s in range(S):
        b = blk[(min(sj, s), max(sj, s))]
        cols[Rp + s * Ap:Rp + s * Ap + A] = S * nr + b * A + np.arange(A)
    return cols


def _match_entries(i_s, j_s, r_s, ref):
    """Index into the oracle's entries of every store entry: same (i, j), nearest r."""
    key = {}
    for e, (i, j) in enumerate(zip(ref["i"], ref["j"])):
        key.setdefault((int(i), int(j)), []).append(e)
    out = np.empty(len(i_s), np.int64)
    for e in range(len(i_s)):
        cand = key[(int(i_s[e]), int(j_s[e]))]
        d = [np.abs(ref["r"][c] - r_s[e]).max() for c in cand]
        out[e] = cand[int(np.argmin(d))]
        assert min(d) < 1e-5
    return out


STORE_CASES = ["molecules16", "carbon16", "tiny_cell", "triclinic", "ragged_edges"]


@pytest.mark.parametrize("name", STORE_CASES)
def test_store_sections_match_oracle(torch_cuda, name):
    wl = _case(name)
    s, d = wl.system, wl.desc
    pot = P.Potential(d, wl.archs)
    sysd = P.DeviceSystem(s)
    st = P.Store(pot, sysd)
    sec = {k: v.cpu().numpy() for k, v in st.sections().items()}
    ref = O.jacobians(s, d)
    G_ref = O.batch(s, d, wl.archs, wl.theta, want_G=True)["G"]
    N = s.n_atoms
    assert st.info.n_entries == len(ref["i"]) and st.info.D == d.D
    # maps: rows grouped by species, in network order
    r_of_a, a_of_r, seg = sec["row_of_atom"], sec["atom_of_row"], sec["seg_off"]
    np.testing.assert_array_equal(a_of_r[r_of_a], np.arange(N))
    np.testing.assert_array_equal(seg, np.concatenate([[0], np.cumsum(np.bincount(s.species, minlength=d.n_species))]))
    for sp in range(d.n_species):
        assert np.all(s.species[a_of_r[seg[sp]:seg[sp + 1]]] == sp)
    np.testing.assert_array_equal(sec["atom_cfg"], np.repeat(np.arange(s.n_cfg), np.diff(s.atom_off)))
    # descriptors
    assert H.descriptor_error(sec["G"][r_of_a].astype(np.float64), G_ref, d) <= H.TOL_G
    # entries: the same set as the oracle's neighbour list, grouped by neighbour species
    off = sec["ent_off"]
    i_s = np.repeat(np.arange(N), np.diff(off))
    j_s, sp_s = sec["ent_idx"][:, 0], sec["ent_idx"][:, 1]
    np.testing.assert_array_equal(sp_s, s.species[j_s])
    for a in range(N):
        assert np.all(np.diff(sp_s[off[a]:off[a + 1]]) >= 0)
    r_s = sec["ent_vec"][:, :3].astype(np.float64)
    m = _match_entries(i_s, j_s, r_s, ref)
    assert len(np.unique(m)) == len(m)
    np.testing.assert_allclose(sec["ent_vec"][:, 3], np.linalg.norm(ref["r"][m], axis=1), rtol=1e-6)
    # Jacobians: compact columns expanded to D, against the oracle's dense dG_i/dr_e
    jac = sec["jac"].astype(np.float64)
    worst = 0.0
    for sp in range(d.n_species):
        cols = _dense_columns(d, sp)
        real = cols >= 0
        sel = np.nonzero(sp_s == sp)[0]
        if not len(sel):
            continue
        assert not np.any(jac[sel][:, :, ~real]), "padding columns hold zeros"
        dense = np.zeros((len(sel), 3, d.D))
        dense[:, :, cols[real]] = jac[sel][:, :, real]
        want = ref["J"][m[sel]].transpose(0, 2, 1)
        scale = np.abs(want).max(axis=(1, 2), keepdims=True) + 1e-30
        worst = max(worst, float((np.abs(dense - want) / scale).max()))
    print("%s: %d atoms, %d entries, width %d, store %.2f MB, worst J error %.3g of the entry's max" % (
        name, N, st.info.n_entries, st.info.width, st.nbytes / 1e6, worst))
    assert worst <= 1e-6


@pytest.mark.parametrize("name", ["molecules16", "carbon16", "triclinic", "ragged_edges"])
@pytest.mark.parametrize("prec", [P.PANNA_MLP_FP32, P.PANNA_MLP_BF16])
def test_store_energy_forces_match_oracle(torch_cuda, name, prec):
    torch = torch_cuda
    wl = _case(name)
    if prec == P.PANNA_MLP_BF16 and wl.desc.D % 8:
        pytest.skip("BF16 networks need D % 8 == 0")
    pot = P.Potential(wl.desc, wl.archs)
    sysd = P.DeviceSystem(wl.system)
    st = P.Store(pot, sysd)
    th32 = wl.theta.astype(np.float32)
    theta = torch.as_tensor(th32, device="cuda")
    E, Ea, F, V = st.energy_forces(sysd, theta, prec)
    ref = O.batch(wl.system, wl.desc, wl.archs, th32.astype(np.float64))
    tol = H.TOL_F_FP32 if prec == P.PANNA_MLP_FP32 else H.TOL_F_BF16
    ferr = H.force_error(F.cpu().numpy().astype(np.float64), ref["F"])[0]
    escale = np.abs(ref["E_atom"]).sum()
    eerr = float(np.abs(E.cpu().numpy() - ref["E_cfg"]).max() / escale)
    verr = float(np.abs(V.cpu().numpy() - ref["virial"]).max() / max(np.abs(ref["virial"]).max(), 1e-30))
    # against the on-the-fly path with the same networks
    E2, _, F2, _ = pot.energy_forces(sysd, theta, prec)
    fdiff = H.force_error(F.cpu().numpy().astype(np.float64), F2.cpu().numpy().astype(np.float64))[0]
    print("%s prec %d from the store: forces %.3g, energies %.3g, virial %.3g; vs on the fly %.3g" % (
        name, prec, ferr, eerr, verr, fdiff))
    assert ferr <= tol and eerr <= (H.TOL_E if prec == P.PANNA_MLP_FP32 else tol) and verr <= 10 * tol
    assert fdiff <= 2 * tol


@pytest.mark.parametrize("opts", [None, dict(e_kind=1, f_kind=1, e_per_atom=1, l1=1e-3, l2=1e-3)])
def test_store_loss_grad_matches_oracle(torch_cuda, opts):
    torch = torch_cuda
    wl = W.make("molecules16")
    pot = P.Potential(wl.desc, wl.archs)
    sysd = P.DeviceSystem(wl.system)
    st = P.Store(pot, sysd)
    th64 = wl.theta.astype(np.float32).astype(np.float64)
    base = O.batch(wl.system, wl.desc, wl.archs, th64)
    rng = np.random.default_rng(3)
    n = np.diff(wl.system.atom_off)
    e_ref = base["E_cfg"] + rng.normal(0.0, 0.2, size=wl.system.n_cfg) * n
    f_ref = (base["F"] + rng.normal(0.0, 0.3, size=base["F"].shape)).astype(np.float32).astype(np.float64)
    if opts:
        P.panna_set_loss_options(pot.ctx, opts["e_kind"], opts["f_kind"], opts["e_per_atom"], opts["l1"], opts["l2"])
    loss, g, E, F = st.loss_grad(sysd, torch.as_tensor(th64.astype(np.float32), device="cuda"),
                                 torch.as_tensor(e_ref, device="cuda"),
                                 torch.as_tensor(f_ref.astype(np.float32), device="cuda"), 0.4)
    ref = O.batch(wl.system, wl.desc, wl.archs, th64, e_ref=e_ref, f_ref=f_ref, w_force=0.4, param_grad=True,
                  loss_options=opts)
    lerr = abs(loss.item() - ref["loss"]) / abs(ref["loss"])
    errs = H.layer_errors(wl.archs, g.cpu().numpy().astype(np.float64), ref["dtheta"])
    ferr = H.force_error(F.cpu().numpy().astype(np.float64), ref["F"])[0]
    print("store training step %s: loss %.3g, dtheta worst layer %.3g, forces %.3g" % (opts, lerr, max(errs), ferr))
    assert lerr <= 1e-5 and max(errs) <= H.TOL_DTHETA and ferr <= H.TOL_F_FP32


def test_store_molecules1024_training_step(torch_cuda):
    """The benchmark's workload from a store: the whole training step against the oracle."""
    torch = torch_cuda
    wl = W.make("molecules1024")
    pot = P.Potential(wl.desc, wl.archs)
    sysd = P.DeviceSystem(wl.system)
    st = P.Store(pot, sysd)
    th32 = wl.theta.astype(np.float32)
    loss, g, E, F = st.loss_grad(sysd, torch.as_tensor(th32, device="cuda"), torch.as_tensor(wl.e_ref, device="cuda"),
                                 torch.as_tensor(wl.f_ref, dtype=torch.float32, device="cuda"), wl.w_force)
    ref = O.batch(wl.system, wl.desc, wl.archs, th32.astype(np.float64), e_ref=wl.e_ref,
                  f_ref=wl.f_ref.astype(np.float32).astype(np.float64), w_force=wl.w_force, param_grad=True)
    lerr = abs(loss.item() - ref["loss"]) / abs(ref["loss"])
    errs = H.layer_errors(wl.archs, g.cpu().numpy().astype(np.float64), ref["dtheta"])
    ferr = H.force_error(F.cpu().numpy().astype(np.float64), ref["F"])[0]
    print("molecules1024 from a %.0f MB store (%d entries): loss %.3g, dtheta worst layer %.3g, forces %.3g" % (
        st.nbytes / 1e6, st.info.n_entries, lerr, max(errs), ferr))
    assert lerr <= 1e-5 and max(errs) <= H.TOL_DTHETA and ferr <= H.TOL_F_FP32


def test_store_arguments(torch_cuda):
    torch = torch_cuda
    wl = W.make("molecules16")
    pot = P.Potential(wl.desc, wl.archs)
    sysd = P.DeviceSystem(wl.system)
    st = P.Store(pot, sysd)
    theta = torch.as_tensor(wl.theta.astype(np.float32), device="cuda")
    E = torch.empty(wl.system.n_cfg, dtype=torch.float64, device="cuda")
    F = torch.empty((wl.system.n_atoms, 3), dtype=torch.float32, device="cuda")
    # another batch
    other = P.DeviceSystem(wl.system.subset([0, 1]))
    with pytest.raises(P.PannaError) as ei:
        P.panna_store_energy_forces(pot.ctx, other, st.info, st.buf, theta, 0, E, None, F, None)
    assert ei.value.status == P.PANNA_ERR_INVALID_ARG
    # misaligned buffer
    with pytest.raises(P.PannaError) as ei:
        P.panna_store_energy_forces(pot.ctx, sysd, st.info, st.buf[16:], theta, 0, E, None, F, None)
    assert ei.value.status == P.PANNA_ERR_INVALID_ARG
    # size that does not match the entry count
    bad = P.panna_store_info.from_buffer_copy(st.info)
    bad.n_entries += 1
    with pytest.raises(P.PannaError) as ei:
        P.panna_store_energy_forces(pot.ctx, sysd, bad, st.buf, theta, 0, E, None, F, None)
    assert ei.value.status == P.PANNA_ERR_INVALID_ARG
    # positions that change the neighbour count between plan and build
    moved = wl.system.pos.copy()
    moved[:wl.system.atom_off[1]] *= 0.7
    msys = P.DeviceSystem(W.System(wl.system.atom_off, moved, wl.system.species, wl.system.cell, wl.system.pbc,
                                   wl.system.n_species))
    with pytest.raises(P.PannaError) as ei:
        P.panna_store_build(pot.ctx, msys, st.info, st.buf)
    assert ei.value.status == P.PANNA_ERR_INVALID_ARG
    # ghost atoms
    ghost = P.DeviceSystem(wl.system, ghost=np.zeros(wl.system.n_atoms, np.uint8))
    with pytest.raises(P.PannaError) as ei:
        P.panna_store_plan(pot.ctx, ghost)
    assert ei.value.status == P.PANNA_ERR_UNSUPPORTED
    # a store evaluates without positions
    nopos = P.DeviceSystem.from_tensors(sysd.atom_off, sysd.pos, sysd.species, sysd.cell, sysd.pbc)
    nopos.s.pos = None
    nopos.s.cell = None
    E1, _, F1, _ = st.energy_forces(nopos, theta)
    E2, _, F2, _ = st.energy_forces(sysd, theta)
    # (force sums use atomics: equal up to the order of the additions)
    assert (F1 - F2).abs().max().item() <= 1e-6 * F2.abs().max().item()
    assert (E1 - E2).abs().max().item() <= 1e-9 * E2.abs().max().item()
