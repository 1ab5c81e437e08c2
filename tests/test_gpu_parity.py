"""GPU parity of the CUDA path (through the C ABI) with the FP64 oracle, at sizes the
oracle finishes in seconds that still span several tiles and a ragged tail."""
import numpy as np
import pytest

from oracle import oracle as O
from paper_2305_11805_gb300 import panna as P
from paper_2305_11805_gb300 import workloads as W
from tests import gpu_common as H

pytestmark = pytest.mark.gpu

SMALL = ["diamond64", "molecules16", "water512", "fcc256", "ragged8"]


@pytest.fixture(scope="module")
def torch_cuda():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2305_11805_gb300 import build
    build.build()
    return torch


def _special(name):
    if name == "tiny_cell":
        wl = W.make("fcc256")
        wl.system = H.tiny_cell_system()
        wl.desc = W.descriptor_params(1, 4.5, 16, 8, 8)
        wl.archs = [W._mlp(wl.desc.D, (32, 16))]
        wl.theta = W.init_weights(np.random.default_rng(0), wl.desc, wl.archs, 0.3, 0.05)
        return wl
    if name == "triclinic":
        return H.workload_with_system("water512", H.triclinic_system())
    if name == "mixed_pbc":
        return H.workload_with_system("water512", H.mixed_pbc_system())
    if name == "edges":
        return H.workload_with_system("ragged8", H.ragged_with_edges())
    return W.make(name)


CASES = SMALL + ["tiny_cell", "triclinic", "mixed_pbc", "edges"]


@pytest.mark.parametrize("name", CASES)
def test_neighbor_list_bit_exact(torch_cuda, name):
    wl = _special(name)
    pot = P.Potential(wl.desc, wl.archs)
    sysd = P.DeviceSystem(wl.system)
    got = H.gpu_neighbor_table(pot, sysd)
    want = H.sorted_pairs(*O.neighbor_list(wl.system, wl.desc.rc))
    assert got.shape == want.shape
    np.testing.assert_array_equal(got, want)


@pytest.mark.parametrize("name", CASES)
def test_descriptors_match_oracle(torch_cuda, name):
    wl = _special(name)
    pot = P.Potential(wl.desc, wl.archs)
    sysd = P.DeviceSystem(wl.system)
    G = pot.descriptors(sysd).cpu().numpy().astype(np.float64)
    Go = O.workload_batch(wl, want_G=True)["G"]
    err, ai, ac, cmax = H.descriptor_error(G, Go, wl.desc, where=True)
    col = H.descriptor_error(G, Go)
    print("%s descriptor max err %.3g of block max (atom %d, column %d of %d, block max %.3g);"
          " per-column %.3g" % (name, err, ai, ac, wl.desc.D, cmax, col))
    assert err <= H.TOL_G


# FP32 networks: the training products of the first layer on the tensor cores as TF32 parts
# (bit mask: 1 forward, 4 tangent, 8 weight gradient; 12 is the default) or everything on the
# CUDA cores (0).  Both must meet the FP32 tolerances.
FP32_PATHS = [12, 0]
FORCE_BOUND = {12: H.TOL_F_FP32, 0: H.TOL_F_FP32}


@pytest.mark.parametrize("path", FP32_PATHS)
@pytest.mark.parametrize("name", CASES)
def test_energy_forces_virial_fp32(torch_cuda, name, path):
    torch = torch_cuda
    wl = _special(name)
    pot = P.Potential(wl.desc, wl.archs)
    P.panna_set_tuning(pot.ctx, "mlp_fp32", path)
    sysd = P.DeviceSystem(wl.system)
    theta = torch.as_tensor(wl.theta, dtype=torch.float32, device="cuda")
    E, Ea, F, V = pot.energy_forces(sysd, theta, P.PANNA_MLP_FP32)
    # the oracle sees the same FP32-rounded parameters
    th32 = wl.theta.astype(np.float32).astype(np.float64)
    ref = O.batch(wl.system, wl.desc, wl.archs, th32)
    ferr, rms = H.force_error(F.cpu().numpy().astype(np.float64), ref["F"])
    scale = np.abs(ref["E_atom"]).sum() + 1e-30
    eerr = float(np.abs(E.cpu().numpy() - ref["E_cfg"]).max() / scale)
    verr = float(np.abs(V.cpu().numpy() - ref["virial"]).max() / (np.abs(ref["virial"]).max() + 1e-30))
    aerr = float(np.abs(Ea.cpu().numpy() - ref["E_atom"]).max() / (np.abs(ref["E_atom"]).max() + 1e-30))
    print("%s path %d: max|dF|/rms %.3g (rms %.3g), |dE|/sum|Ei| %.3g, virial %.3g, atom E %.3g" % (
        name, path, ferr, rms, eerr, verr, aerr))
    assert eerr <= H.TOL_E
    assert aerr <= 10 * H.TOL_E
    if rms > 0:
        assert ferr <= FORCE_BOUND[path]
    assert verr <= 10 * H.TOL_F_FP32


@pytest.mark.parametrize("path", FP32_PATHS)
@pytest.mark.parametrize("name", ["molecules16", "ragged8", "diamond64", "water512"])
def test_loss_gradient_fp32(torch_cuda, name, path):
    torch = torch_cuda
    wl = W.make(name)
    rng = np.random.default_rng(1)
    if wl.e_ref is None:
        wl.e_ref = rng.normal(size=wl.system.n_cfg) * 10
        wl.f_ref = rng.normal(size=(wl.system.n_atoms, 3))
    pot = P.Potential(wl.desc, wl.archs)
    P.panna_set_tuning(pot.ctx, "mlp_fp32", path)
    sysd = P.DeviceSystem(wl.system)
    th32 = wl.theta.astype(np.float32)
    theta = torch.as_tensor(th32, device="cuda")
    E_ref = torch.as_tensor(wl.e_ref, dtype=torch.float64, device="cuda")
    F_ref = torch.as_tensor(wl.f_ref, dtype=torch.float32, device="cuda")
    loss, g, E, F = pot.loss_grad(sysd, theta, E_ref, F_ref, wl.w_force)
    ref = O.batch(wl.system, wl.desc, wl.archs, th32.astype(np.float64), e_ref=wl.e_ref,
                  f_ref=wl.f_ref.astype(np.float32).astype(np.float64), w_force=wl.w_force, param_grad=True)
    lerr = abs(float(loss.item()) - ref["loss"]) / abs(ref["loss"])
    errs = H.layer_errors(wl.archs, g.cpu().numpy().astype(np.float64), ref["dtheta"])
    print("%s path %d: loss rel err %.3g, dtheta layer errs %s" % (name, path, lerr, ["%.2g" % e for e in errs]))
    assert lerr <= 1e-5
    assert max(errs) <= H.TOL_DTHETA


def test_param_vjp_matches_loss_gradient(torch_cuda):
    torch = torch_cuda
    wl = W.make("molecules16")
    pot = P.Potential(wl.desc, wl.archs)
    sysd = P.DeviceSystem(wl.system)
    theta = torch.as_tensor(wl.theta.astype(np.float32), device="cuda")
    E_ref = torch.as_tensor(wl.e_ref, dtype=torch.float64, device="cuda")
    F_ref = torch.as_tensor(wl.f_ref, dtype=torch.float32, device="cuda")
    loss, g, E, F = pot.loss_grad(sysd, theta, E_ref, F_ref, wl.w_force)
    C, N = sysd.n_cfg, sysd.n_atoms
    dE = 2.0 * (E - E_ref) / C
    dF = (2.0 * wl.w_force / (3 * N) * (F.double() - F_ref.double())).float()
    g2 = pot.param_vjp(sysd, theta, dE, dF)
    scale = g.abs().max().item()
    assert (g2 - g).abs().max().item() <= 1e-5 * scale
    # energy-only and force-only parts add up
    gE = pot.param_vjp(sysd, theta, dE, None)
    gF = pot.param_vjp(sysd, theta, None, dF)
    assert (gE + gF - g2).abs().max().item() <= 1e-5 * scale


def test_neighbor_capacity_overflow_is_retried(torch_cuda):
    torch = torch_cuda
    wl = W.make("diamond64")
    pot = P.Potential(wl.desc, wl.archs, neighbor_capacity=4)
    sysd = P.DeviceSystem(wl.system)
    theta = torch.as_tensor(wl.theta, dtype=torch.float32, device="cuda")
    E, Ea, F, V = pot.energy_forces(sysd, theta)
    assert P.panna_neighbor_capacity(pot.ctx) >= 20
    ref = O.batch(wl.system, wl.desc, wl.archs, wl.theta.astype(np.float32).astype(np.float64))
    assert H.force_error(F.cpu().numpy().astype(np.float64), ref["F"])[0] <= H.TOL_F_FP32


def test_bad_species_is_reported(torch_cuda):
    torch = torch_cuda
    wl = W.make("diamond64")
    wl.system.species = wl.system.species.copy()
    wl.system.species[5] = 3
    pot = P.Potential(wl.desc, wl.archs)
    sysd = P.DeviceSystem(wl.system)
    theta = torch.as_tensor(wl.theta, dtype=torch.float32, device="cuda")
    with pytest.raises(P.PannaError) as ei:
        pot.energy_forces(sysd, theta)
    assert ei.value.status == P.PANNA_ERR_BAD_INPUT
    # the context stays usable
    wl2 = W.make("diamond64")
    E, Ea, F, V = pot.energy_forces(P.DeviceSystem(wl2.system), theta)
    assert torch.isfinite(F).all()


VARIANTS = [0, 1, 2, 3, 4]   # blocked, flattened, compensated with 32 / 16 / 8 lanes per unit
# the adjoint's 4 is the flattened compensated walk, 5 the diagonal-order walk without atomics
ADJ_VARIANTS = VARIANTS + [5]


@pytest.mark.parametrize("variant", VARIANTS)
def test_results_are_deterministic(torch_cuda, variant):
    # descriptors and energies bit for bit with every descriptor kernel variant.  Forces are summed over centres with atomics (F_j -= q_ij from every centre
    # i), so they and the training gradient that depends on them agree to rounding only.
    torch = torch_cuda
    wl = W.make("water512")
    pot = P.Potential(wl.desc, wl.archs)
    P.panna_set_tuning(pot.ctx, "descriptor", variant)
    P.panna_set_tuning(pot.ctx, "jvp", variant)
    sysd = P.DeviceSystem(wl.system)
    theta = torch.as_tensor(wl.theta, dtype=torch.float32, device="cuda")
    G1 = pot.descriptors(sysd)
    G2 = pot.descriptors(sysd)
    assert torch.equal(G1, G2)
    E1 = pot.energy_forces(sysd, theta)[0]
    E2 = pot.energy_forces(sysd, theta)[0]
    assert torch.equal(E1, E2)
    E_ref = torch.zeros(sysd.n_cfg, dtype=torch.float64, device="cuda")
    F_ref = torch.zeros((sysd.n_atoms, 3), dtype=torch.float32, device="cuda")
    g1 = pot.loss_grad(sysd, theta, E_ref, F_ref, 0.1)[1]
    g2 = pot.loss_grad(sysd, theta, E_ref, F_ref, 0.1)[1]
    assert (g1 - g2).abs().max().item() <= 1e-5 * g1.abs().max().item()


@pytest.mark.parametrize("name", CASES)
@pytest.mark.parametrize("variant", VARIANTS)
def test_descriptor_variants(torch_cuda, name, variant):
    torch = torch_cuda
    wl = _special(name)
    pot = P.Potential(wl.desc, wl.archs)
    P.panna_set_tuning(pot.ctx, "descriptor", variant)
    sysd = P.DeviceSystem(wl.system)
    theta = torch.as_tensor(wl.theta, dtype=torch.float32, device="cuda")
    # panna_descriptors (rows in atom order) and the energy path (rows in network order)
    G = pot.descriptors(sysd).cpu().numpy().astype(np.float64)
    Go = O.workload_batch(wl, want_G=True)["G"]
    err = H.descriptor_error(G, Go, wl.desc)
    E = pot.energy_forces(sysd, theta, P.PANNA_MLP_FP32)[1].cpu().numpy().astype(np.float64)
    ref = O.batch(wl.system, wl.desc, wl.archs, wl.theta.astype(np.float32).astype(np.float64))
    aerr = float(np.abs(E - ref["E_atom"]).max() / (np.abs(ref["E_atom"]).max() + 1e-30))
    print("%s descriptor variant %d: G err %.3g, atomic energies %.3g" % (name, variant, err, aerr))
    assert err <= H.TOL_G
    assert aerr <= 10 * H.TOL_E


@pytest.mark.parametrize("name", ["molecules16", "fcc256", "ragged8", "tiny_cell", "water512", "diamond64",
                                  "triclinic", "mixed_pbc", "edges"])
@pytest.mark.parametrize("variant", ADJ_VARIANTS)
def test_adjoint_and_descriptor_variants(torch_cuda, name, variant):
    torch = torch_cuda
    wl = _special(name)
    pot = P.Potential(wl.desc, wl.archs)
    P.panna_set_tuning(pot.ctx, "adjoint", variant)
    P.panna_set_tuning(pot.ctx, "descriptor", min(variant, 4))
    sysd = P.DeviceSystem(wl.system)
    theta = torch.as_tensor(wl.theta, dtype=torch.float32, device="cuda")
    E, Ea, F, V = pot.energy_forces(sysd, theta, P.PANNA_MLP_FP32)
    ref = O.batch(wl.system, wl.desc, wl.archs, wl.theta.astype(np.float32).astype(np.float64))
    Fn = F.cpu().numpy().astype(np.float64)
    rms = float(np.sqrt((ref["F"] ** 2).mean()))
    if rms > 0:
        assert H.force_error(Fn, ref["F"])[0] <= H.TOL_F_FP32
    else:
        assert np.abs(Fn).max() <= 1e-5
    verr = float(np.abs(V.cpu().numpy() - ref["virial"]).max() / (np.abs(ref["virial"]).max() + 1e-30))
    assert verr <= 10 * H.TOL_F_FP32
    aerr = float(np.abs(Ea.cpu().numpy() - ref["E_atom"]).max() / (np.abs(ref["E_atom"]).max() + 1e-30))
    print("%s adjoint/descriptor variant %d: max|dF|/rms %.3g, virial %.3g" % (
        name, variant, H.force_error(Fn, ref["F"])[0] if rms > 0 else 0.0, verr))
    assert aerr <= 10 * H.TOL_E


@pytest.mark.parametrize("name", ["molecules16", "ragged8", "diamond64", "water512"])
@pytest.mark.parametrize("variant", VARIANTS)
def test_jvp_variants_training_gradient(torch_cuda, name, variant):
    torch = torch_cuda
    wl = W.make(name)
    rng = np.random.default_rng(3)
    e_ref = rng.normal(size=wl.system.n_cfg) * 10
    f_ref = rng.normal(size=(wl.system.n_atoms, 3))
    pot = P.Potential(wl.desc, wl.archs)
    P.panna_set_tuning(pot.ctx, "jvp", variant)
    sysd = P.DeviceSystem(wl.system)
    th32 = wl.theta.astype(np.float32)
    loss, g, E, F = pot.loss_grad(sysd, torch.as_tensor(th32, device="cuda"),
                                  torch.as_tensor(e_ref, dtype=torch.float64, device="cuda"),
                                  torch.as_tensor(f_ref, dtype=torch.float32, device="cuda"), 0.5)
    ref = O.batch(wl.system, wl.desc, wl.archs, th32.astype(np.float64), e_ref=e_ref,
                  f_ref=f_ref.astype(np.float32).astype(np.float64), w_force=0.5, param_grad=True)
    errs = H.layer_errors(wl.archs, g.cpu().numpy().astype(np.float64), ref["dtheta"])
    print("%s jvp variant %d: dtheta worst layer %.3g" % (name, variant, max(errs)))
    assert max(errs) <= H.TOL_DTHETA
