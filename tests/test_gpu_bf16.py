"""BF16 tensor-core networks (tcgen05, FP32 accumulation): energies and forces against the
FP64 oracle and against the FP32-network GPU path.

PANNA_MLP_BF16 (operands as hi + lo BF16 pairs, three MMAs per product) meets the force bar
max |dF| <= 1e-2 RMS(F).  PANNA_MLP_BF16_FAST (one BF16 rounding per operand) does not: its
errors (2.6e-2 to 4.3e-2 of RMS on these inputs) are reported and only guarded against
regressions."""
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


@pytest.mark.parametrize("name", ["water512", "fcc256", "ragged8", "diamond64", "molecules16"])
def test_bf16_energy_forces(torch_cuda, name):
    torch = torch_cuda
    wl = W.make(name)
    pot = P.Potential(wl.desc, wl.archs)
    sysd = P.DeviceSystem(wl.system)
    th32 = wl.theta.astype(np.float32)
    theta = torch.as_tensor(th32, device="cuda")
    E16, Ea16, F16, V16 = pot.energy_forces(sysd, theta, P.PANNA_MLP_BF16)
    E8, Ea8, F8, V8 = pot.energy_forces(sysd, theta, P.PANNA_MLP_BF16_FAST)
    E32, Ea32, F32, V32 = pot.energy_forces(sysd, theta, P.PANNA_MLP_FP32)
    ref = O.batch(wl.system, wl.desc, wl.archs, th32.astype(np.float64))
    ferr, rms = H.force_error(F16.cpu().numpy().astype(np.float64), ref["F"])
    f32err, _ = H.force_error(F32.cpu().numpy().astype(np.float64), ref["F"])
    escale = np.abs(ref["E_atom"]).sum()
    eerr = float(np.abs(E16.cpu().numpy() - ref["E_cfg"]).max() / escale)
    aerr = float(np.abs(Ea16.cpu().numpy() - ref["E_atom"]).max() / np.abs(ref["E_atom"]).max())
    f8err, _ = H.force_error(F8.cpu().numpy().astype(np.float64), ref["F"])
    a8err = float(np.abs(Ea8.cpu().numpy() - ref["E_atom"]).max() / np.abs(ref["E_atom"]).max())
    verr = float(np.abs(V16.cpu().numpy() - ref["virial"]).max() / np.abs(ref["virial"]).max())
    print("%s BF16: max|dF|/rms %.3g (FP32 path %.3g, BF16_FAST %.3g), |dE|/sum|Ei| %.3g, atom E %.3g "
          "(FAST %.3g), virial %.3g" % (name, ferr, f32err, f8err, eerr, aerr, a8err, verr))
    assert aerr <= H.TOL_F_BF16
    assert eerr <= H.TOL_F_BF16
    assert ferr <= H.TOL_F_BF16
    assert verr <= H.TOL_F_BF16
    assert f8err <= 6e-2 and a8err <= 2e-2
