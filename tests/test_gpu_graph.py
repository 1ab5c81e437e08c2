"""Ragged batch through one captured CUDA graph: replays match plain calls, follow in-place
input updates, and report status through panna_check."""
import numpy as np
import pytest

from paper_2305_11805_gb300 import panna as P
from paper_2305_11805_gb300 import workloads as W

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def torch_cuda():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2305_11805_gb300 import build
    build.build()
    return torch


@pytest.mark.parametrize("prec", [0, 1])
def test_graph_replay_matches_calls(torch_cuda, prec):
    torch = torch_cuda
    wl = W.make("ragged8")
    pot = P.Potential(wl.desc, wl.archs)
    sysd = P.DeviceSystem(wl.system)
    theta = torch.as_tensor(wl.theta.astype(np.float32), device="cuda")
    N, C = sysd.n_atoms, sysd.n_cfg
    E = torch.empty(C, dtype=torch.float64, device="cuda")
    Ea = torch.empty(N, dtype=torch.float32, device="cuda")
    F = torch.empty((N, 3), dtype=torch.float32, device="cuda")
    V = torch.empty((C, 3, 3), dtype=torch.float64, device="cuda")
    P.panna_capture(pot.ctx, sysd, theta, prec, E, Ea, F, V)
    ref = [t.clone() for t in pot.energy_forces(sysd, theta, prec)]
    for t in (E, Ea, F, V):
        t.fill_(float("nan"))
    stream = torch.cuda.Stream()
    with torch.cuda.stream(stream):
        P.panna_replay(pot.ctx, stream)
        P.panna_check(pot.ctx, stream)
    torch.cuda.synchronize()
    for a, b in zip((E, Ea, F, V), ref):
        assert torch.allclose(a, b, rtol=1e-5, atol=1e-5 * float(b.abs().max()))
    # inputs updated in place are picked up by the next replay
    sysd.pos.add_(torch.randn_like(sysd.pos) * 0.01)
    P.panna_replay(pot.ctx)
    P.panna_check(pot.ctx)
    ref2 = pot.energy_forces(sysd, theta, prec)
    assert torch.allclose(F, ref2[2], rtol=1e-5, atol=1e-5 * float(ref2[2].abs().max()))
    assert not torch.allclose(F, ref[2])
    assert P.panna_last_launch_count(pot.ctx) > 0
