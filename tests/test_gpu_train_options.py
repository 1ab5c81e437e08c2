"""GPU parity of the training options of Sec. II.A through the C ABI: loss variants
(quadratic/exponential terms, per-atom energies, L1/L2 weight penalty) in panna_loss_grad,
and the fused Adam step with a decaying learning rate and frozen layers, against the oracle."""
import numpy as np
import pytest

from oracle import oracle as O
from paper_2305_11805_gb300 import panna as P
from paper_2305_11805_gb300 import workloads as W
from tests import gpu_common as H

pytestmark = pytest.mark.gpu

OPTS = [dict(e_kind=0, f_kind=0, e_per_atom=0, l1=0.0, l2=0.0),
        dict(e_kind=1, f_kind=0, e_per_atom=1, l1=1e-3, l2=0.0),
        dict(e_kind=0, f_kind=1, e_per_atom=0, l1=0.0, l2=1e-2),
        dict(e_kind=1, f_kind=1, e_per_atom=1, l1=2e-3, l2=5e-3)]


@pytest.fixture(scope="module")
def torch_cuda():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2305_11805_gb300 import build
    build.build()
    return torch


@pytest.fixture(scope="module")
def problem():
    wl = W.make("molecules16")
    th64 = wl.theta.astype(np.float32).astype(np.float64)
    base = O.batch(wl.system, wl.desc, wl.archs, th64)
    rng = np.random.default_rng(8)
    n = np.diff(wl.system.atom_off)
    # labels near the predictions, so that the exponential terms stay O(1)
    e_ref = base["E_cfg"] + rng.normal(0.0, 0.2, size=wl.system.n_cfg) * n
    f_ref = (base["F"] + rng.normal(0.0, 0.3, size=base["F"].shape)).astype(np.float32).astype(np.float64)
    return wl, th64, e_ref, f_ref


@pytest.mark.parametrize("k", range(len(OPTS)))
def test_loss_options_match_oracle(torch_cuda, problem, k):
    torch = torch_cuda
    wl, th64, e_ref, f_ref = problem
    o = OPTS[k]
    pot = P.Potential(wl.desc, wl.archs)
    P.panna_set_loss_options(pot.ctx, o["e_kind"], o["f_kind"], o["e_per_atom"], o["l1"], o["l2"])
    sysd = P.DeviceSystem(wl.system)
    loss, g, _, _ = pot.loss_grad(sysd, torch.as_tensor(th64.astype(np.float32), device="cuda"),
                                  torch.as_tensor(e_ref, device="cuda"),
                                  torch.as_tensor(f_ref.astype(np.float32), device="cuda"), 0.4)
    ref = O.batch(wl.system, wl.desc, wl.archs, th64, e_ref=e_ref, f_ref=f_ref, w_force=0.4, param_grad=True,
                  loss_options=o)
    lerr = abs(loss.item() - ref["loss"]) / abs(ref["loss"])
    errs = H.layer_errors(wl.archs, g.cpu().numpy().astype(np.float64), ref["dtheta"])
    print("options %s: loss %.3g, dtheta worst layer %.3g" % (o, lerr, max(errs)))
    assert lerr <= 1e-5 and max(errs) <= H.TOL_DTHETA
    # default options restored by NULL
    P.panna_set_loss_options(pot.ctx)


def test_adam_steps_match_oracle(torch_cuda):
    torch = torch_cuda
    wl = W.make("molecules16")
    pot = P.Potential(wl.desc, wl.archs)
    rng = np.random.default_rng(2)
    Pn = pot.P
    th = wl.theta.astype(np.float32)
    P.panna_set_frozen(pot.ctx, 1, 0, True)      # species 1, first layer
    P.panna_set_frozen(pot.ctx, 3, 2, True)      # species 3, output layer
    off = W.param_offsets(wl.archs)
    frozen = np.zeros(Pn, np.uint8)
    for s, l in ((1, 0), (3, 2)):
        a = wl.archs[s]
        o = off[s] + sum(a.widths[q + 1] * (a.widths[q] + 1) for q in range(l))
        frozen[o:o + a.widths[l + 1] * (a.widths[l] + 1)] = 1
    t_th = torch.as_tensor(th, device="cuda").clone()
    t_m = torch.zeros(Pn, device="cuda")
    t_v = torch.zeros(Pn, device="cuda")
    r_th, r_m, r_v = th.astype(np.float64), np.zeros(Pn), np.zeros(Pn)
    for t in range(1, 4):
        g = (rng.normal(size=Pn) * rng.lognormal(size=Pn) * 1e-2).astype(np.float32)
        P.panna_adam_step(pot.ctx, t_th, torch.as_tensor(g, device="cuda"), t_m, t_v, t, 1e-3, decay_rate=0.5,
                          decay_steps=4.0)
        r_th, r_m, r_v = O.adam_step(r_th, g.astype(np.float64), r_m, r_v, t, 1e-3, rate=0.5, steps=4.0,
                                     frozen=frozen)
    torch.cuda.synchronize()
    got = t_th.cpu().numpy().astype(np.float64)
    step = np.abs(r_th - th).max()
    print("3 Adam steps: max|dtheta - oracle| %.3g (largest move %.3g)" % (np.abs(got - r_th).max(), step))
    assert np.abs(got - r_th).max() <= 1e-4 * step + 1e-7 * np.abs(th).max()
    assert np.array_equal(got[frozen == 1], th[frozen == 1].astype(np.float64))
    # FP32 moments: m = b1 m + (1 - b1) g cancels when g changes sign, so its error scales with
    # the largest moment; v sums positive terms (1 - b2 rounded to FP32: ~1.3e-5 relative)
    assert np.abs(t_m.cpu().numpy() - r_m).max() <= 1e-6 * np.abs(r_m).max()
    np.testing.assert_allclose(t_v.cpu().numpy(), r_v, rtol=5e-5, atol=1e-6 * np.abs(r_v).max())


def test_training_option_arguments(torch_cuda):
    torch = torch_cuda
    wl = W.make("molecules16")
    pot = P.Potential(wl.desc, wl.archs)
    for bad in (dict(energy_loss=2), dict(force_loss=-1), dict(l1=-1.0)):
        with pytest.raises(P.PannaError) as ei:
            P.panna_set_loss_options(pot.ctx, **bad)
        assert ei.value.status == P.PANNA_ERR_INVALID_ARG
    with pytest.raises(P.PannaError):
        P.panna_set_frozen(pot.ctx, 4, 0, True)
    x = torch.zeros(pot.P, device="cuda")
    for kw in (dict(t=0, lr=1e-3), dict(t=1, lr=0.0), dict(t=1, lr=1e-3, beta1=1.0)):
        t = kw.pop("t")
        with pytest.raises(P.PannaError) as ei:
            P.panna_adam_step(pot.ctx, x, x, x, x, t, **kw)
        assert ei.value.status == P.PANNA_ERR_INVALID_ARG
