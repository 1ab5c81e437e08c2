"""Pins of the oracle's loss options and Adam step (Sec. II.A: quadratic or exponential terms,
per-configuration or per-atom energies, L1/L2 weight penalty; Adam with a constant or
exponentially decaying learning rate; frozen layers).

The exponential term is read as exp(x^2) - 1 (the paper names it without a formula).  Pinned
against: the loss rebuilt from the returned energies and forces, central differences of
that loss on parameters of every layer, and closed forms of Adam's first and constant-
gradient steps, its scale invariance and schedule.
"""
import numpy as np

from oracle import oracle as O
from paper_2305_11805_gb300 import workloads as W

OPTS = [dict(e_kind=0, f_kind=0, e_per_atom=0, l1=0.0, l2=0.0),
        dict(e_kind=1, f_kind=0, e_per_atom=1, l1=1e-3, l2=0.0),
        dict(e_kind=0, f_kind=1, e_per_atom=0, l1=0.0, l2=1e-2),
        dict(e_kind=1, f_kind=1, e_per_atom=1, l1=2e-3, l2=5e-3)]


def _small_problem():
    wl = W.make("molecules16")
    sysm = wl.system.subset([0, 1, 2])
    d = W.descriptor_params(4, 5.2, 6, 3, 2)
    archs = [W._mlp(d.D, (5, 3)) for _ in range(4)]
    rng = np.random.default_rng(21)
    theta = W.init_weights(rng, d, archs, 2.0, 2.0)
    base = O.batch(sysm, d, archs, theta)
    n = np.diff(sysm.atom_off)
    # labels near the predictions, so the exponential terms stay O(1)
    e_ref = base["E_cfg"] + rng.normal(0.0, 0.3, size=sysm.n_cfg) * n
    f_ref = base["F"] + rng.normal(0.0, 0.3, size=base["F"].shape)
    return sysm, d, archs, theta, e_ref, f_ref


def _weights_mask(archs):
    mask = []
    for a in archs:
        for l in range(a.n_layers):
            mask += [1] * (a.widths[l + 1] * a.widths[l]) + [0] * a.widths[l + 1]
    return np.array(mask, bool)


def test_loss_options_closed_form():
    sysm, d, archs, theta, e_ref, f_ref = _small_problem()
    n = np.diff(sysm.atom_off).astype(np.float64)
    wmask = _weights_mask(archs)
    for o in OPTS:
        out = O.batch(sysm, d, archs, theta, e_ref=e_ref, f_ref=f_ref, w_force=0.4, loss_options=o)
        de = out["E_cfg"] - e_ref
        if o["e_per_atom"]:
            de = de / n
        ef = (out["F"] - f_ref).ravel()
        le = np.mean(np.exp(de ** 2) - 1.0 if o["e_kind"] else de ** 2)
        lf = np.mean(np.exp(ef ** 2) - 1.0 if o["f_kind"] else ef ** 2)
        want = le + 0.4 * lf + o["l1"] * np.abs(theta[wmask]).sum() + o["l2"] * (theta[wmask] ** 2).sum()
        assert abs(out["loss"] - want) < 1e-12 * abs(want), o


def test_loss_options_gradient_fd():
    sysm, d, archs, theta, e_ref, f_ref = _small_problem()
    rng = np.random.default_rng(4)
    off = W.param_offsets(archs)
    present = set(sysm.species.tolist())
    idx = []
    for s in present:
        idx += list(rng.choice(np.arange(off[s], off[s + 1]), 5, replace=False))
    h = 1e-6
    for o in OPTS[1:]:
        g = O.batch(sysm, d, archs, theta, e_ref=e_ref, f_ref=f_ref, w_force=0.4, param_grad=True,
                    loss_options=o)["dtheta"]
        for k in idx:
            tp = theta.copy(); tp[k] += h
            tm = theta.copy(); tm[k] -= h
            lp = O.batch(sysm, d, archs, tp, e_ref=e_ref, f_ref=f_ref, w_force=0.4, loss_options=o)["loss"]
            lm = O.batch(sysm, d, archs, tm, e_ref=e_ref, f_ref=f_ref, w_force=0.4, loss_options=o)["loss"]
            assert abs((lp - lm) / (2 * h) - g[k]) < 1e-6 * max(1.0, abs(g[k])) + 1e-7 * np.abs(g).max(), (o, k)


def test_adam_closed_forms():
    rng = np.random.default_rng(0)
    n = 1000
    th0 = rng.normal(size=n)
    g = rng.normal(size=n) * rng.lognormal(size=n)
    z = np.zeros(n)
    lr, eps = 1e-3, 1e-8
    # first step: m_hat = g, v_hat = g^2
    th1, m1, v1 = O.adam_step(th0, g, z, z, 1, lr, eps=eps)
    np.testing.assert_allclose(th1, th0 - lr * g / (np.abs(g) + eps), rtol=0, atol=1e-15)
    np.testing.assert_allclose(m1, 0.1 * g, rtol=1e-15)
    # a constant gradient keeps the bias-corrected ratio at g / |g| every step
    th, m, v = th0, z, z
    for t in range(1, 26):
        th, m, v = O.adam_step(th, g, m, v, t, lr, eps=0.0)
    np.testing.assert_allclose(th, th0 - 25 * lr * np.sign(g), rtol=0, atol=1e-12)
    # invariance to the gradient's scale (eps = 0)
    a, _, _ = O.adam_step(th0, g, z, z, 1, lr, eps=0.0)
    b, _, _ = O.adam_step(th0, 37.5 * g, z, z, 1, lr, eps=0.0)
    np.testing.assert_allclose(a, b, rtol=0, atol=1e-15)
    # exponential decay: at t = steps the rate is lr0 * rate; frozen entries untouched
    fr = (np.arange(n) % 3 == 0).astype(np.uint8)
    c, mc, vc = O.adam_step(th0, g, z, z, 10, lr, rate=0.5, steps=10.0, eps=0.0, frozen=fr)
    m_hat = (0.1 * g) / (1 - 0.9 ** 10)
    v_hat = (0.001 * g * g) / (1 - 0.999 ** 10)
    want = th0 - 0.5 * lr * m_hat / np.sqrt(v_hat)
    np.testing.assert_allclose(c[fr == 0], want[fr == 0], rtol=0, atol=1e-13)
    assert np.array_equal(c[fr == 1], th0[fr == 1]) and not np.any(mc[fr == 1]) and not np.any(vc[fr == 1])
