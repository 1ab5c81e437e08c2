"""Pins of the oracle's Langevin dynamics (the MD loop the paper times, Sec. III.B).

The paper states only that its timing runs Langevin dynamics at 300 K through ASE; the
integrator read here is BAOAB (Leimkuhler and Matthews) with a Philox4x32-10 noise stream.
Pinned against: the generator's published known-answer vectors; the normal distribution
of the Box-Muller numbers; second-order energy conservation of the deterministic limit
(velocity Verlet); the exact Ornstein-Uhlenbeck update of force-free atoms.
"""
import math
import os

import numpy as np

from oracle import oracle as O
from paper_2305_11805_gb300 import workloads as W

GOLD = os.path.join(os.path.dirname(__file__), "golden")
ACC = 9.648533212e-3      # (eV/A)/amu in A/fs^2
KB = 8.617333262e-5       # eV/K


def test_philox_known_answers():
    rows = [l.split() for l in open(os.path.join(GOLD, "philox4x32_10_kat.txt")) if l.strip() and l[0] != "#"]
    assert len(rows) == 3
    for r in rows:
        v = [int(x, 16) for x in r]
        got = O.philox4x32_10(v[0:4], v[4:6])
        assert [int(x) for x in got] == v[6:10]


def test_box_muller_normals():
    g = np.array([O.gauss3(12345, a, 7) for a in range(20000)])
    n = g.size
    assert abs(g.mean()) < 4.0 / math.sqrt(n)
    assert abs(g.var() - 1.0) < 0.04
    assert abs(((g - g.mean()) ** 4).mean() / g.var() ** 2 - 3.0) < 0.2
    c = np.corrcoef(g.T)
    assert np.abs(c - np.eye(3)).max() < 0.04
    # different steps and seeds give different streams
    assert not np.allclose(O.gauss3(1, 0, 0), O.gauss3(1, 0, 1))
    assert not np.allclose(O.gauss3(1, 0, 0), O.gauss3(2, 0, 0))


def _total_energy(wl, res, mass):
    ekin = 0.5 * (mass[wl.system.species][:, None] * res["vel"] ** 2).sum() / ACC
    return res["E_traj"][-1].sum() + ekin


def test_velocity_verlet_limit_is_second_order():
    # temperature 0 and friction 0: BAOAB is velocity Verlet; the energy error over a fixed
    # time falls 4x when the step halves
    wl = W.make("carbon16")
    mass = np.array([12.011])
    rng = np.random.default_rng(3)
    v0 = rng.normal(0.0, math.sqrt(KB * 600.0 * ACC / 12.011), size=(wl.system.n_atoms, 3))
    v0 -= v0.mean(0)
    e0 = O.batch(wl.system, wl.desc, wl.archs, wl.theta)["E_cfg"].sum() + 0.5 * 12.011 * (v0 ** 2).sum() / ACC
    errs = []
    for dt, n in ((1.0, 8), (0.5, 16)):
        res = O.md_baoab(wl.system, wl.desc, wl.archs, wl.theta, v0, mass, dt, 0.0, 0.0, 0, 0, n)
        errs.append(abs(_total_energy(wl, res, mass) - e0))
    assert errs[0] > 0
    assert 2.5 < errs[0] / errs[1] < 6.0, errs


def test_ornstein_uhlenbeck_step_of_free_atoms():
    # atoms 20 A apart feel no force; one step from rest: v = c2 sqrt(kB T a) g exactly, with
    # g the generator's normals, and x moves by dt/2 v (the first A-step sees v = 0)
    n = 2000
    k = np.arange(n)
    pos = np.stack([k % 10, (k // 10) % 10, k // 100], 1).astype(np.float64) * 20.0
    wl = W.make("carbon16")
    sysm = W.System(np.array([0, n], np.int64), pos, np.zeros(n, np.int32), np.zeros((1, 9)),
                    np.zeros((1, 3), np.uint8), 1)
    dt, T, gam, seed = 0.5, 300.0, 0.02, 99
    mass = np.array([12.011])
    res = O.md_baoab(sysm, wl.desc, wl.archs, wl.theta, np.zeros((n, 3)), mass, dt, T, gam, seed, 5, 1)
    c1 = math.exp(-gam * dt)
    sig = math.sqrt(1.0 - c1 * c1) * math.sqrt(KB * T * ACC / 12.011)
    g = np.array([O.gauss3(seed, a, 5) for a in range(n)])
    np.testing.assert_allclose(res["vel"], sig * g, rtol=1e-12, atol=1e-15)
    np.testing.assert_allclose(res["pos"] - pos, 0.5 * dt * res["vel"], rtol=1e-9, atol=1e-13)
    assert not np.any(res["F"])
    assert abs(res["vel"].std() / sig - 1.0) < 0.03
