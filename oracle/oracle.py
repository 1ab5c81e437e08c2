"""ctypes front end of the FP64 CPU oracle (``panna_oracle.c``).

TEST INFRASTRUCTURE ONLY: imported by ``tests/``, ``__graft_entry__.smoke()`` and the
CPU-baseline leg of ``bench.py``.  The product path never imports it.

The shared library is compiled from the single C file with the system C compiler the
first time it is needed (or by :func:`build`) into ``oracle/_build/``.
"""
from __future__ import annotations

import ctypes as C
import math
import os
import subprocess
from typing import Optional, Sequence

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "panna_oracle.c")
_LIB = os.path.join(_HERE, "_build", "libpanna_oracle.so")
MAXL = 8

_dp = C.POINTER(C.c_double)
_i64p = C.POINTER(C.c_int64)
_i32p = C.POINTER(C.c_int32)
_u8p = C.POINTER(C.c_uint8)
_u32p = C.POINTER(C.c_uint32)


class OrcDesc(C.Structure):
    _fields_ = [("n_species", C.c_int), ("rc", C.c_double),
                ("n_rad", C.c_int), ("rs_rad", _dp), ("eta_rad", C.c_double),
                ("n_ang_r", C.c_int), ("rs_ang", _dp),
                ("n_theta", C.c_int), ("theta_s", _dp),
                ("eta_ang", C.c_double), ("zeta", C.c_double), ("eps_theta", C.c_double),
                ("angular_kind", C.c_int), ("bp_lambda", _dp), ("bp_zeta", _dp), ("bp_eta", _dp)]


class OrcArch(C.Structure):
    _fields_ = [("n_layers", C.c_int), ("widths", C.c_int * (MAXL + 1)), ("act", C.c_int * MAXL)]


def build(force: bool = False) -> str:
    """Compile the oracle (plain C, IEEE double, no fast-math) if it is missing or stale."""
    if force or not os.path.exists(_LIB) or os.path.getmtime(_LIB) < os.path.getmtime(_SRC):
        os.makedirs(os.path.dirname(_LIB), exist_ok=True)
        tmp = _LIB + ".%d.tmp" % os.getpid()
        subprocess.check_call(["gcc", "-O2", "-std=c99", "-D_DEFAULT_SOURCE", "-fPIC", "-shared",
                               "-fno-fast-math", "-ffp-contract=off", "-o", tmp, _SRC, "-lm"])
        os.replace(tmp, _LIB)
    return _LIB


_lib = None


def lib():
    global _lib
    if _lib is None:
        L = C.CDLL(build())
        L.orc_descriptor_size.restype = C.c_int
        L.orc_descriptor_size.argtypes = [C.POINTER(OrcDesc)]
        L.orc_center.restype = None
        L.orc_center.argtypes = [C.POINTER(OrcDesc), C.c_int, _dp, _i32p, _dp, _dp]
        L.orc_mlp.restype = None
        L.orc_mlp.argtypes = [C.POINTER(OrcArch), _dp, _dp, _dp, _dp, _dp, C.c_double, C.c_double, _dp]
        L.orc_neighbor_list.restype = C.c_int64
        L.orc_neighbor_list.argtypes = [C.c_int64, _i64p, _dp, _dp, _u8p, C.c_double, C.c_int64,
                                        _i64p, _i64p, _i32p]
        L.orc_batch.restype = C.c_int
        L.orc_batch.argtypes = [C.c_int64, _i64p, _dp, _i32p, _dp, _u8p, C.POINTER(OrcDesc),
                                C.POINTER(OrcArch), _dp, _i64p, _dp, _dp, _dp, _dp, _dp,
                                _dp, _dp, C.c_double, _dp, _dp, _u8p, C.c_double, C.c_double, C.POINTER(OrcLoss)]
        L.orc_adam_step.restype = None
        L.orc_adam_step.argtypes = [C.c_int64, _dp, _dp, _dp, _dp, C.c_int64, C.c_double, C.c_double, C.c_double,
                                    C.c_double, C.c_double, C.c_double, _u8p]
        L.orc_sampled.restype = C.c_int
        L.orc_sampled.argtypes = [C.c_int64, _dp, _i32p, _dp, _u8p, C.POINTER(OrcDesc),
                                  C.POINTER(OrcArch), _dp, _i64p, C.c_int64, _i64p, C.c_int64,
                                  _i32p, _i32p, _i64p, _dp, _dp, _dp]
        L.orc_philox4x32_10.restype = None
        L.orc_philox4x32_10.argtypes = [_u32p, _u32p, _u32p]
        L.orc_gauss3.restype = None
        L.orc_gauss3.argtypes = [C.c_uint64, C.c_int64, C.c_int64, _dp]
        L.orc_md_baoab.restype = C.c_int
        L.orc_md_baoab.argtypes = [C.c_int64, _i64p, _dp, _dp, _i32p, _dp, _u8p, C.POINTER(OrcDesc),
                                   C.POINTER(OrcArch), _dp, _i64p, _dp, C.c_double, C.c_double,
                                   C.c_double, C.c_uint64, C.c_int64, C.c_int64, _dp, _dp]
        _lib = L
    return _lib


class OrcLoss(C.Structure):
    _fields_ = [("e_kind", C.c_int32), ("f_kind", C.c_int32), ("e_per_atom", C.c_int32),
                ("l1", C.c_double), ("l2", C.c_double)]


def _ptr(a: Optional[np.ndarray], t):
    if a is None:
        return C.cast(None, t)
    assert a.flags["C_CONTIGUOUS"]
    return a.ctypes.data_as(t)


class _DescHolder:
    """Keeps the parameter arrays alive while C holds pointers into them."""

    def __init__(self, d):
        self.rs_rad = np.ascontiguousarray(d.rs_rad, np.float64)
        self.rs_ang = np.ascontiguousarray(d.rs_ang, np.float64)
        self.theta_s = np.ascontiguousarray(d.theta_s, np.float64)
        bp = getattr(d, "angular", "mbp") == "bp"
        self.bp = [np.ascontiguousarray(a, np.float64) for a in (d.bp_lambda, d.bp_zeta, d.bp_eta)] if bp else None
        self.s = OrcDesc(int(d.n_species), float(d.rc), len(self.rs_rad), _ptr(self.rs_rad, _dp),
                         float(d.eta_rad), d.n_ang_r, _ptr(self.rs_ang, _dp),
                         d.n_theta, _ptr(self.theta_s, _dp), float(d.eta_ang),
                         float(d.zeta), float(d.eps_theta), 1 if bp else 0,
                         *([_ptr(a, _dp) for a in self.bp] if bp else [None, None, None]))


def _arch(a) -> OrcArch:
    s = OrcArch()
    s.n_layers = a.n_layers
    for k, w in enumerate(a.widths):
        s.widths[k] = int(w)
    for k, t in enumerate(a.acts):
        s.act[k] = int(t)
    return s


def _archs(archs) -> C.Array:
    arr = (OrcArch * len(archs))()
    for k, a in enumerate(archs):
        arr[k] = _arch(a)
    return arr


def _theta_off(archs) -> np.ndarray:
    off = [0]
    for a in archs:
        off.append(off[-1] + a.n_params)
    return np.asarray(off, np.int64)


def descriptor_size(desc) -> int:
    h = _DescHolder(desc)
    return lib().orc_descriptor_size(C.byref(h.s))


def center(desc, rv: np.ndarray, sp: np.ndarray, jacobian: bool = True):
    """Descriptor G[D] of one centre with neighbour vectors rv[k,3] of species sp[k];
    with ``jacobian`` also J[D,k,3] = dG/dr."""
    h = _DescHolder(desc)
    rv = np.ascontiguousarray(rv, np.float64).reshape(-1, 3)
    sp = np.ascontiguousarray(sp, np.int32)
    k = rv.shape[0]
    D = lib().orc_descriptor_size(C.byref(h.s))
    G = np.zeros(D)
    J = np.zeros((D, k, 3)) if jacobian else None
    lib().orc_center(C.byref(h.s), k, _ptr(rv, _dp), _ptr(sp, _i32p), _ptr(G, _dp), _ptr(J, _dp))
    return (G, J) if jacobian else G


def mlp(arch, theta_s: np.ndarray, x: np.ndarray, xdot: Optional[np.ndarray] = None,
        alpha: float = 0.0, beta: float = 0.0, param_grad: bool = False):
    """(E, g = dE/dx, dtheta) for one input vector through one species' network."""
    a = _arch(arch)
    th = np.ascontiguousarray(theta_s, np.float64)
    x = np.ascontiguousarray(x, np.float64)
    xd = None if xdot is None else np.ascontiguousarray(xdot, np.float64)
    E = np.zeros(1)
    g = np.zeros(len(x))
    dth = np.zeros(len(th)) if param_grad else None
    lib().orc_mlp(C.byref(a), _ptr(th, _dp), _ptr(x, _dp), _ptr(E, _dp), _ptr(g, _dp),
                  _ptr(xd, _dp), float(alpha), float(beta), _ptr(dth, _dp))
    return float(E[0]), g, dth


def neighbor_list(system, rc: float):
    """Sorted (i, j, shift[.,3]) of every neighbour entry, global atom indices."""
    s = system
    off = np.ascontiguousarray(s.atom_off, np.int64)
    pos = np.ascontiguousarray(s.pos, np.float64)
    cell = np.ascontiguousarray(s.cell, np.float64)
    pbc = np.ascontiguousarray(s.pbc, np.uint8)
    L = lib()
    cap = 0
    while True:
        ii = np.zeros(max(cap, 1), np.int64)
        jj = np.zeros(max(cap, 1), np.int64)
        sh = np.zeros((max(cap, 1), 3), np.int32)
        n = L.orc_neighbor_list(s.n_cfg, _ptr(off, _i64p), _ptr(pos, _dp), _ptr(cell, _dp),
                                _ptr(pbc, _u8p), float(rc), cap, _ptr(ii, _i64p), _ptr(jj, _i64p),
                                _ptr(sh, _i32p))
        if n <= cap:
            return ii[:n], jj[:n], sh[:n]
        cap = int(n)


def jacobians(system, desc):
    """Per neighbour entry e = (i, j, n) of the sorted neighbour list, J[e] = dG_i/dr_e as a
    [D, 3] array (Sec. II: the derivative the forces contract with dE_i/dG_i), from the
    centre routine's Jacobian.  Returns dict(i, j, shift, r[P,3], J[P,D,3])."""
    s = system
    ii, jj, sh = neighbor_list(s, desc.rc)
    D = descriptor_size(desc)
    cfg = np.searchsorted(np.asarray(s.atom_off), ii, side="right") - 1
    cells = np.asarray(s.cell, np.float64).reshape(-1, 3, 3)
    r = np.asarray(s.pos)[jj] - np.asarray(s.pos)[ii] + np.einsum("pa,pab->pb", sh.astype(np.float64), cells[cfg])
    J = np.zeros((len(ii), D, 3))
    starts = np.searchsorted(ii, np.arange(s.n_atoms + 1))
    for i in range(s.n_atoms):
        a, b = starts[i], starts[i + 1]
        if b > a:
            _, Ji = center(desc, r[a:b], np.asarray(s.species)[jj[a:b]])
            J[a:b] = Ji.transpose(1, 0, 2)
    return dict(i=ii, j=jj, shift=sh, r=r, J=J)


def batch(system, desc, archs, theta, want_G: bool = False, e_ref=None, f_ref=None,
          w_force: float = 0.1, param_grad: bool = False, ghost=None, norm=None, loss_options=None):
    """Whole-batch FP64 evaluation; returns a dict of numpy arrays (see orc_batch).

    ghost: optional [n_atoms] flags of atoms that are neighbours only (not centres).
    norm: optional (C, N) loss normalisers replacing the batch's own counts.
    loss_options: optional dict(e_kind, f_kind (0 quadratic, 1 exponential), e_per_atom, l1, l2)."""
    s = system
    h = _DescHolder(desc)
    D = lib().orc_descriptor_size(C.byref(h.s))
    N, Cn = s.n_atoms, s.n_cfg
    off = np.ascontiguousarray(s.atom_off, np.int64)
    pos = np.ascontiguousarray(s.pos, np.float64)
    spec = np.ascontiguousarray(s.species, np.int32)
    cell = np.ascontiguousarray(s.cell, np.float64)
    pbc = np.ascontiguousarray(s.pbc, np.uint8)
    arr = _archs(archs)
    th = np.ascontiguousarray(theta, np.float64)
    toff = _theta_off(archs)
    out = dict(E_atom=np.zeros(N), E_cfg=np.zeros(Cn), F=np.zeros((N, 3)), virial=np.zeros((Cn, 3, 3)))
    G = np.zeros((N, D)) if want_G else None
    er = None if e_ref is None else np.ascontiguousarray(e_ref, np.float64)
    fr = None if f_ref is None else np.ascontiguousarray(f_ref, np.float64)
    loss = np.zeros(1)
    dth = np.zeros(len(th)) if (param_grad and er is not None) else None
    gh = None if ghost is None else np.ascontiguousarray(ghost, np.uint8)
    lo = None
    if loss_options is not None:
        o = dict(e_kind=0, f_kind=0, e_per_atom=0, l1=0.0, l2=0.0)
        o.update(loss_options)
        lo = OrcLoss(int(o["e_kind"]), int(o["f_kind"]), int(o["e_per_atom"]), float(o["l1"]), float(o["l2"]))
    lib().orc_batch(Cn, _ptr(off, _i64p), _ptr(pos, _dp), _ptr(spec, _i32p), _ptr(cell, _dp),
                    _ptr(pbc, _u8p), C.byref(h.s), arr, _ptr(th, _dp), _ptr(toff, _i64p),
                    _ptr(G, _dp), _ptr(out["E_atom"], _dp), _ptr(out["E_cfg"], _dp),
                    _ptr(out["F"], _dp), _ptr(out["virial"], _dp), _ptr(er, _dp), _ptr(fr, _dp),
                    float(w_force), _ptr(loss, _dp), _ptr(dth, _dp), _ptr(gh, _u8p),
                    float(norm[0]) if norm else 0.0, float(norm[1]) if norm else 0.0,
                    C.byref(lo) if lo is not None else None)
    if want_G:
        out["G"] = G
    if er is not None:
        out["loss"] = float(loss[0])
    if dth is not None:
        out["dtheta"] = dth
    return out


def workload_batch(wl, want_G=False, train=False):
    return batch(wl.system, wl.desc, wl.archs, wl.theta, want_G=want_G,
                 e_ref=wl.e_ref if train else None, f_ref=wl.f_ref if train else None,
                 w_force=wl.w_force, param_grad=train)


def adam_step(theta, grad, m, v, t, lr0, rate=1.0, steps=0.0, b1=0.9, b2=0.999, eps=1e-8, frozen=None):
    """One FP64 Adam step (see orc_adam_step); returns new (theta, m, v)."""
    th = np.array(theta, np.float64, copy=True)
    mm = np.array(m, np.float64, copy=True)
    vv = np.array(v, np.float64, copy=True)
    g = np.ascontiguousarray(grad, np.float64)
    fr = None if frozen is None else np.ascontiguousarray(frozen, np.uint8)
    lib().orc_adam_step(len(th), _ptr(th, _dp), _ptr(g, _dp), _ptr(mm, _dp), _ptr(vv, _dp), int(t), float(lr0),
                        float(rate), float(steps), float(b1), float(b2), float(eps), _ptr(fr, _u8p))
    return th, mm, vv


def philox4x32_10(ctr, key):
    """Philox4x32-10 of a counter of four 32-bit words and a key of two (see orc_philox4x32_10)."""
    c = np.ascontiguousarray(ctr, np.uint32)
    k = np.ascontiguousarray(key, np.uint32)
    out = np.zeros(4, np.uint32)
    lib().orc_philox4x32_10(_ptr(c, _u32p), _ptr(k, _u32p), _ptr(out, _u32p))
    return out


def gauss3(seed: int, atom: int, step: int):
    g = np.zeros(3)
    lib().orc_gauss3(int(seed), int(atom), int(step), _ptr(g, _dp))
    return g


def md_baoab(system, desc, archs, theta, vel, mass, dt, temperature, friction, seed, step0, n_steps):
    """BAOAB Langevin trajectory in FP64 (forces recomputed from scratch every step).
    Returns dict(pos, vel, F, E_traj [n_steps, n_cfg])."""
    s = system
    h = _DescHolder(desc)
    off = np.ascontiguousarray(s.atom_off, np.int64)
    pos = np.array(s.pos, np.float64, copy=True)
    v = np.array(vel, np.float64, copy=True).reshape(-1, 3)
    spec = np.ascontiguousarray(s.species, np.int32)
    cell = np.ascontiguousarray(s.cell, np.float64)
    pbc = np.ascontiguousarray(s.pbc, np.uint8)
    arr = _archs(archs)
    th = np.ascontiguousarray(theta, np.float64)
    toff = _theta_off(archs)
    m = np.ascontiguousarray(mass, np.float64)
    F = np.zeros((s.n_atoms, 3))
    E = np.zeros((max(int(n_steps), 1), s.n_cfg))
    lib().orc_md_baoab(s.n_cfg, _ptr(off, _i64p), _ptr(pos, _dp), _ptr(v, _dp), _ptr(spec, _i32p),
                       _ptr(cell, _dp), _ptr(pbc, _u8p), C.byref(h.s), arr, _ptr(th, _dp), _ptr(toff, _i64p),
                       _ptr(m, _dp), float(dt), float(temperature), float(friction), int(seed), int(step0),
                       int(n_steps), _ptr(F, _dp), _ptr(E, _dp))
    return dict(pos=pos, vel=v, F=F, E_traj=E[:int(n_steps)])


def sampled(system, cfg: int, desc, archs, theta, samples: Sequence[int], cap: int = 512):
    """Per sampled atom (indices local to configuration ``cfg``): neighbour list, G, E_i,
    force.  For configurations too large for :func:`batch`."""
    s = system
    a0, a1 = int(s.atom_off[cfg]), int(s.atom_off[cfg + 1])
    n = a1 - a0
    h = _DescHolder(desc)
    D = lib().orc_descriptor_size(C.byref(h.s))
    pos = np.ascontiguousarray(s.pos[a0:a1], np.float64)
    spec = np.ascontiguousarray(s.species[a0:a1], np.int32)
    cell = np.ascontiguousarray(s.cell[cfg], np.float64)
    pbc = np.ascontiguousarray(s.pbc[cfg], np.uint8)
    smp = np.ascontiguousarray(samples, np.int64)
    ns = len(smp)
    arr = _archs(archs)
    th = np.ascontiguousarray(theta, np.float64)
    toff = _theta_off(archs)
    nbj = np.zeros((ns, cap), np.int32)
    nbs = np.zeros((ns, cap, 3), np.int32)
    nnb = np.zeros(ns, np.int64)
    G = np.zeros((ns, D))
    E = np.zeros(ns)
    F = np.zeros((ns, 3))
    lib().orc_sampled(n, _ptr(pos, _dp), _ptr(spec, _i32p), _ptr(cell, _dp), _ptr(pbc, _u8p),
                      C.byref(h.s), arr, _ptr(th, _dp), _ptr(toff, _i64p), ns, _ptr(smp, _i64p),
                      cap, _ptr(nbj, _i32p), _ptr(nbs, _i32p), _ptr(nnb, _i64p), _ptr(G, _dp),
                      _ptr(E, _dp), _ptr(F, _dp))
    if np.any(nnb > cap):
        raise RuntimeError("neighbour capacity %d exceeded" % cap)
    return dict(nnb=nnb, nb_j=nbj, nb_shift=nbs, G=G, E=E, F=F)


# ------------------------------------------------------------------ charge equilibration

KE_EV_A = 14.399645478425668     # e^2 / (4 pi eps_0) in eV A


def _act(t, z):
    return np.exp(-z * z) if t == 1 else (np.maximum(z, 0.0) if t == 2 else (np.tanh(z) if t == 3 else z))


def _act_d1(t, z):
    if t == 1:
        return -2.0 * z * np.exp(-z * z)
    if t == 2:
        return (z > 0.0).astype(np.float64)
    if t == 3:
        return 1.0 - np.tanh(z) ** 2
    return np.ones_like(z)


def mlp_rows(arch, theta_s, X, seeds=None):
    """Eq. 1 on the rows of X (any output width): returns the outputs [n, w_L] and, with
    seeds [n, w_L], the input gradient sum_k seeds_k d out_k / dX."""
    X = np.atleast_2d(np.asarray(X, np.float64))
    Ws, bs, o = [], [], 0
    for l in range(arch.n_layers):
        fi, fo = arch.widths[l], arch.widths[l + 1]
        Ws.append(np.asarray(theta_s[o:o + fo * fi]).reshape(fo, fi))
        o += fo * fi
        bs.append(np.asarray(theta_s[o:o + fo]))
        o += fo
    a, zs = X, []
    for l in range(arch.n_layers):
        z = a @ Ws[l].T + bs[l]
        zs.append(z)
        a = _act(arch.acts[l], z)
    if seeds is None:
        return a
    bar = np.asarray(seeds, np.float64)
    for l in range(arch.n_layers - 1, -1, -1):
        bar = (bar * _act_d1(arch.acts[l], zs[l])) @ Ws[l]
    return a, bar


def qeq_kernel(r, sig_i, sig_j, ke=KE_EV_A):
    """Interaction of two unit Gaussian charges of widths sig_i, sig_j at distance r > 0, and
    its derivative with respect to r (scalars)."""
    g = math.sqrt(2.0 * (sig_i ** 2 + sig_j ** 2))
    e = math.erf(r / g)
    K = ke * e / r
    dK = ke * (2.0 / math.sqrt(math.pi) * math.exp(-(r / g) ** 2) / (g * r) - e / r ** 2)
    return K, dK


def qeq_solve(pos, sigma, chi, hard, Q, ke=KE_EV_A):
    """Charges of one configuration: the stationary point of
        E(q) = sum_i (chi_i q_i + J_i q_i^2 / 2) + 1/2 sum_ij q_i q_j K_ij
    subject to sum_i q_i = Q, with K_ij the Gaussian-charge interaction and K_ii the self
    energy ke / (sigma_i sqrt(pi)).  Solved as the (n+1) x (n+1) linear system
    [A 1; 1^T 0] [q; lam] = [-chi; Q], A = diag(J) + K.  Returns q, lam, K."""
    pos = np.asarray(pos, np.float64)
    n = len(pos)
    K = np.zeros((n, n))
    for i in range(n):
        K[i, i] = ke / (sigma[i] * math.sqrt(math.pi))
        for j in range(n):
            if j != i:
                K[i, j] = qeq_kernel(np.linalg.norm(pos[i] - pos[j]), sigma[i], sigma[j], ke)[0]
    M = np.zeros((n + 1, n + 1))
    M[:n, :n] = K + np.diag(hard)
    M[:n, n] = 1.0
    M[n, :n] = 1.0
    rhs = np.concatenate([-np.asarray(chi, np.float64), [Q]])
    x = np.linalg.solve(M, rhs)
    return x[:n], x[n], K


def qeq_batch(system, desc, archs, theta, qeq, charge=None, ke=KE_EV_A):
    """Energies, charges and forces with the charge-equilibration layer (Sec. II.B): every
    atom's network gives (e_i, dchi_i, dJ_i); chi_i = chi0_s + dchi_i, J_i = J0_s + dJ_i; the
    charges solve the constrained stationarity of qeq_solve for each (non-periodic)
    configuration, and
        E_c = sum_i (e_i + chi_i q_i + J_i q_i^2 / 2) + 1/2 sum_ij q_i q_j K_ij.
    Forces are -dE/dx at the equilibrated charges (the constraint's multiplier absorbs the
    charges' response): the networks' input gradients with seeds (1, q_i, q_i^2 / 2) through
    the descriptor Jacobians, plus the Gaussian-charge pair forces.
    E_atom_i = e_i + chi_i q_i + J_i q_i^2 / 2 + q_i (K q)_i / 2."""
    s = system
    G = batch(s, desc, archs, theta, want_G=True)["G"]
    toff = _theta_off(archs)
    N = s.n_atoms
    out3 = np.zeros((N, 3))
    for sp in range(len(archs)):
        rows = np.nonzero(s.species == sp)[0]
        if len(rows):
            out3[rows] = mlp_rows(archs[sp], theta[toff[sp]:toff[sp + 1]], G[rows])
    sig = np.asarray(qeq["sigma"])[s.species]
    chi = np.asarray(qeq["chi0"])[s.species] + out3[:, 1]
    hard = np.asarray(qeq["hard0"])[s.species] + out3[:, 2]
    q = np.zeros(N)
    E_atom = np.zeros(N)
    F = np.zeros((N, 3))
    lam = np.zeros(s.n_cfg)
    for c in range(s.n_cfg):
        a0, a1 = int(s.atom_off[c]), int(s.atom_off[c + 1])
        if a1 == a0:
            continue
        Qc = 0.0 if charge is None else float(charge[c])
        qc, lam[c], K = qeq_solve(s.pos[a0:a1], sig[a0:a1], chi[a0:a1], hard[a0:a1], Qc, ke)
        q[a0:a1] = qc
        E_atom[a0:a1] = out3[a0:a1, 0] + chi[a0:a1] * qc + 0.5 * hard[a0:a1] * qc ** 2 + 0.5 * qc * (K @ qc)
        for i in range(a0, a1):
            for j in range(a0, a1):
                if i != j:
                    d = s.pos[i] - s.pos[j]
                    r = np.linalg.norm(d)
                    F[i] -= q[i] * q[j] * qeq_kernel(r, sig[i], sig[j], ke)[1] * d / r
    seeds = np.stack([np.ones(N), q, 0.5 * q ** 2], 1)
    g = np.zeros_like(G)
    for sp in range(len(archs)):
        rows = np.nonzero(s.species == sp)[0]
        if len(rows):
            g[rows] = mlp_rows(archs[sp], theta[toff[sp]:toff[sp + 1]], G[rows], seeds[rows])[1]
    jac = jacobians(s, desc)
    qe = np.einsum("ed,edc->ec", g[jac["i"]], jac["J"])
    np.add.at(F, jac["i"], qe)
    np.add.at(F, jac["j"], -qe)
    E_cfg = np.array([E_atom[int(s.atom_off[c]):int(s.atom_off[c + 1])].sum() for c in range(s.n_cfg)])
    return dict(E_cfg=E_cfg, E_atom=E_atom, q=q, F=F, lam=lam, chi=chi, hard=hard, out=out3)


def mlp_rows_train(arch, theta_s, X, Xdot, seeds, tseeds):
    """Eq. 1 on rows with a forward tangent along Xdot: returns (outputs, output tangents,
    dtheta) where dtheta = d/dtheta sum_rows [seeds . out + tseeds . outdot] (the reverse pass
    over the forward and tangent computations, as orc_mlp does for one output)."""
    X = np.atleast_2d(np.asarray(X, np.float64))
    Xd = np.atleast_2d(np.asarray(Xdot, np.float64))
    Ws, bs, offs, o = [], [], [], 0
    for l in range(arch.n_layers):
        fi, fo = arch.widths[l], arch.widths[l + 1]
        offs.append(o)
        Ws.append(np.asarray(theta_s[o:o + fo * fi]).reshape(fo, fi))
        o += fo * fi
        bs.append(np.asarray(theta_s[o:o + fo]))
        o += fo
    a, ad, As, Ads, Zs, Zds = X, Xd, [X], [Xd], [], []
    for l in range(arch.n_layers):
        z = a @ Ws[l].T + bs[l]
        zd = ad @ Ws[l].T
        t = arch.acts[l]
        a, ad = _act(t, z), _act_d1(t, z) * zd
        Zs.append(z); Zds.append(zd); As.append(a); Ads.append(ad)
    dth = np.zeros(o)
    bar = np.asarray(seeds, np.float64)
    bard = np.asarray(tseeds, np.float64)
    for l in range(arch.n_layers - 1, -1, -1):
        t, z, zd = arch.acts[l], Zs[l], Zds[l]
        d1 = _act_d1(t, z)
        if t == 1:
            d2 = (4.0 * z * z - 2.0) * np.exp(-z * z)
        elif t == 3:
            th = np.tanh(z)
            d2 = -2.0 * th * (1.0 - th * th)
        else:
            d2 = np.zeros_like(z)
        zb = bar * d1 + bard * d2 * zd
        zdb = bard * d1
        fo, fi = Ws[l].shape
        dth[offs[l]:offs[l] + fo * fi] += (zb.T @ As[l] + zdb.T @ Ads[l]).ravel()
        dth[offs[l] + fo * fi:offs[l] + fo * fi + fo] += zb.sum(0)
        bar = zb @ Ws[l]
        bard = zdb @ Ws[l]
    return As[-1], Ads[-1], dth


def qeq_loss_grad(system, desc, archs, theta, qeq, charge, e_ref, f_ref, w_force, q_ref=None, w_charge=0.0,
                  ke=KE_EV_A):
    """Training through the charge layer: loss
        L = (1/C) sum_c (E_c - E_ref_c)^2 + w_F/(3N) sum (F - F_ref)^2 + w_q sum_i (q_i - q_ref_i)^2
    (the charge term only with q_ref) and dL/dtheta, by the chain rule in the order of the
    definition: dE_c/dtheta and the force term's derivative at fixed charges, plus the charges'
    response dq/dtheta from differentiating the constrained stationarity (one more solve with
    the same symmetric matrix)."""
    s = system
    base = qeq_batch(system, desc, archs, theta, qeq, charge, ke)
    N, C = s.n_atoms, s.n_cfg
    q, chi, hard, E_cfg, F = base["q"], base["chi"], base["hard"], base["E_cfg"], base["F"]
    dE = E_cfg - e_ref
    dF = F - f_ref
    loss = (dE ** 2).sum() / C + w_force / (3 * N) * (dF ** 2).sum()
    if q_ref is not None:
        loss += w_charge * ((q - q_ref) ** 2).sum()
    alpha = 2 * dE / C
    u = 2 * w_force / (3 * N) * dF
    # descriptor tangent along u: w_i = sum_e J_e (u_j(e) - u_i)
    G = batch(s, desc, archs, theta, want_G=True)["G"]
    jac = jacobians(s, desc)
    w = np.zeros_like(G)
    np.add.at(w, jac["i"], np.einsum("edc,ec->ed", jac["J"], u[jac["j"]] - u[jac["i"]]))
    toff = _theta_off(archs)
    cfg = np.searchsorted(s.atom_off, np.arange(N), side="right") - 1
    sq = np.stack([np.ones(N), q, 0.5 * q ** 2], 1)
    # output tangents (network part of u . d(dE/dq)/dx)
    odot = np.zeros((N, 3))
    for sp in range(len(archs)):
        rows = np.nonzero(s.species == sp)[0]
        if len(rows):
            odot[rows] = mlp_rows_train(archs[sp], theta[toff[sp]:toff[sp + 1]], G[rows], w[rows],
                                        np.zeros((len(rows), 3)), np.zeros((len(rows), 3)))[1]
    sig = np.asarray(qeq["sigma"])[s.species]
    mu = np.zeros(N)
    for c in range(C):
        a0, a1 = int(s.atom_off[c]), int(s.atom_off[c + 1])
        if a1 == a0:
            continue
        n = a1 - a0
        # v_i = sum_m u_m d/dx_m (dE/dq_i) at fixed charges
        v = odot[a0:a1, 1] + q[a0:a1] * odot[a0:a1, 2]
        for i in range(a0, a1):
            for j in range(a0, a1):
                if i != j:
                    d = s.pos[i] - s.pos[j]
                    r = np.linalg.norm(d)
                    v[i - a0] += q[j] * qeq_kernel(r, sig[i], sig[j], ke)[1] * d @ (u[i] - u[j]) / r
        h = -v
        if q_ref is not None:
            h = h + 2 * w_charge * (q[a0:a1] - q_ref[a0:a1])
        _, _, K = qeq_solve(s.pos[a0:a1], sig[a0:a1], chi[a0:a1], hard[a0:a1], 0.0, ke)
        M = np.zeros((n + 1, n + 1))
        M[:n, :n] = K + np.diag(hard[a0:a1])
        M[:n, n] = 1.0
        M[n, :n] = 1.0
        mu[a0:a1] = np.linalg.solve(M, np.concatenate([h, [0.0]]))[:n]
    seeds = alpha[cfg][:, None] * sq
    seeds[:, 1] -= mu
    seeds[:, 2] -= mu * q
    dth = np.zeros(len(theta))
    for sp in range(len(archs)):
        rows = np.nonzero(s.species == sp)[0]
        if len(rows):
            dth[toff[sp]:toff[sp + 1]] = mlp_rows_train(archs[sp], theta[toff[sp]:toff[sp + 1]], G[rows], w[rows],
                                                        seeds[rows], -sq[rows])[2]
    return dict(loss=loss, dtheta=dth, E_cfg=E_cfg, F=F, q=q, mu=mu)
