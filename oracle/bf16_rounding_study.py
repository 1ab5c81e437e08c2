"""Which BF16 rounding in the per-species networks moves the forces, and by how much.

Test infrastructure (analysis run by hand, not part of the library's path): the networks of
Eq. 1 are emulated in numpy with FP32 accumulation and round-to-nearest-even BF16 at chosen
GEMM operands (the first layer's input G and weights W1, the hidden layers' activations and
weights, the backward seeds z-bar of the hidden layers and of the first layer), on the FP64
oracle's descriptors; forces are formed from g = dE/dG through the oracle's descriptor
Jacobians (F_i += q_e, F_j -= q_e, q_e = g_i . dG_i/dr_e), so only the networks' rounding
enters.  Prints max |dF| / RMS(F) against the oracle's forces for one rounded operand class at
a time, for all of them, and for the hi + lo pairs (two BF16 numbers per operand).

    python oracle/bf16_rounding_study.py [ragged8|water512|fcc256|...]
"""
import os
import sys

import numpy as np

sys.path.insert(0, os.path.dirname(os.path.dirname(os.path.abspath(__file__))))
from oracle import oracle as O                      # noqa: E402
from paper_2305_11805_gb300 import workloads as W   # noqa: E402


def bf16(x):
    """Round FP32 values to the nearest BF16 (ties to even), returned as FP32."""
    x = np.asarray(x, np.float32)
    u = x.view(np.uint32).astype(np.uint64)
    u = ((u + 0x7FFF + ((u >> 16) & 1)) >> 16) << 16
    return u.astype(np.uint32).view(np.float32)


def rnd(x, mode):
    """mode 0: FP32 as is; 1: one BF16 rounding; 2: hi + lo pair of BF16 numbers."""
    x = np.asarray(x, np.float32)
    if mode == 0:
        return x
    h = bf16(x)
    return h if mode == 1 else h + bf16(x - h)


def _gauss(z):
    return np.exp(-z * z)


def _dgauss(z):
    return -2 * z * np.exp(-z * z)


def input_gradient(arch, th, G, R):
    """dE/dG of one species' network (Gaussian hidden units, linear output) with the
    roundings R (keys G, W1, A, W, Zb, Zb1 -> mode)."""
    off = 0
    Ws, bs = [], []
    for l in range(arch.n_layers):
        no, ni = arch.widths[l + 1], arch.widths[l]
        Ws.append(th[off:off + no * ni].reshape(no, ni).astype(np.float32))
        off += no * ni
        bs.append(th[off:off + no].astype(np.float32))
        off += no
    L = arch.n_layers
    zs, x = [], G.astype(np.float32)
    for l in range(L - 1):
        xin = rnd(x, R['G'] if l == 0 else R['A'])
        w = rnd(Ws[l], R['W1'] if l == 0 else R['W'])
        z = (xin.astype(np.float64) @ w.T.astype(np.float64)).astype(np.float32) + bs[l]
        zs.append(z)
        x = _gauss(z).astype(np.float32)
    ab = np.tile(Ws[-1][0], (len(G), 1)).astype(np.float32)
    for l in range(L - 2, -1, -1):
        zb = (ab * _dgauss(zs[l])).astype(np.float32)
        w = rnd(Ws[l], R['W1'] if l == 0 else R['W'])
        ab = (rnd(zb, R['Zb1'] if l == 0 else R['Zb']).astype(np.float64) @ w.astype(np.float64)).astype(np.float32)
    return ab.astype(np.float64)


def main(name):
    wl = W.make(name)
    th = wl.theta.astype(np.float32).astype(np.float64)
    ref = O.batch(wl.system, wl.desc, wl.archs, th, want_G=True)
    G = ref["G"]
    jac = O.jacobians(wl.system, wl.desc)
    sp = wl.system.species
    rms = np.sqrt((ref["F"] ** 2).mean())
    offs = wl.param_offsets

    def error(R):
        g = np.zeros_like(G)
        for s in range(wl.desc.n_species):
            m = sp == s
            if m.any():
                g[m] = input_gradient(wl.archs[s], th[offs[s]:offs[s + 1]], G[m], R)
        q = np.einsum("pd,pdk->pk", g[jac["i"]], jac["J"])
        F = np.zeros((wl.system.n_atoms, 3))
        np.add.at(F, jac["i"], q)
        np.add.at(F, jac["j"], -q)
        return np.abs(F - ref["F"]).max() / rms

    base = dict(G=0, W1=0, A=0, W=0, Zb=0, Zb1=0)
    print("%s: FP32 emulation %.2e" % (name, error(base)))
    for k in base:
        for m in (1, 2):
            R = dict(base)
            R[k] = m
            print("  %-3s %s: %.2e" % (k, "rounded once" if m == 1 else "hi + lo     ", error(R)))
    print("  all rounded once: %.2e" % error({k: 1 for k in base}))
    print("  all hi + lo:      %.2e" % error({k: 2 for k in base}))


if __name__ == "__main__":
    main(sys.argv[1] if len(sys.argv) > 1 else "ragged8")
