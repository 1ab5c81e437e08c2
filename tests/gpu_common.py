"""Shared helpers of the GPU parity tests (CUDA path through the C ABI vs the FP64 oracle)."""
import math

import numpy as np

from paper_2305_11805_gb300 import workloads as W

# Tolerances: FP32 path.
TOL_F_FP32 = 1e-5        # max |dF| / RMS(F_oracle)
TOL_F_BF16 = 1e-2
TOL_E = 1e-5             # |dE_c| / sum_i |E_i|
TOL_G = 1e-5             # per descriptor component, relative to its species block's max
TOL_DTHETA = 1e-4        # per layer: max |d dW| / max |dW|


def sorted_pairs(i, j, sh):
    key = np.lexsort((sh[:, 2], sh[:, 1], sh[:, 0], j, i))
    return np.stack([i[key], j[key], sh[key, 0], sh[key, 1], sh[key, 2]], 1)


def gpu_neighbor_table(pot, sysd):
    off, j, sh = pot.neighbors(sysd)
    off = off.cpu().numpy()
    i = np.repeat(np.arange(sysd.n_atoms), np.diff(off))
    return sorted_pairs(i, j.cpu().numpy(), sh.cpu().numpy())


def block_scales(desc, Go):
    """Max |G| over each species block (radial block per species, angular block per species
    pair), broadcast to the block's components."""
    colmax = np.abs(Go).max(0) if len(Go) else np.zeros(desc.D)
    out = np.empty(desc.D)
    S, nr, na = desc.n_species, desc.n_rad, desc.n_theta * desc.n_ang_r
    edges = [s * nr for s in range(S + 1)] + [S * nr + b * na for b in range(1, S * (S + 1) // 2 + 1)]
    for a, b in zip(edges[:-1], edges[1:]):
        out[a:b] = colmax[a:b].max() if b > a else 0.0
    return out


def descriptor_error(G, Go, desc=None, where=False):
    """max |G - Go| relative to the largest value of the component's species block."""
    scale = block_scales(desc, Go) if desc is not None else np.abs(Go).max(0)
    floor = 1e-6 * max(np.abs(Go).max(), 1e-30)
    rel = np.abs(G - Go) / np.maximum(scale, floor)
    if where:
        i, c = np.unravel_index(np.argmax(rel), rel.shape)
        return float(rel.max()), int(i), int(c), float(scale[c])
    return float(rel.max())


def force_error(F, Fo):
    """max |F - Fo| / RMS(Fo); absolute max when every reference force vanishes."""
    rms = math.sqrt((Fo ** 2).mean())
    d = float(np.abs(F - Fo).max()) if F.size else 0.0
    return (d / rms if rms > 0 else d), rms


def layer_errors(archs, g, go):
    """max |g - go| / max |go| over each layer block (W and b) of each species."""
    out = []
    off = 0
    for a in archs:
        for l in range(a.n_layers):
            n = a.widths[l + 1] * a.widths[l] + a.widths[l + 1]
            ref = go[off:off + n]
            scale = np.abs(ref).max()
            if scale > 0:
                out.append(float(np.abs(g[off:off + n] - ref).max() / scale))
            else:
                out.append(float(np.abs(g[off:off + n]).max()))
            off += n
    return out


def tiny_cell_system():
    """One atom in a cube of side 2 A with rc 4.5: neighbours are 56 of its own images."""
    return W.System(np.array([0, 1], np.int64), np.array([[0.5, 0.5, 0.5]]), np.zeros(1, np.int32),
                    (np.eye(3) * 2.0).reshape(1, 9), np.ones((1, 3), np.uint8), 1)


def triclinic_system(seed=3, n=24):
    rng = np.random.default_rng(seed)
    cell = np.array([[9.0, 0.0, 0.0], [2.7, 8.6, 0.0], [-1.9, 2.1, 9.3]])
    frac = rng.uniform(0, 1, (n, 3))
    pos = frac @ cell + rng.integers(-2, 3, (n, 3)) @ cell     # unwrapped on purpose
    return W.System(np.array([0, n], np.int64), pos, rng.integers(0, 2, n).astype(np.int32),
                    cell.reshape(1, 9), np.ones((1, 3), np.uint8), 2)


def mixed_pbc_system(seed=4, n=30):
    rng = np.random.default_rng(seed)
    L = 8.0
    pos = rng.uniform(0, L, (n, 3))
    pos[:, 2] = rng.uniform(-3, 12, n)
    return W.System(np.array([0, n], np.int64), pos, rng.integers(0, 2, n).astype(np.int32),
                    (np.eye(3) * L).reshape(1, 9), np.array([[1, 1, 0]], np.uint8), 2)


def ragged_with_edges(seed=5):
    """A batch with an empty configuration, a single atom and a dimer between real ones."""
    base = W.make("ragged8", seed).system
    parts = [base.subset([0]), None, None, None, base.subset([1])]
    sys_list = []
    sys_list.append(parts[0])
    sys_list.append(W.System(np.array([0, 0], np.int64), np.zeros((0, 3)), np.zeros(0, np.int32),
                             (np.eye(3) * 9.0).reshape(1, 9), np.ones((1, 3), np.uint8), 3))
    sys_list.append(W.System(np.array([0, 1], np.int64), np.array([[1.0, 2.0, 3.0]]), np.array([2], np.int32),
                             np.zeros((1, 9)), np.zeros((1, 3), np.uint8), 3))
    sys_list.append(W.System(np.array([0, 2], np.int64), np.array([[0.0, 0.0, 0.0], [1.3, 0.4, -0.2]]),
                             np.array([0, 1], np.int32), np.zeros((1, 9)), np.zeros((1, 3), np.uint8), 3))
    sys_list.append(parts[4])
    off = [0]
    for s in sys_list:
        off.append(off[-1] + s.n_atoms)
    return W.System(np.asarray(off, np.int64), np.concatenate([s.pos for s in sys_list]),
                    np.concatenate([s.species for s in sys_list]),
                    np.concatenate([s.cell for s in sys_list]), np.concatenate([s.pbc for s in sys_list]), 3)


def workload_with_system(name, system):
    wl = W.make(name)
    wl.system = system
    return wl
