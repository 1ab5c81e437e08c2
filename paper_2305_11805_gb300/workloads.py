"""Seeded synthetic inputs shaped like the workloads of PANNA 2.0 (arXiv 2305.11805).

This module only draws random numbers and lays out arrays: atomic positions, species,
cells, periodic flags, descriptor parameter grids, network architectures, initial weights
and training labels.  It holds none of the method's arithmetic (no descriptor, network,
force or loss evaluation), so the FP64 CPU oracle and the CUDA path can both consume it
without sharing any code.  The only geometry it does is input validation: minimum pair
separations and the guarantee that no pair distance lies within ``CUTOFF_MARGIN`` of the
cutoff (so neighbour sets are well defined and can be compared bit for bit).

Workloads (sizes follow the paper's experiments, Sec. III, and the five benchmark shapes):

* ``diamond64``      64-atom periodic diamond Si-like lattice, one species (Sec. III.B sizes).
* ``molecules1024``  1024 isolated bonded chains of 5..29 atoms, H/C/N/O, training step.
* ``water32k``       32,768-atom periodic two-species liquid-like box (O:H = 1:2).
* ``fcc1m``          1,048,576-atom periodic FCC box, one species, 64 radial + 128 angular.
* ``ragged4096``     4096 periodic cubic boxes of 32..4096 atoms, three species.

Each has smaller variants with the same recipe for the CPU oracle (``*_small`` and
``water512``).
"""
from __future__ import annotations

import dataclasses
import math
from typing import List, Optional, Sequence

import numpy as np

# No pair distance may lie within this many Angstrom of the cutoff (either side).
CUTOFF_MARGIN = 1e-6

ACT_LINEAR, ACT_GAUSSIAN, ACT_RELU, ACT_TANH = 0, 1, 2, 3


@dataclasses.dataclass
class System:
    """A ragged batch of configurations.

    atom_off: int64 [C+1], atoms of configuration c are rows atom_off[c]:atom_off[c+1].
    pos:      float64 [N,3] Cartesian positions (Angstrom).
    species:  int32 [N] in 0..n_species-1.
    cell:     float64 [C,9], row-major 3x3 whose rows are the lattice vectors.
    pbc:      uint8 [C,3] periodic flags per lattice direction.
    """
    atom_off: np.ndarray
    pos: np.ndarray
    species: np.ndarray
    cell: np.ndarray
    pbc: np.ndarray
    n_species: int

    @property
    def n_atoms(self) -> int:
        return int(self.atom_off[-1])

    @property
    def n_cfg(self) -> int:
        return int(self.atom_off.shape[0] - 1)

    def config_of_atom(self) -> np.ndarray:
        counts = np.diff(self.atom_off)
        return np.repeat(np.arange(self.n_cfg, dtype=np.int64), counts)

    def subset(self, cfgs: Sequence[int]) -> "System":
        """The configurations ``cfgs`` (in that order) as a new batch."""
        rows, off = [], [0]
        for c in cfgs:
            a, b = int(self.atom_off[c]), int(self.atom_off[c + 1])
            rows.append(np.arange(a, b))
            off.append(off[-1] + b - a)
        idx = np.concatenate(rows) if rows else np.zeros(0, np.int64)
        cfgs = np.asarray(cfgs, dtype=np.int64)
        return System(np.asarray(off, np.int64), self.pos[idx].copy(),
                      self.species[idx].copy(), self.cell[cfgs].copy(),
                      self.pbc[cfgs].copy(), self.n_species)


@dataclasses.dataclass
class DescriptorParams:
    """Parameters of the species-resolved radial + angular descriptor: the modified angular
    term (angular = "mbp": theta_s, rs_ang, eta_ang, zeta) or the standard BP term
    (angular = "bp": per-sector lambda and zeta, per-shell eta)."""
    n_species: int
    rc: float
    rs_rad: np.ndarray
    eta_rad: float
    rs_ang: np.ndarray
    theta_s: np.ndarray
    eta_ang: float
    zeta: float
    eps_theta: float = 1e-6
    angular: str = "mbp"
    bp_lambda: Optional[np.ndarray] = None
    bp_zeta: Optional[np.ndarray] = None
    bp_eta: Optional[np.ndarray] = None

    @property
    def n_rad(self) -> int:
        return int(len(self.rs_rad))

    @property
    def n_ang_r(self) -> int:
        return int(len(self.bp_eta)) if self.angular == "bp" else int(len(self.rs_ang))

    @property
    def n_theta(self) -> int:
        return int(len(self.bp_lambda)) if self.angular == "bp" else int(len(self.theta_s))

    @property
    def D(self) -> int:
        s = self.n_species
        return s * self.n_rad + s * (s + 1) // 2 * self.n_theta * self.n_ang_r


@dataclasses.dataclass
class MLPArch:
    """widths = (D, h1, ..., 1); acts[l] is the activation of layer l+1."""
    widths: tuple
    acts: tuple

    @property
    def n_layers(self) -> int:
        return len(self.widths) - 1

    @property
    def n_params(self) -> int:
        return sum(self.widths[l + 1] * self.widths[l] + self.widths[l + 1]
                   for l in range(self.n_layers))


@dataclasses.dataclass
class Workload:
    name: str
    system: System
    desc: DescriptorParams
    archs: List[MLPArch]          # one per species
    theta: np.ndarray             # float64, all species' parameters, see pack order below
    mlp_bf16: bool                # precision the workload asks for in the network
    e_ref: Optional[np.ndarray] = None   # float64 [C] training labels
    f_ref: Optional[np.ndarray] = None   # float64 [N,3]
    w_force: float = 0.1
    seed: int = 0
    # charge equilibration (3-output networks): per-species Gaussian widths, reference
    # electronegativities and hardnesses, and the total charge of every configuration
    qeq: Optional[dict] = None
    charge: Optional[np.ndarray] = None

    @property
    def param_offsets(self) -> np.ndarray:
        return param_offsets(self.archs)


def param_offsets(archs: Sequence[MLPArch]) -> np.ndarray:
    """Start of each species' block in the flat parameter vector (int64 [S+1]).

    Inside a species block the layers follow in order, each as W (row-major
    [n_out, n_in]) followed by b [n_out]; layer l computes z = W a + b.
    """
    off = [0]
    for a in archs:
        off.append(off[-1] + a.n_params)
    return np.asarray(off, dtype=np.int64)


# ----------------------------------------------------------------------------------
# geometry helpers (input validation only)
# ----------------------------------------------------------------------------------

def _pairs_cubic_box(pos: np.ndarray, L: float, rmax: float):
    """All atom pairs (i<j) closer than rmax under the minimum image (needs L > 2 rmax)."""
    from scipy.spatial import cKDTree
    p = np.mod(pos, L)
    p[p >= L] = 0.0
    tree = cKDTree(p, boxsize=L)
    pairs = tree.query_pairs(rmax, output_type="ndarray")
    if len(pairs) == 0:
        return pairs, np.zeros(0)
    d = p[pairs[:, 1]] - p[pairs[:, 0]]
    d -= L * np.round(d / L)
    return pairs, np.sqrt((d * d).sum(1))


def _all_image_distances(pos: np.ndarray, L: Optional[float], rmax: float):
    """(i, j, r) for every pair of entries with r < rmax, all periodic images (small boxes)."""
    n = len(pos)
    if L is None:
        shifts = np.zeros((1, 3))
    else:
        k = int(math.ceil(rmax / L)) + 1
        g = np.arange(-k, k + 1)
        shifts = np.stack(np.meshgrid(g, g, g, indexing="ij"), -1).reshape(-1, 3) * L
    out_i, out_j, out_r = [], [], []
    for s in shifts:
        d = pos[None, :, :] + s[None, None, :] - pos[:, None, :]
        r = np.sqrt((d * d).sum(-1))
        if not np.any(s):
            r[np.arange(n), np.arange(n)] = np.inf
        ii, jj = np.nonzero(r < rmax)
        out_i.append(ii)
        out_j.append(jj)
        out_r.append(r[ii, jj])
    return np.concatenate(out_i), np.concatenate(out_j), np.concatenate(out_r)


def _violations(r: np.ndarray, rc: float, dmin: float) -> np.ndarray:
    return (r < dmin) | (np.abs(r - rc) < 2 * CUTOFF_MARGIN)


def _bad_atoms_cubic(pos: np.ndarray, L: Optional[float], rc: float, dmin: float,
                     only: Optional[np.ndarray] = None) -> np.ndarray:
    """Atoms taking part in a pair closer than dmin or within CUTOFF_MARGIN of rc.

    With ``only`` given, just the pairs that involve those atoms are examined and the
    offending atoms among ``only`` are returned.
    """
    rmax = rc + 4 * CUTOFF_MARGIN
    if L is None or L <= 2 * rmax:
        ii, jj, r = _all_image_distances(pos, L, rmax)
        bad = _violations(r, rc, dmin)
        if only is None:
            return np.unique(np.maximum(ii[bad], jj[bad]))
        sel = np.isin(ii[bad], only)
        return np.unique(ii[bad][sel])
    if only is None:
        pairs, r = _pairs_cubic_box(pos, L, rmax)
        if len(r) == 0:
            return np.zeros(0, np.int64)
        return np.unique(pairs[_violations(r, rc, dmin), 1])
    from scipy.spatial import cKDTree
    p = np.mod(pos, L)
    p[p >= L] = 0.0
    tree = cKDTree(p, boxsize=L)
    out = []
    for a, nb in zip(only, tree.query_ball_point(p[only], rmax)):
        nb = np.asarray([b for b in nb if b != a], dtype=np.int64)
        if len(nb) == 0:
            continue
        d = p[nb] - p[a]
        d -= L * np.round(d / L)
        if np.any(_violations(np.sqrt((d * d).sum(1)), rc, dmin)):
            out.append(a)
    return np.asarray(out, dtype=np.int64)


def _random_box(rng: np.random.Generator, n: int, L: float, rc: float, dmin: float) -> np.ndarray:
    """Uniform random positions in a periodic cube with a minimum separation (re-draws)."""
    pos = rng.uniform(0.0, L, size=(n, 3))
    bad = _bad_atoms_cubic(pos, L, rc, dmin)
    for _ in range(10000):
        if len(bad) == 0:
            return pos
        pos[bad] = rng.uniform(0.0, L, size=(len(bad), 3))
        bad = _bad_atoms_cubic(pos, L, rc, dmin, only=bad)
    raise RuntimeError("could not place atoms")


def _perturbed_lattice(rng, frac_basis, ncell, a, sigma, rc) -> np.ndarray:
    g = np.arange(ncell)
    cells = np.stack(np.meshgrid(g, g, g, indexing="ij"), -1).reshape(-1, 1, 3)
    ideal = ((cells + frac_basis[None, :, :]) * a).reshape(-1, 3)
    L = ncell * a
    pos = ideal + rng.normal(0.0, sigma, size=ideal.shape)
    bad = _bad_atoms_cubic(pos, L, rc, 0.0)
    for _ in range(10000):
        if len(bad) == 0:
            return np.mod(pos, L)
        pos[bad] = ideal[bad] + rng.normal(0.0, sigma, size=(len(bad), 3))
        bad = _bad_atoms_cubic(pos, L, rc, 0.0, only=bad)
    raise RuntimeError("could not displace lattice")


DIAMOND_BASIS = np.array([[0, 0, 0], [0, .5, .5], [.5, 0, .5], [.5, .5, 0],
                          [.25, .25, .25], [.25, .75, .75], [.75, .25, .75], [.75, .75, .25]])
FCC_BASIS = np.array([[0, 0, 0], [0, .5, .5], [.5, 0, .5], [.5, .5, 0]])


def _chain_molecule(rng, n: int, rc: float, dmin: float = 0.9) -> np.ndarray:
    """Random bonded chain: bond lengths U[1.0, 1.5], every pair at least dmin apart."""
    while True:
        pos = np.zeros((n, 3))
        ok = True
        for k in range(1, n):
            for _ in range(200):
                v = rng.normal(size=3)
                v /= np.linalg.norm(v)
                p = pos[k - 1] + rng.uniform(1.0, 1.5) * v
                d = np.sqrt(((pos[:k] - p) ** 2).sum(1))
                if d.min() >= dmin and np.all(np.abs(d - rc) >= 2 * CUTOFF_MARGIN):
                    pos[k] = p
                    break
            else:
                ok = False
                break
        if ok:
            return pos


# ----------------------------------------------------------------------------------
# parameters and weights
# ----------------------------------------------------------------------------------

def descriptor_params(n_species, rc, n_rad, n_theta, n_ang_r, eta_rad=16.0, eta_ang=12.0,
                      zeta=50.0, r_min=0.5, eps_theta=1e-6) -> DescriptorParams:
    """Uniform grids as inclusive linspaces: R_s on [r_min, rc], theta_s on [0, pi]."""
    return DescriptorParams(
        n_species=n_species, rc=float(rc),
        rs_rad=np.linspace(r_min, rc, n_rad), eta_rad=float(eta_rad),
        rs_ang=np.linspace(r_min, rc, n_ang_r),
        theta_s=np.linspace(0.0, math.pi, n_theta), eta_ang=float(eta_ang),
        zeta=float(zeta), eps_theta=float(eps_theta))


def init_weights(rng, desc: DescriptorParams, archs: Sequence[MLPArch],
                 rad_gain: float, ang_gain: float) -> np.ndarray:
    """Xavier/Glorot-uniform weights, small uniform biases.

    The first layer's columns are multiplied by a per-block gain (radial columns by
    ``rad_gain``, angular columns by ``ang_gain``); the gains are recipe constants per
    workload, picked so that first-layer pre-activations are O(1) and Gaussian units do
    not saturate on these geometries.
    """
    n_rad_cols = desc.n_species * desc.n_rad
    theta = []
    for a in archs:
        for l in range(a.n_layers):
            fi, fo = a.widths[l], a.widths[l + 1]
            lim = math.sqrt(6.0 / (fi + fo))
            W = rng.uniform(-lim, lim, size=(fo, fi))
            if l == 0:
                W[:, :n_rad_cols] *= rad_gain
                W[:, n_rad_cols:] *= ang_gain
            b = rng.uniform(-0.5, 0.5, size=fo)
            theta.append(W.ravel())
            theta.append(b)
    return np.concatenate(theta).astype(np.float64)


def _mlp(D, hidden, act=ACT_GAUSSIAN) -> MLPArch:
    widths = (D,) + tuple(hidden) + (1,)
    return MLPArch(widths, tuple([act] * len(hidden) + [ACT_LINEAR]))


# ----------------------------------------------------------------------------------
# the workloads
# ----------------------------------------------------------------------------------

def diamond64(seed: int = 0, ncell: int = 2) -> Workload:
    """Diamond lattice, a=5.43 A, sigma=0.1 A displacements, one species, rc=4.6 A."""
    rng = np.random.default_rng(seed)
    a, rc = 5.43, 4.6
    pos = _perturbed_lattice(rng, DIAMOND_BASIS, ncell, a, 0.1, rc)
    n = len(pos)
    L = ncell * a
    sysm = System(np.array([0, n], np.int64), pos, np.zeros(n, np.int32),
                  (np.eye(3) * L).reshape(1, 9), np.ones((1, 3), np.uint8), 1)
    desc = descriptor_params(1, rc, 32, 8, 8)
    archs = [_mlp(desc.D, (256, 128, 32))]
    theta = init_weights(rng, desc, archs, *GAINS["diamond64"])
    return Workload("diamond64", sysm, desc, archs, theta, mlp_bf16=False, seed=seed)


def molecules(seed: int = 0, n_mol: int = 1024) -> Workload:
    """Isolated random bonded chains, 5..29 atoms, H/C/N/O = .5/.3/.1/.1, rc=5.2 A."""
    rng = np.random.default_rng(seed)
    rc = 5.2
    sizes = rng.integers(5, 30, size=n_mol)
    pos, spec, off = [], [], [0]
    for n in sizes:
        pos.append(_chain_molecule(rng, int(n), rc))
        spec.append(rng.choice(4, size=int(n), p=[0.5, 0.3, 0.1, 0.1]).astype(np.int32))
        off.append(off[-1] + int(n))
    sysm = System(np.asarray(off, np.int64), np.concatenate(pos), np.concatenate(spec),
                  np.zeros((n_mol, 9)), np.zeros((n_mol, 3), np.uint8), 4)
    desc = descriptor_params(4, rc, 32, 8, 8)
    archs = [_mlp(desc.D, (128, 32)) for _ in range(4)]
    theta = init_weights(rng, desc, archs, *GAINS["molecules1024"])
    counts = np.diff(sysm.atom_off).astype(np.float64)
    e_ref = rng.normal(0.0, 1.0, size=n_mol) * np.sqrt(counts)
    f_ref = rng.normal(0.0, 0.5, size=(sysm.n_atoms, 3))
    name = "molecules1024" if n_mol == 1024 else "molecules%d" % n_mol
    return Workload(name, sysm, desc, archs, theta, mlp_bf16=False,
                    e_ref=e_ref, f_ref=f_ref, w_force=0.1, seed=seed)


def water(seed: int = 0, n_atoms: int = 32768) -> Workload:
    """Random liquid-like box, O:H = 1:2, 0.1003 atoms/A^3 (1 g/cm^3 water), rc=6 A."""
    rng = np.random.default_rng(seed)
    rc = 6.0
    L = (n_atoms / 0.1003) ** (1.0 / 3.0)
    pos = _random_box(rng, n_atoms, L, rc, 0.9)
    n_o = int(round(n_atoms / 3))
    spec = np.ones(n_atoms, np.int32)
    spec[rng.permutation(n_atoms)[:n_o]] = 0
    sysm = System(np.array([0, n_atoms], np.int64), pos, spec,
                  (np.eye(3) * L).reshape(1, 9), np.ones((1, 3), np.uint8), 2)
    desc = descriptor_params(2, rc, 32, 8, 8)
    archs = [_mlp(desc.D, (256, 128)) for _ in range(2)]
    theta = init_weights(rng, desc, archs, *GAINS["water32k"])
    name = "water32k" if n_atoms == 32768 else "water%d" % n_atoms
    return Workload(name, sysm, desc, archs, theta, mlp_bf16=True, seed=seed)


def fcc(seed: int = 0, ncell: int = 64) -> Workload:
    """FCC lattice, a=4.05 A, sigma=0.05 A, one species, rc=5 A, 64 + 16x8 components."""
    rng = np.random.default_rng(seed)
    a, rc = 4.05, 5.0
    pos = _perturbed_lattice(rng, FCC_BASIS, ncell, a, 0.05, rc)
    n = len(pos)
    sysm = System(np.array([0, n], np.int64), pos, np.zeros(n, np.int32),
                  (np.eye(3) * ncell * a).reshape(1, 9), np.ones((1, 3), np.uint8), 1)
    desc = descriptor_params(1, rc, 64, 16, 8)
    archs = [_mlp(desc.D, (128, 64))]
    theta = init_weights(rng, desc, archs, *GAINS["fcc1m"])
    name = "fcc1m" if ncell == 64 else "fcc%d" % n
    return Workload(name, sysm, desc, archs, theta, mlp_bf16=True, seed=seed)


def ragged(seed: int = 0, n_cfg: int = 4096, n_min: int = 32, n_max: int = 4096) -> Workload:
    """Periodic cubic boxes, N log-uniform on [n_min, n_max], 3 species in Dirichlet(1,1,1)
    proportions, 0.05 atoms/A^3, minimum separation 0.9 A, rc=5.5 A."""
    rng = np.random.default_rng(seed)
    rc = 5.5
    sizes = np.rint(np.exp(rng.uniform(math.log(n_min), math.log(n_max), size=n_cfg))).astype(np.int64)
    pos, spec, cells, off = [], [], [], [0]
    for n in sizes:
        L = (n / 0.05) ** (1.0 / 3.0)
        pos.append(_random_box(rng, int(n), L, rc, 0.9))
        p = rng.dirichlet([1.0, 1.0, 1.0])
        spec.append(rng.choice(3, size=int(n), p=p).astype(np.int32))
        cells.append((np.eye(3) * L).ravel())
        off.append(off[-1] + int(n))
    sysm = System(np.asarray(off, np.int64), np.concatenate(pos), np.concatenate(spec),
                  np.asarray(cells), np.ones((n_cfg, 3), np.uint8), 3)
    desc = descriptor_params(3, rc, 32, 8, 8)
    archs = [_mlp(desc.D, (128, 32)) for _ in range(3)]
    theta = init_weights(rng, desc, archs, *GAINS["ragged4096"])
    name = "ragged4096" if n_cfg == 4096 else "ragged%d" % n_cfg
    return Workload(name, sysm, desc, archs, theta, mlp_bf16=True, seed=seed)


# First-layer gains (radial, angular) per workload; see init_weights.
def _small_cell_margin_ok(pos, L, rc) -> bool:
    """Brute force over every image in an orthorhombic box: no pair distance within
    CUTOFF_MARGIN of rc (small boxes only)."""
    L = np.asarray(L, np.float64)
    m = np.ceil(rc / L).astype(int) + 1
    shifts = np.stack(np.meshgrid(*[np.arange(-k, k + 1) for k in m], indexing="ij"), -1).reshape(-1, 3) * L
    d = pos[None, :, None, :] + shifts[None, None, :, :] - pos[:, None, None, :]
    r = np.sqrt((d ** 2).sum(-1))
    return not np.any(np.abs(r - rc) < CUTOFF_MARGIN)


def carbon16(seed: int = 0, replicas: int = 1) -> Workload:
    """Diamond carbon, 2 x 1 x 1 conventional cells (16 atoms, a = 3.567 A, sigma = 0.05 A),
    rc = 5.0 A; descriptor 24 radial shells + 8 R x 16 theta angular bins (D = 152) and the
    small network 64 - 32 of the paper's carbon tests (Sec. III.B).  `replicas` independent
    copies (each its own displacements) form a batch for batched dynamics."""
    rng = np.random.default_rng(seed)
    a, rc = 3.567, 5.0
    L = np.array([2 * a, a, a])
    ideal = np.concatenate([(DIAMOND_BASIS + np.array([cx, 0, 0])) * a for cx in range(2)])
    pos_all = []
    for _ in range(replicas):
        for _ in range(10000):
            pos = np.mod(ideal + rng.normal(0.0, 0.05, size=ideal.shape), L)
            if _small_cell_margin_ok(pos, L, rc):
                break
        else:
            raise RuntimeError("could not displace the carbon cell")
        pos_all.append(pos)
    n = len(ideal)
    off = np.arange(replicas + 1, dtype=np.int64) * n
    sysm = System(off, np.concatenate(pos_all), np.zeros(n * replicas, np.int32),
                  np.tile(np.diag(L).reshape(1, 9), (replicas, 1)), np.ones((replicas, 3), np.uint8), 1)
    desc = descriptor_params(1, rc, 24, 16, 8)
    archs = [_mlp(desc.D, (64, 32))]
    theta = init_weights(rng, desc, archs, *GAINS["carbon16"])
    return Workload("carbon16" if replicas == 1 else "carbon16x%d" % replicas, sysm, desc, archs, theta,
                    mlp_bf16=False, seed=seed)


def nacl(seed: int = 0, n_clusters: int = 2) -> Workload:
    """Charged sodium chloride clusters shaped like those of Sec. III.C: Na9Cl8+ (a 3 x 3 x 2
    rock-salt block, a = 5.64 A, with one Cl removed) and Na8Cl8+ (a corner Na removed as
    well), alternating, each with total charge +1, displaced by sigma = 0.1 A and rotated at
    random; no periodicity.  Species Na = 0, Cl = 1.  Descriptor of size 45 (9 radial shells
    per species, 3 theta x 3 R angular bins), rc = 6 A; networks 45-15-15-3 (local energy,
    electronegativity and hardness corrections).  Charge-equilibration constants: Gaussian
    widths 1.0 / 1.2 A and reference electronegativity / hardness from the atoms' Mulliken
    values (2.85 / 8.30 eV and 4.59 / 9.35 eV)."""
    rng = np.random.default_rng(seed)
    a, rc = 5.64, 6.0
    sites, spec = [], []
    for i in range(3):
        for j in range(3):
            for k in range(2):
                sites.append([i, j, k])
                spec.append((i + j + k) % 2)     # Na on even sites: 9 Na, 9 Cl
    sites = np.array(sites, np.float64) * (a / 2)
    spec = np.array(spec, np.int32)
    cl = np.nonzero(spec == 1)[0]
    drop_cl = cl[len(cl) // 2]                    # a central-layer Cl
    na9 = np.array([q for q in range(len(spec)) if q != drop_cl])
    na8 = na9[1:]                                  # the corner Na at the origin as well
    pos_all, spec_all, off = [], [], [0]
    for c in range(n_clusters):
        keep = na9 if c % 2 == 0 else na8
        x = sites[keep] - sites[keep].mean(0)
        q, _ = np.linalg.qr(rng.normal(size=(3, 3)))
        x = x @ q.T + rng.normal(0.0, 0.1, size=x.shape) + rng.uniform(-20, 20, size=3)
        pos_all.append(x)
        spec_all.append(spec[keep])
        off.append(off[-1] + len(keep))
    C = n_clusters
    sysm = System(np.asarray(off, np.int64), np.concatenate(pos_all), np.concatenate(spec_all),
                  np.zeros((C, 9)), np.zeros((C, 3), np.uint8), 2)
    desc = descriptor_params(2, rc, 9, 3, 3, eta_rad=2.0, eta_ang=1.5, zeta=4.0)
    archs = [MLPArch((desc.D, 15, 15, 3), (ACT_GAUSSIAN, ACT_GAUSSIAN, ACT_LINEAR)) for _ in range(2)]
    theta = init_weights(rng, desc, archs, *GAINS["nacl"])
    # small output layers: corrections of O(0.1) to the reference constants
    off_p = param_offsets(archs)
    for sp in range(2):
        o = off_p[sp] + 45 * 15 + 15 + 15 * 15 + 15
        theta[o:o + 3 * 15 + 3] *= 0.2
    qeq = dict(sigma=np.array([1.0, 1.2]), chi0=np.array([2.85, 8.30]), hard0=np.array([4.59, 9.35]))
    return Workload("nacl%d" % n_clusters, sysm, desc, archs, theta, mlp_bf16=False, seed=seed, qeq=qeq,
                    charge=np.ones(C))


GAINS = {
    "diamond64": (3.5, 4.5),
    "molecules1024": (4.0, 2.0),
    "water32k": (1.5, 0.3),
    "fcc1m": (0.9, 0.9),
    "ragged4096": (3.5, 2.2),
    "carbon16": (0.7, 0.1),
    "nacl": (0.6, 0.4),
}


def bp_variant(wl: Workload, rad_gain: float, ang_gain: float, lambdas=(1.0, -1.0, 1.0, -1.0),
               zetas=(1.0, 1.0, 4.0, 4.0), etas=(0.005, 0.05)) -> Workload:
    """The same configurations with the standard BP angular term (Sec. II.A) in place of the
    modified one: sectors (lambda_m, zeta_m), shells eta_n (A^-2); networks re-sized to the new D
    and re-drawn (first-layer angular columns scaled by ang_gain)."""
    rng = np.random.default_rng(wl.seed + 7)
    desc = dataclasses.replace(wl.desc, angular="bp", bp_lambda=np.asarray(lambdas, np.float64),
                               bp_zeta=np.asarray(zetas, np.float64), bp_eta=np.asarray(etas, np.float64))
    archs = [MLPArch((desc.D,) + tuple(a.widths[1:]), a.acts) for a in wl.archs]
    theta = init_weights(rng, desc, archs, rad_gain, ang_gain)
    return dataclasses.replace(wl, name=wl.name + "_bp", desc=desc, archs=archs, theta=theta)


# Workloads whose generation takes more than a few seconds are kept in a per-machine cache
# (a pickle keyed by name, seed and a hash of this file, so any change of the recipe makes
# a new entry); PANNA_WORKLOAD_CACHE="" switches it off.
_CACHED = ("ragged4096", "fcc1m")


def _cache_path(name: str, seed: int) -> Optional[str]:
    import hashlib
    import os
    import tempfile
    root = os.environ.get("PANNA_WORKLOAD_CACHE", os.path.join(tempfile.gettempdir(), "panna_workloads"))
    if not root:
        return None
    with open(os.path.abspath(__file__), "rb") as f:
        h = hashlib.sha256(f.read()).hexdigest()[:16]
    return os.path.join(root, "%s_seed%d_%s.pkl" % (name, seed, h))


def make(name: str, seed: int = 0) -> Workload:
    """Workload by name, including the small variants used by the CPU oracle."""
    path = _cache_path(name, seed) if name in _CACHED else None
    if path:
        import os
        import pickle
        try:
            with open(path, "rb") as f:
                return pickle.load(f)
        except (OSError, EOFError, pickle.UnpicklingError):
            pass
        wl = _make(name, seed)
        try:
            os.makedirs(os.path.dirname(path), exist_ok=True)
            tmp = "%s.%d.tmp" % (path, os.getpid())
            with open(tmp, "wb") as f:
                pickle.dump(wl, f, protocol=pickle.HIGHEST_PROTOCOL)
            os.replace(tmp, path)
        except OSError:
            pass
        return wl
    return _make(name, seed)


def _make(name: str, seed: int) -> Workload:
    table = {
        "diamond64": lambda: diamond64(seed),
        "molecules1024": lambda: molecules(seed, 1024),
        "molecules16": lambda: molecules(seed, 16),
        "water32k": lambda: water(seed, 32768),
        "water512": lambda: water(seed, 512),
        "fcc1m": lambda: fcc(seed, 64),
        "fcc256": lambda: fcc(seed, 4),
        "fcc4000": lambda: fcc(seed, 10),
        "fcc32k": lambda: fcc(seed, 20),
        "ragged4096": lambda: ragged(seed, 4096),
        "ragged8": lambda: ragged(seed, 8, 32, 160),
        "carbon16": lambda: carbon16(seed),
        "carbon16x64": lambda: carbon16(seed, 64),
        "carbon16x4096": lambda: carbon16(seed, 4096),
        "molecules16_bp": lambda: bp_variant(molecules(seed, 16), 1.0, 0.3),
        "molecules1024_bp": lambda: bp_variant(molecules(seed, 1024), 1.0, 0.3),
        "water512_bp": lambda: bp_variant(water(seed, 512), 1.0, 0.05),
        "nacl2": lambda: nacl(seed, 2),
        "nacl64": lambda: nacl(seed, 64),
        "nacl4096": lambda: nacl(seed, 4096),
    }
    return table[name]()
