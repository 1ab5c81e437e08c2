"""How the path shards over ranks, one process per GPU (host-side layout and exchanges).

The energy is a sum of atomic terms, each a function of the atom's neighbours within the
cutoff rc (Sec. I, Sec. II), so the work splits in two ways:

* By configuration.  A ragged batch of independent configurations is cut into contiguous
  ranges of nearly equal cost (angular pairs plus radial entries).  Energies and forces
  need no exchange at all.  For training each rank normalises its loss by the GLOBAL
  counts (``panna_set_loss_normalization``), so that the ranks' losses and parameter
  gradients add up, with one all-reduce, to those of the whole batch (Sec. II.A).

* By space.  One large configuration is cut into slabs along its third lattice vector
  (in fractional coordinates, so triclinic cells work too).  A rank holds the atoms of its
  slab, followed by every periodic image of any atom that lies within rc (+ skin) of the
  slab: the ghosts.  It evaluates its own centres only (``panna_system.ghost``); forces on
  ghosts go back to the atoms they stand for (reverse halo exchange), energies and
  virials are summed over ranks.  Ghost positions are refreshed from their owners with
  the forward halo exchange.  A plan stays valid while no atom has moved more than skin/2
  (the usual Verlet-skin argument); then it is rebuilt.

Nothing here does arithmetic of the method; the exchanges move positions and forces
(``torch.distributed.all_to_all_single``: NCCL on GPUs, gloo on CPU).
"""
from __future__ import annotations

import dataclasses
import math
from typing import List, Optional, Sequence

import numpy as np

from .workloads import System


# ------------------------------------------------------------------ by configuration

def exact_costs(nbr_off: np.ndarray, atom_off: np.ndarray) -> np.ndarray:
    """Cost of each configuration from a neighbour list's CSR offsets: sum over its atoms
    of nb (radial entries) + nb(nb-1)/2 (angular pairs)."""
    nb = np.diff(np.asarray(nbr_off, np.int64)).astype(np.float64)
    per_atom = nb + nb * (nb - 1.0) / 2.0
    csum = np.concatenate([[0.0], np.cumsum(per_atom)])
    off = np.asarray(atom_off, np.int64)
    return csum[off[1:]] - csum[off[:-1]]


def estimated_costs(system: System, rc: float) -> np.ndarray:
    """Cost estimate without a neighbour list: nb from the number density of a periodic
    configuration, n - 1 for an isolated one (small molecules lie within rc)."""
    n = np.diff(system.atom_off).astype(np.float64)
    cost = np.zeros(system.n_cfg)
    ball = 4.0 / 3.0 * math.pi * rc ** 3
    for c in range(system.n_cfg):
        if system.pbc[c].any():
            vol = abs(np.linalg.det(system.cell[c].reshape(3, 3)))
            nb = n[c] / vol * ball
        else:
            nb = max(n[c] - 1.0, 0.0)
        cost[c] = n[c] * (nb + nb * max(nb - 1.0, 0.0) / 2.0)
    return cost


def shard_bounds(costs: Sequence[float], world: int) -> np.ndarray:
    """Contiguous ranges of configurations, rank r taking bounds[r]:bounds[r+1], cut where
    the cumulative cost (at each configuration's midpoint) crosses r / world of the total.
    A rank may get an empty range when there are fewer configurations than ranks."""
    c = np.asarray(costs, np.float64)
    if world < 1:
        raise ValueError("world must be >= 1")
    total = float(c.sum())
    if c.size == 0 or total <= 0.0:
        return np.linspace(0, c.size, world + 1).round().astype(np.int64)
    mid = np.cumsum(c) - c / 2.0
    cuts = np.searchsorted(mid, total * np.arange(1, world) / world, side="left")
    return np.concatenate([[0], cuts, [c.size]]).astype(np.int64)


def global_counts(n_cfg: int, n_atoms: int, group=None):
    """(configurations, atoms) summed over the ranks of ``group`` (all-reduce)."""
    import torch
    import torch.distributed as dist
    dev = "cuda" if dist.get_backend(group) == "nccl" else "cpu"
    t = torch.tensor([n_cfg, n_atoms], dtype=torch.int64, device=dev)
    dist.all_reduce(t, group=group)
    return int(t[0].item()), int(t[1].item())


# ------------------------------------------------------------------ by space

@dataclasses.dataclass
class LocalDomain:
    """Rank-local view of a slab decomposition.

    Local atoms are the owned ones (global indices ``owned``, ascending) followed by the
    ghosts, ordered by owning rank; ghost g stands for global atom ``ghost_src[g]`` shifted
    by ``ghost_img[g]`` third lattice vectors (relative to the folded position)."""
    rank: int
    owned: np.ndarray
    ghost_src: np.ndarray
    ghost_img: np.ndarray
    recv_counts: np.ndarray      # [world] ghosts owned by each rank
    send_idx: List[np.ndarray]   # [world] owned-local rows that rank q holds as ghosts, in q's order
    system: System               # one configuration: owned then ghosts, no PBC along a3
    ghost: np.ndarray            # [n_local] uint8 flags

    @property
    def n_owned(self) -> int:
        return int(self.owned.size)


class SlabPlan:
    """Slab decomposition of ONE configuration over ``world`` ranks along lattice vector a3.

    Built identically on every rank from the same positions.  ``width`` = rc + skin is the
    ghost shell thickness; slabs may be thinner than it (ghosts then come from several
    slabs and images)."""

    def __init__(self, system: System, rc: float, world: int, skin: float = 0.0):
        if system.n_cfg != 1:
            raise ValueError("a slab plan decomposes a single configuration")
        if world < 1:
            raise ValueError("world must be >= 1")
        cell = system.cell[0].reshape(3, 3).astype(np.float64)
        det = float(np.linalg.det(cell))
        if abs(det) < 1e-12:
            raise ValueError("slab decomposition needs a non-singular cell")
        self.world = int(world)
        self.rc = float(rc)
        self.skin = float(skin)
        self.cell = cell
        self.pbc = system.pbc[0].astype(np.uint8).copy()
        self.species = system.species.astype(np.int32)
        self.n_atoms = system.n_atoms
        a3 = cell[2]
        h3 = abs(det) / float(np.linalg.norm(np.cross(cell[0], cell[1])))   # spacing of planes s3 = const
        s3 = (system.pos @ np.linalg.inv(cell))[:, 2]
        if self.pbc[2]:
            fold = np.floor(s3)
            f = s3 - fold
            wrap = f >= 1.0                  # rounding of s3 - floor(s3) for tiny negative s3
            f[wrap] -= 1.0
            fold[wrap] += 1.0
            bounds = np.arange(world + 1, dtype=np.float64) / world
        else:
            fold = np.zeros_like(s3)
            f = s3.copy()
            lo3 = float(s3.min()) if s3.size else 0.0
            span = (float(s3.max()) - lo3) * (1.0 + 1e-12) + 1e-12 if s3.size else 1.0
            bounds = lo3 + span * np.arange(world + 1, dtype=np.float64) / world
        self.bounds3 = bounds
        self.pos_folded = system.pos - fold[:, None] * a3[None, :]
        self._pos_ref = system.pos.copy()
        # ownership and the ghost intervals below use the same bounds, so an atom on a
        # boundary is owned by exactly one rank and a ghost wherever it is needed
        self.owner = np.clip(np.searchsorted(bounds, f, side="right") - 1, 0, world - 1).astype(np.int64)
        w = (rc + skin) / h3
        M = int(math.ceil(w)) + 1 if self.pbc[2] else 0
        ghosts = []   # per rank: (owner, src, img)
        for r in range(world):
            lo, hi = bounds[r], bounds[r + 1]
            rows = []
            for m in range(-M, M + 1):
                fm = f + m
                sel = ((fm >= lo - w) & (fm < lo)) | ((fm >= hi) & (fm < hi + w))
                if m == 0:
                    sel &= self.owner != r
                idx = np.nonzero(sel)[0]
                rows.append(np.stack([self.owner[idx], idx, np.full(idx.size, m)], axis=1))
            g = np.concatenate(rows) if rows else np.zeros((0, 3), np.int64)
            g = g[np.lexsort((g[:, 2], g[:, 1], g[:, 0]))]
            ghosts.append(g.astype(np.int64))
        owned = [np.nonzero(self.owner == r)[0] for r in range(world)]
        local_row = np.zeros(self.n_atoms, np.int64)
        for r in range(world):
            local_row[owned[r]] = np.arange(owned[r].size)
        self.domains: List[LocalDomain] = []
        for r in range(world):
            g = ghosts[r]
            recv = np.bincount(g[:, 0], minlength=world).astype(np.int64)
            send = []
            for q in range(world):
                gq = ghosts[q]
                send.append(local_row[gq[gq[:, 0] == r, 1]])
            src, img = g[:, 1], g[:, 2]
            pos = np.concatenate([self.pos_folded[owned[r]], self.pos_folded[src] + img[:, None] * a3[None, :]])
            spec = np.concatenate([self.species[owned[r]], self.species[src]]).astype(np.int32)
            n_loc = pos.shape[0]
            pbc = self.pbc.copy()
            pbc[2] = 0
            sysr = System(np.array([0, n_loc], np.int64), pos, spec, cell.reshape(1, 9).copy(),
                          pbc.reshape(1, 3), system.n_species)
            flags = np.concatenate([np.zeros(owned[r].size, np.uint8), np.ones(src.size, np.uint8)])
            self.domains.append(LocalDomain(r, owned[r], src, img, recv, send, sysr, flags))

    # ---------------------------------------------------------------- single process
    def gather_forces(self, F_local: Sequence[np.ndarray]) -> np.ndarray:
        """Global forces from every rank's local forces (owned rows plus ghost rows summed
        into the atoms they stand for): the reverse exchange done in one process."""
        F = np.zeros((self.n_atoms, 3))
        for d, Fl in zip(self.domains, F_local):
            Fl = np.asarray(Fl, np.float64).reshape(-1, 3)
            F[d.owned] += Fl[:d.n_owned]
            np.add.at(F, d.ghost_src, Fl[d.n_owned:])
        return F

    # ---------------------------------------------------------------- distributed
    def halo(self, rank: int, x_owned, group=None):
        """Forward halo exchange: positions [n_owned, 3] of this rank's atoms (folded frame)
        -> local positions [n_local, 3] (owned, then ghosts from their owners + image)."""
        import torch
        import torch.distributed as dist
        d = self.domains[rank]
        send_rows = torch.as_tensor(np.concatenate(d.send_idx), device=x_owned.device)
        sbuf = x_owned.index_select(0, send_rows).contiguous()
        rbuf = torch.empty((int(d.recv_counts.sum()), 3), dtype=x_owned.dtype, device=x_owned.device)
        dist.all_to_all_single(rbuf, sbuf, [int(k) for k in d.recv_counts],
                               [len(s) for s in d.send_idx], group=group)
        a3 = torch.as_tensor(self.cell[2], dtype=x_owned.dtype, device=x_owned.device)
        img = torch.as_tensor(d.ghost_img, dtype=x_owned.dtype, device=x_owned.device)
        return torch.cat([x_owned, rbuf + img[:, None] * a3[None, :]])

    def reverse(self, rank: int, F_local, group=None):
        """Reverse halo exchange: local forces [n_local, 3] -> complete forces on this rank's
        own atoms [n_owned, 3] (ghost rows added into the atoms they stand for)."""
        import torch
        import torch.distributed as dist
        d = self.domains[rank]
        n = d.n_owned
        sbuf = F_local[n:].contiguous()
        counts = [len(s) for s in d.send_idx]
        rbuf = torch.empty((sum(counts), 3), dtype=F_local.dtype, device=F_local.device)
        dist.all_to_all_single(rbuf, sbuf, counts, [int(k) for k in d.recv_counts], group=group)
        out = F_local[:n].clone()
        rows = torch.as_tensor(np.concatenate(d.send_idx), device=F_local.device)
        out.index_add_(0, rows, rbuf)
        return out

    def still_valid(self, pos_now: np.ndarray) -> bool:
        """True while no atom has moved more than skin/2 from the positions the plan was
        built from (same frame as those positions): every pair within rc is then still
        covered by the shell of width rc + skin."""
        d = np.sqrt(((np.asarray(pos_now) - self._pos_ref) ** 2).sum(1))
        return bool(d.max(initial=0.0) <= self.skin / 2)


class LocalSlabPlan:
    """The slab decomposition of SlabPlan, planned by every rank from its own atoms only.

    No rank holds the global positions: rank r is given the atoms it owns (those whose
    fractional coordinate along a3, folded into [0, 1) on a periodic a3, lies in
    [bounds3[r], bounds3[r + 1])), with their global indices and species.  Construction is
    collective over ``group``:

      1. each rank finds, among its own atoms and their images m along a3, those within
         w = (rc + skin) / h3 (fractional) of another slab (or of its own slab, through an
         image, when slabs are thinner than w): its send lists, one per destination rank,
         ordered by (global index, image);
      2. one all-to-all of the counts, one of (global index, species, image) records and one of
         the positions builds every rank's ghosts, ordered by owning rank, then as sent.

    ``halo`` refreshes the ghost positions from their owners and ``reverse`` returns the ghost
    forces to them (all-to-all exchanges of packed device tensors: index_select on the sender,
    index_add on the receiver); the rank's local system, ghost flags and exchange lists have
    the layout of SlabPlan's LocalDomain, so a rank's results equal those of the global plan.
    """

    def __init__(self, rank: int, world: int, cell, pbc, rc: float, skin: float, pos_owned: np.ndarray,
                 species_owned: np.ndarray, gid_owned: np.ndarray, bounds3: np.ndarray, n_species: int, group=None):
        import torch
        import torch.distributed as dist
        cell = np.asarray(cell, np.float64).reshape(3, 3)
        det = float(np.linalg.det(cell))
        if abs(det) < 1e-12:
            raise ValueError("slab decomposition needs a non-singular cell")
        self.rank, self.world = int(rank), int(world)
        self.cell = cell
        self.pbc = np.asarray(pbc, np.uint8).reshape(3).copy()
        self.rc, self.skin = float(rc), float(skin)
        self.bounds3 = np.asarray(bounds3, np.float64)
        a3 = cell[2]
        h3 = abs(det) / float(np.linalg.norm(np.cross(cell[0], cell[1])))
        w = (rc + skin) / h3
        pos = np.asarray(pos_owned, np.float64).reshape(-1, 3)
        s3 = (pos @ np.linalg.inv(cell))[:, 2] if len(pos) else np.zeros(0)
        if self.pbc[2]:
            fold = np.floor(s3)
            f = s3 - fold
            wrap = f >= 1.0
            f[wrap] -= 1.0
            fold[wrap] += 1.0
        else:
            fold = np.zeros_like(s3)
            f = s3.copy()
        lo_r, hi_r = self.bounds3[rank], self.bounds3[rank + 1]
        if np.any((f < lo_r) | (f >= hi_r)) and not (rank == world - 1 and np.all(f <= hi_r)):
            raise ValueError("rank %d was given atoms outside its slab" % rank)
        self.pos_folded = pos - fold[:, None] * a3[None, :]
        self._pos_ref = pos.copy()
        self.gid = np.asarray(gid_owned, np.int64)
        spec = np.asarray(species_owned, np.int32)
        M = int(math.ceil(w)) + 1 if self.pbc[2] else 0
        # 1. send lists
        send_rows, send_img = [], []
        for q in range(world):
            lo, hi = self.bounds3[q], self.bounds3[q + 1]
            rows, imgs = [], []
            for m in range(-M, M + 1):
                fm = f + m
                sel = ((fm >= lo - w) & (fm < lo)) | ((fm >= hi) & (fm < hi + w))
                idx = np.nonzero(sel)[0]
                rows.append(idx)
                imgs.append(np.full(idx.size, m, np.int64))
            rows = np.concatenate(rows) if rows else np.zeros(0, np.int64)
            imgs = np.concatenate(imgs) if imgs else np.zeros(0, np.int64)
            order = np.lexsort((imgs, self.gid[rows]))
            send_rows.append(rows[order].astype(np.int64))
            send_img.append(imgs[order])
        self.send_idx = send_rows
        # 2. exchanges: counts, records, positions
        scount = torch.tensor([len(r) for r in send_rows], dtype=torch.int64)
        rcount = torch.empty(world, dtype=torch.int64)
        dist.all_to_all_single(rcount, scount, group=group)
        self.recv_counts = rcount.numpy().astype(np.int64)
        rec = np.concatenate([np.stack([self.gid[r], spec[r].astype(np.int64), m], 1)
                              for r, m in zip(send_rows, send_img)]) if world else np.zeros((0, 3), np.int64)
        rrec = torch.empty((int(self.recv_counts.sum()), 3), dtype=torch.int64)
        dist.all_to_all_single(rrec, torch.as_tensor(rec.reshape(-1, 3)), [int(k) for k in self.recv_counts],
                               [len(r) for r in send_rows], group=group)
        rrec = rrec.numpy()
        self.ghost_src, ghost_spec, self.ghost_img = rrec[:, 0].copy(), rrec[:, 1].astype(np.int32), rrec[:, 2].copy()
        gpos = self.halo_numpy(self.pos_folded, group)
        n_own = len(pos)
        pbc_l = self.pbc.copy()
        pbc_l[2] = 0
        loc = np.concatenate([self.pos_folded, gpos])
        self.system = System(np.array([0, len(loc)], np.int64), loc, np.concatenate([spec, ghost_spec]),
                             cell.reshape(1, 9).copy(), pbc_l.reshape(1, 3), n_species)
        self.ghost = np.concatenate([np.zeros(n_own, np.uint8), np.ones(len(gpos), np.uint8)])
        self.n_owned = n_own

    def halo_numpy(self, x_owned: np.ndarray, group=None) -> np.ndarray:
        """Ghost positions (owners' folded positions plus the image shifts) as a numpy array."""
        import torch
        out = self._exchange_forward(torch.as_tensor(np.asarray(x_owned, np.float64)), group)
        return out.numpy()

    def _exchange_forward(self, x_owned, group=None):
        import torch
        import torch.distributed as dist
        rows = torch.as_tensor(np.concatenate(self.send_idx) if self.send_idx else np.zeros(0, np.int64),
                               device=x_owned.device)
        sbuf = x_owned.index_select(0, rows).contiguous()
        rbuf = torch.empty((int(self.recv_counts.sum()), 3), dtype=x_owned.dtype, device=x_owned.device)
        dist.all_to_all_single(rbuf, sbuf, [int(k) for k in self.recv_counts], [len(s) for s in self.send_idx],
                               group=group)
        a3 = torch.as_tensor(self.cell[2], dtype=x_owned.dtype, device=x_owned.device)
        img = torch.as_tensor(self.ghost_img, dtype=x_owned.dtype, device=x_owned.device)
        return rbuf + img[:, None] * a3[None, :]

    def halo(self, x_owned, group=None):
        """Forward halo exchange: this rank's folded positions [n_owned, 3] (a tensor on any
        device) -> local positions [n_local, 3], owned rows then ghosts."""
        import torch
        return torch.cat([x_owned, self._exchange_forward(x_owned, group)])

    def reverse(self, F_local, group=None):
        """Reverse halo exchange: local forces [n_local, 3] -> complete forces on the owned atoms."""
        import torch
        import torch.distributed as dist
        n = self.n_owned
        sbuf = F_local[n:].contiguous()
        counts = [len(s) for s in self.send_idx]
        rbuf = torch.empty((sum(counts), 3), dtype=F_local.dtype, device=F_local.device)
        dist.all_to_all_single(rbuf, sbuf, counts, [int(k) for k in self.recv_counts], group=group)
        out = F_local[:n].clone()
        rows = torch.as_tensor(np.concatenate(self.send_idx) if self.send_idx else np.zeros(0, np.int64),
                               device=F_local.device)
        out.index_add_(0, rows, rbuf)
        return out

    def still_valid(self, pos_now: np.ndarray, group=None) -> bool:
        """True on every rank while no atom of any rank has moved more than skin/2 since the
        plan was built (one all-reduce of the largest local displacement)."""
        import torch
        import torch.distributed as dist
        d = np.sqrt(((np.asarray(pos_now) - self._pos_ref) ** 2).sum(1))
        t = torch.tensor([float(d.max(initial=0.0))], dtype=torch.float64)
        dist.all_reduce(t, op=dist.ReduceOp.MAX, group=group)
        return bool(t.item() <= self.skin / 2)


def periodic_slab_bounds(world: int) -> np.ndarray:
    """Equal fractional slabs along a periodic a3: rank r owns [r / world, (r + 1) / world)."""
    return np.arange(world + 1, dtype=np.float64) / world


def owned_by_slab(system: System, bounds3: np.ndarray, rank: int) -> np.ndarray:
    """Indices of the atoms of a one-configuration system that rank ``rank`` owns under the
    slab bounds (folded fractional coordinate along a periodic a3): the initial distribution
    of atoms to ranks, after which each rank keeps only its own."""
    cell = system.cell[0].reshape(3, 3)
    s3 = (system.pos @ np.linalg.inv(cell))[:, 2]
    if system.pbc[0, 2]:
        f = s3 - np.floor(s3)
        f[f >= 1.0] -= 1.0
    else:
        f = s3
    world = len(bounds3) - 1
    owner = np.clip(np.searchsorted(bounds3, f, side="right") - 1, 0, world - 1)
    return np.nonzero(owner == rank)[0]
