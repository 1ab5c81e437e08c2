"""Host logic of the multi-rank path, on CPU: sharding by configuration, slab
decomposition with ghost atoms, and the exchanges themselves over torch.distributed
(gloo, world size 2), with the FP64 oracle doing each rank's arithmetic.

What must hold (Sec. II: the energy is a sum of atomic terms within rc):
* the ranks' energies, forces and virials combine to those of the whole configuration;
* with the global loss normalisers, the ranks' losses and parameter gradients sum to the
  whole batch's;
* every neighbour of every owned atom is present on its rank, at the same relative vector.
"""
import dataclasses
import os
import socket

import numpy as np
import pytest

from oracle import oracle as O
from paper_2305_11805_gb300 import domain as Dm
from paper_2305_11805_gb300 import workloads as W


def _triclinic(system):
    shear = np.array([[1.0, 0.0, 0.0], [0.15, 1.0, 0.0], [0.1, -0.2, 1.0]])
    return dataclasses.replace(system, pos=system.pos @ shear,
                               cell=(system.cell.reshape(3, 3) @ shear).reshape(1, 9))


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


# ------------------------------------------------------------------ by configuration

def test_shard_bounds_cover_and_balance():
    rng = np.random.default_rng(0)
    costs = rng.lognormal(size=257)
    for world in (1, 2, 3, 8):
        b = Dm.shard_bounds(costs, world)
        assert b[0] == 0 and b[-1] == costs.size and np.all(np.diff(b) >= 0)
        loads = np.array([costs[b[r]:b[r + 1]].sum() for r in range(world)])
        # a cut at a configuration's midpoint misses the ideal by at most that configuration
        assert loads.max() - costs.sum() / world <= costs.max() + 1e-9
    b = Dm.shard_bounds(np.ones(3), 5)          # fewer configurations than ranks
    assert b[0] == 0 and b[-1] == 3 and np.all(np.diff(b) >= 0)


def test_exact_costs_from_neighbour_offsets():
    wl = W.make("ragged8")
    i, _, _ = O.neighbor_list(wl.system, wl.desc.rc)
    nb = np.bincount(i, minlength=wl.system.n_atoms)
    off = np.concatenate([[0], np.cumsum(nb)])
    costs = Dm.exact_costs(off, wl.system.atom_off)
    for c in range(wl.system.n_cfg):
        a0, a1 = wl.system.atom_off[c], wl.system.atom_off[c + 1]
        want = sum(int(n) + int(n) * (int(n) - 1) // 2 for n in nb[a0:a1])
        assert costs[c] == want
    est = Dm.estimated_costs(wl.system, wl.desc.rc)
    assert np.corrcoef(est, costs)[0, 1] > 0.9


def test_shards_with_global_normalisers_add_up():
    wl = W.make("molecules16")
    s = wl.system
    b = Dm.shard_bounds(Dm.estimated_costs(s, wl.desc.rc), 3)
    full = O.batch(s, wl.desc, wl.archs, wl.theta, e_ref=wl.e_ref, f_ref=wl.f_ref, w_force=wl.w_force,
                   param_grad=True)
    loss, g = 0.0, 0.0
    for r in range(3):
        cfgs = list(range(b[r], b[r + 1]))
        sub = s.subset(cfgs)
        a0, a1 = s.atom_off[b[r]], s.atom_off[b[r + 1]]
        out = O.batch(sub, wl.desc, wl.archs, wl.theta, e_ref=wl.e_ref[cfgs], f_ref=wl.f_ref[a0:a1],
                      w_force=wl.w_force, param_grad=True, norm=(s.n_cfg, s.n_atoms))
        loss += out["loss"]
        g = g + out["dtheta"]
    assert abs(loss - full["loss"]) < 1e-12 * full["loss"]
    np.testing.assert_allclose(g, full["dtheta"], rtol=1e-9, atol=1e-12 * np.abs(full["dtheta"]).max())


# ------------------------------------------------------------------ by space

def _rel_vectors(system, rc, atom):
    i, j, sh = O.neighbor_list(system, rc)
    cell = system.cell[0].reshape(3, 3)
    sel = i == atom
    v = system.pos[j[sel]] + sh[sel] @ cell - system.pos[atom]
    return v[np.lexsort(v.T[::-1])]


@pytest.mark.parametrize("world", [1, 2, 3, 5])
def test_slab_plan_ownership_and_halo_cover_every_neighbour(world):
    wl = W.make("fcc256")
    for sysg in (wl.system, _triclinic(wl.system)):
        plan = Dm.SlabPlan(sysg, wl.desc.rc, world)
        owned = np.concatenate([d.owned for d in plan.domains])
        np.testing.assert_array_equal(np.sort(owned), np.arange(sysg.n_atoms))
        rng = np.random.default_rng(world)
        for d in plan.domains:
            assert d.system.pbc[0, 2] == 0 and d.ghost.sum() == d.ghost_src.size
            for q in rng.choice(d.n_owned, 3, replace=False):
                got = _rel_vectors(d.system, wl.desc.rc, int(q))
                want = _rel_vectors(sysg, wl.desc.rc, int(d.owned[q]))
                assert got.shape == want.shape
                np.testing.assert_allclose(got, want, atol=1e-9)


@pytest.mark.parametrize("world", [1, 2, 3, 5])
def test_slab_decomposition_matches_whole_configuration(world):
    wl = W.make("fcc256")
    for sysg in (wl.system, _triclinic(wl.system)):
        ref = O.batch(sysg, wl.desc, wl.archs, wl.theta)
        plan = Dm.SlabPlan(sysg, wl.desc.rc, world)
        parts = [O.batch(d.system, wl.desc, wl.archs, wl.theta, ghost=d.ghost) for d in plan.domains]
        F = plan.gather_forces([p["F"] for p in parts])
        E = sum(p["E_cfg"][0] for p in parts)
        V = sum(p["virial"][0] for p in parts)
        scale = np.abs(ref["F"]).max()
        assert np.abs(F - ref["F"]).max() < 1e-12 * scale
        assert abs(E - ref["E_cfg"][0]) < 1e-12 * np.abs(ref["E_atom"]).sum()
        assert np.abs(V - ref["virial"][0]).max() < 1e-11 * np.abs(ref["virial"]).max()
        for p, d in zip(parts, plan.domains):
            np.testing.assert_allclose(p["E_atom"][:d.n_owned], ref["E_atom"][d.owned], rtol=1e-12)


def test_slab_plan_skin_validity():
    wl = W.make("fcc256")
    plan = Dm.SlabPlan(wl.system, wl.desc.rc, 2, skin=0.4)
    p = wl.system.pos.copy()
    assert plan.still_valid(p)
    p[5, 0] += 0.19
    assert plan.still_valid(p)
    p[5, 0] += 0.02
    assert not plan.still_valid(p)


def test_non_periodic_split_axis():
    wl = W.make("fcc256")
    s = dataclasses.replace(wl.system, pbc=np.array([[1, 1, 0]], np.uint8))
    ref = O.batch(s, wl.desc, wl.archs, wl.theta)
    plan = Dm.SlabPlan(s, wl.desc.rc, 3)
    parts = [O.batch(d.system, wl.desc, wl.archs, wl.theta, ghost=d.ghost) for d in plan.domains]
    F = plan.gather_forces([p["F"] for p in parts])
    assert np.abs(F - ref["F"]).max() < 1e-12 * np.abs(ref["F"]).max()


# ------------------------------------------------------------------ real ranks (gloo)

def _rank_main(rank, world, port, errors):
    import torch
    import torch.distributed as dist
    try:
        os.environ["MASTER_ADDR"] = "127.0.0.1"
        os.environ["MASTER_PORT"] = str(port)
        dist.init_process_group("gloo", rank=rank, world_size=world)
        # --- slab decomposition of one periodic configuration
        wl = W.make("fcc256")
        sysg = _triclinic(wl.system)
        plan = Dm.SlabPlan(sysg, wl.desc.rc, world)
        d = plan.domains[rank]
        x_owned = torch.as_tensor(plan.pos_folded[d.owned])
        x_local = plan.halo(rank, x_owned)
        assert torch.equal(x_local, torch.as_tensor(d.system.pos)), "halo positions"
        part = O.batch(d.system, wl.desc, wl.archs, wl.theta, ghost=d.ghost)
        F_own = plan.reverse(rank, torch.as_tensor(part["F"])).numpy()
        ev = torch.tensor([part["E_cfg"][0]] + list(part["virial"][0].ravel()), dtype=torch.float64)
        dist.all_reduce(ev)
        ref = O.batch(sysg, wl.desc, wl.archs, wl.theta)
        assert np.abs(F_own - ref["F"][d.owned]).max() < 1e-12 * np.abs(ref["F"]).max(), "forces"
        assert abs(ev[0].item() - ref["E_cfg"][0]) < 1e-12 * np.abs(ref["E_atom"]).sum(), "energy"
        assert np.abs(ev[1:].numpy() - ref["virial"][0].ravel()).max() < 1e-11 * np.abs(ref["virial"]).max()
        # --- data-parallel training step, configurations sharded by cost
        wl = W.make("molecules16")
        s = wl.system
        b = Dm.shard_bounds(Dm.estimated_costs(s, wl.desc.rc), world)
        cfgs = list(range(b[rank], b[rank + 1]))
        a0, a1 = s.atom_off[b[rank]], s.atom_off[b[rank + 1]]
        C, N = Dm.global_counts(len(cfgs), int(a1 - a0))
        assert (C, N) == (s.n_cfg, s.n_atoms)
        out = O.batch(s.subset(cfgs), wl.desc, wl.archs, wl.theta, e_ref=wl.e_ref[cfgs], f_ref=wl.f_ref[a0:a1],
                      w_force=wl.w_force, param_grad=True, norm=(C, N))
        t = torch.as_tensor(np.concatenate([[out["loss"]], out["dtheta"]]))
        dist.all_reduce(t)
        full = O.batch(s, wl.desc, wl.archs, wl.theta, e_ref=wl.e_ref, f_ref=wl.f_ref, w_force=wl.w_force,
                       param_grad=True)
        assert abs(t[0].item() - full["loss"]) < 1e-12 * full["loss"], "loss"
        g = t[1:].numpy()
        assert np.abs(g - full["dtheta"]).max() < 1e-9 * np.abs(full["dtheta"]).max(), "gradient"
        dist.barrier()
        dist.destroy_process_group()
    except Exception as e:   # reported to the parent
        errors.put("rank %d: %r" % (rank, e))
        raise


def test_gloo_two_ranks_slabs_and_data_parallel_training():
    import torch.multiprocessing as mp
    ctx = mp.get_context("spawn")
    errors = ctx.SimpleQueue()
    port = _free_port()
    mp.start_processes(_rank_main, args=(2, port, errors), nprocs=2, join=True, start_method="spawn")
    assert errors.empty()


# ------------------------------------------------------------------ locally planned slabs

def _local_rank_main(rank, world, port, errors):
    import torch
    import torch.distributed as dist
    try:
        os.environ["MASTER_ADDR"] = "127.0.0.1"
        os.environ["MASTER_PORT"] = str(port)
        dist.init_process_group("gloo", rank=rank, world_size=world)
        wl = W.make("fcc256")
        sysg = _triclinic(wl.system)
        bounds = Dm.periodic_slab_bounds(world)
        # the initial distribution: this rank keeps only its own atoms
        own = Dm.owned_by_slab(sysg, bounds, rank)
        plan = Dm.LocalSlabPlan(rank, world, sysg.cell[0], sysg.pbc[0], wl.desc.rc, 0.3, sysg.pos[own],
                                sysg.species[own], own, bounds, sysg.n_species)
        # the same ghosts and local layout as the plan built from the global positions
        ref_plan = Dm.SlabPlan(sysg, wl.desc.rc, world, skin=0.3)
        d = ref_plan.domains[rank]
        np.testing.assert_array_equal(plan.gid, d.owned)
        np.testing.assert_array_equal(plan.recv_counts, d.recv_counts)
        got = np.stack([plan.ghost_src, plan.ghost_img], 1)
        want = np.stack([d.ghost_src, d.ghost_img], 1)
        np.testing.assert_array_equal(got, want)
        np.testing.assert_allclose(plan.system.pos, d.system.pos, rtol=0, atol=1e-12)
        # a displacement refreshed through the halo, then forces back to their owners
        x = torch.as_tensor(plan.pos_folded + 1e-3 * np.sin(np.arange(3 * plan.n_owned)).reshape(-1, 3))
        x_local = plan.halo(x)
        moved = dataclasses.replace(sysg, pos=sysg.pos.copy())
        moved.pos[own] = x.numpy()
        # every rank's moved atoms are needed for the whole-configuration reference
        allx = [torch.zeros(0)] * world
        dist.all_gather_object(allx, (own, x.numpy()))
        for o, xx in allx:
            moved.pos[o] = xx
        loc = dataclasses.replace(plan.system, pos=x_local.numpy())
        part = O.batch(loc, wl.desc, wl.archs, wl.theta, ghost=plan.ghost)
        F_own = plan.reverse(torch.as_tensor(part["F"])).numpy()
        ref = O.batch(moved, wl.desc, wl.archs, wl.theta)
        assert np.abs(F_own - ref["F"][own]).max() < 1e-12 * np.abs(ref["F"]).max(), "forces"
        e = torch.tensor([part["E_cfg"][0]], dtype=torch.float64)
        dist.all_reduce(e)
        assert abs(e.item() - ref["E_cfg"][0]) < 1e-12 * np.abs(ref["E_atom"]).sum(), "energy"
        assert plan.still_valid(x.numpy())
        dist.barrier()
        dist.destroy_process_group()
    except Exception as e:
        errors.put("rank %d: %r" % (rank, e))
        raise


@pytest.mark.parametrize("world", [2, 3])
def test_gloo_locally_planned_slabs(world):
    import torch.multiprocessing as mp
    ctx = mp.get_context("spawn")
    errors = ctx.SimpleQueue()
    port = _free_port()
    mp.start_processes(_local_rank_main, args=(world, port, errors), nprocs=world, join=True, start_method="spawn")
    assert errors.empty()
