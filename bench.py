"""Benchmark: one training step of the PANNA energy + force potential (arXiv 2305.11805).

Workload (default): 1024 isolated molecules of 5..29 atoms (H/C/N/O 0.5/0.3/0.1/0.1,
random bonded chains, no PBC, rc 5.2 A), 4-species descriptor of size 768 (32 radial
shells per species, 8 x 8 angular bins per species pair), per-species networks
768-128-32-1 with Gaussian activations.  One step = neighbour search, descriptors,
networks, energies, forces (adjoint), energy + 0.1 force MSE loss and its gradient with
respect to every network parameter (descriptor JVP + double backward), all in the CUDA
library, FP32 kernels and FP64 reductions.  Metric: atoms per second.

    python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]

--impl reference times the FP64 CPU oracle (single thread) on a bounded sample of the
same workload.  Under torchrun each rank runs its own batch of 1024 molecules (weak
scaling), normalises its loss by the global counts, and the gradients are summed over
ranks with one all-reduce per step: the gradient of the global batch (data parallel).
"""
from __future__ import annotations

import argparse
import json
import math
import os
import statistics
import subprocess
import sys
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

METRIC = "energy+force atoms/sec at stated force error vs FP64; % HBM/tensor roofline"
UNIT = "atoms/s"
WORKLOAD = "molecules1024"
PEAKS_FILE = os.path.join(ROOT, "MEASURED_PEAKS.json")
N_SM, FP32_LANES = 152, 128


def workload_desc(wl):
    return ("%d isolated molecules (5-29 atoms, H/C/N/O .5/.3/.1/.1, bonded chains, no PBC, rc %.1f A), "
            "%d atoms; descriptor D=%d (32 radial x 4 species + 8x8 angular x 10 species pairs); "
            "networks %s per species, Gaussian; training step: energy+force loss (w_F=%.1f) and "
            "weight gradient" % (wl.system.n_cfg, wl.desc.rc, wl.system.n_atoms, wl.desc.D,
                                 "-".join(str(w) for w in wl.archs[0].widths), wl.w_force))


def dist_env():
    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return rank, world, local


TRAFFIC_FILE = "profiles/geometry_kernels_molecules1024.md"


STORE_TRAFFIC_FILE = "profiles/store_kernels_molecules1024.md"


def measured_traffic(kernel, path=TRAFFIC_FILE):
    """DRAM bytes per launch of `kernel` from the committed ncu summary, or None when there is
    none or the kernel source has changed since the counters were taken."""
    import hashlib
    try:
        with open(os.path.join(ROOT, path)) as f:
            line = [l for l in f if l.startswith("traffic_bytes_per_launch")][0]
    except (OSError, IndexError):
        return None
    kv = dict(t.split("=", 1) for t in line.split()[1:])
    try:
        with open(os.path.join(ROOT, kv["source"]), "rb") as f:
            if hashlib.sha256(f.read()).hexdigest()[:16] != kv["sha256_16"]:
                return None
    except (OSError, KeyError):
        return None
    v = kv.get("k_" + kernel)
    return int(v) if v is not None else None


def load_peaks():
    try:
        with open(PEAKS_FILE) as f:
            return json.load(f), "measured"
    except Exception:
        return {"hbm_gbs": 6800.0, "bf16_tflops": 1900.0, "sm_max_mhz": 2070.0}, "fallback"


# ------------------------------------------------------------------ clocks

class ClockSampler:
    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, device_index: int):
        self.dev = device_index
        self.proc = None
        self.path = None

    def start(self):
        import tempfile
        fd, self.path = tempfile.mkstemp(suffix=".csv")
        os.close(fd)
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", str(self.dev), "--query-gpu=" + self.FIELDS, "--format=csv,noheader,nounits",
                 "-lms", "200"], stdout=open(self.path, "w"), stderr=subprocess.DEVNULL)
        except Exception:
            self.proc = None

    def stop(self):
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except Exception:
            self.proc.kill()
        rows = []
        for line in open(self.path):
            parts = [p.strip() for p in line.split(",")]
            if len(parts) >= 9:
                rows.append(parts)
        os.unlink(self.path)
        if not rows:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["no samples"]}
        sm = [float(r[1]) for r in rows if r[1].replace(".", "").isdigit()]
        mx = [float(r[2]) for r in rows if r[2].replace(".", "").isdigit()]
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        reasons = sorted({names[k] for r in rows for k in range(4) if r[5 + k].lower() == "active"})
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": max(mx) if mx else None,
                "reasons": reasons, "samples": len(rows)}


# ------------------------------------------------------------------ reference arm (oracle)

def run_reference(args):
    rank, world, _ = dist_env()
    if rank != 0:
        return 0
    import numpy as np
    from oracle import oracle as O
    from paper_2305_11805_gb300 import workloads as W
    wl = W.make(WORKLOAD, seed=args.seed)
    n_mol = args.ref_molecules
    sub = wl.system.subset(range(n_mol))
    er = wl.e_ref[:n_mol]
    fr = wl.f_ref[:sub.n_atoms]
    th = wl.theta.astype(np.float32).astype(np.float64)

    def step():
        O.batch(sub, wl.desc, wl.archs, th, e_ref=er, f_ref=fr, w_force=wl.w_force, param_grad=True)

    for _ in range(args.warmup):
        step()
    t0 = time.perf_counter()
    for _ in range(args.steps):
        step()
    dt = time.perf_counter() - t0
    v = sub.n_atoms * args.steps / dt
    sample = "first %d of the 1024 molecules (%d atoms), full training step, FP64 oracle, 1 thread" % (
        n_mol, sub.n_atoms)
    out = {"impl": "reference", "metric": METRIC, "value": v, "unit": UNIT, "n_gpus": world,
           "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * dt / args.steps,
           "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
           "data": "synthetic", "config": {"workload": workload_desc(wl), "sample": sample},
           "cpu_baseline": {"value": v, "unit": UNIT, "cores": 1, "kind": "oracle", "sample": sample},
           "e2e": {"value": v, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(out))
    return 0


def cpu_baseline(wl, seconds: float):
    """The oracle as it stands, single thread, on batches of 32 molecules until ~seconds."""
    import numpy as np
    from oracle import oracle as O
    th = wl.theta.astype(np.float32).astype(np.float64)
    atoms, t0, k = 0, time.perf_counter(), 0
    while True:
        cfgs = range(32 * k, 32 * (k + 1))
        sub = wl.system.subset(cfgs)
        O.batch(sub, wl.desc, wl.archs, th, e_ref=wl.e_ref[32 * k:32 * (k + 1)],
                f_ref=wl.f_ref[int(wl.system.atom_off[32 * k]):int(wl.system.atom_off[32 * (k + 1)])],
                w_force=wl.w_force, param_grad=True)
        atoms += sub.n_atoms
        k += 1
        dt = time.perf_counter() - t0
        if dt >= seconds or 32 * (k + 1) > wl.system.n_cfg:
            break
    return {"value": atoms / dt, "unit": UNIT, "cores": 1, "kind": "oracle",
            "sample": "training step on the first %d molecules (%d atoms) in batches of 32, %.1f s, "
                      "FP64, 1 thread" % (32 * k, atoms, dt)}


# ------------------------------------------------------------------ our arm

def run_ours(args):
    import numpy as np
    import torch
    rank, world, local = dist_env()
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl")
    torch.cuda.set_device(local)
    from paper_2305_11805_gb300 import build
    if rank == 0 and not os.path.exists(build.LIB):
        build.build()
    if world > 1:
        dist.barrier()
    from paper_2305_11805_gb300 import panna as P
    from paper_2305_11805_gb300 import workloads as W

    wl = W.make(WORKLOAD, seed=args.seed + rank)
    N, C = wl.system.n_atoms, wl.system.n_cfg
    dev = torch.device("cuda", local)
    pot = P.Potential(wl.desc, wl.archs)
    if world > 1:
        # every rank normalises its loss by the global counts: the summed gradients are
        # then exactly those of the global batch (world x 1024 molecules)
        from paper_2305_11805_gb300 import domain as Dm
        C_tot, N_tot = Dm.global_counts(C, N)
        P.panna_set_loss_normalization(pot.ctx, C_tot, N_tot)
    sysd = P.DeviceSystem(wl.system)
    theta = torch.as_tensor(wl.theta.astype(np.float32), device=dev)
    E_ref = torch.as_tensor(wl.e_ref, dtype=torch.float64, device=dev)
    F_ref = torch.as_tensor(wl.f_ref, dtype=torch.float32, device=dev)
    loss = torch.empty(1, dtype=torch.float64, device=dev)
    grad = torch.empty(pot.P, dtype=torch.float32, device=dev)
    stream = torch.cuda.current_stream()
    flush = torch.empty(256 * 1024 * 1024 // 4, dtype=torch.float32, device=dev)   # 256 MiB > L2

    def step():
        P.panna_loss_grad(pot.ctx, sysd, theta, E_ref, F_ref, wl.w_force, loss, grad)
        if world > 1:
            torch.distributed.all_reduce(grad)

    for _ in range(args.warmup):
        step()
    torch.cuda.synchronize()
    launches_per_step = P.panna_last_launch_count(pot.ctx)

    # ---- device-timed region: inputs resident in HBM, L2 flushed between steps
    P.panna_set_profiling(pot.ctx, True)
    stages = ["neighbors", "descriptor", "mlp", "adjoint", "forces", "loss", "jvp", "mlp_grad"]
    stage_ms = {s: 0.0 for s in stages}
    starts = [torch.cuda.Event(enable_timing=True) for _ in range(args.steps)]
    ends = [torch.cuda.Event(enable_timing=True) for _ in range(args.steps)]
    clocks = ClockSampler(local)
    if world > 1:
        torch.distributed.barrier()
    torch.cuda.synchronize()
    clocks.start()
    time.sleep(0.3)
    for k in range(args.steps):
        flush.fill_(float(k))
        starts[k].record(stream)
        step()
        ends[k].record(stream)
        for s in stages:
            v = P.panna_stage_ms(pot.ctx, s)
            if v > 0:
                stage_ms[s] += v
    torch.cuda.synchronize()
    clk = clocks.stop()
    P.panna_set_profiling(pot.ctx, False)
    t_ms = sum(s.elapsed_time(e) for s, e in zip(starts, ends))
    if world > 1:
        t = torch.tensor([t_ms], dtype=torch.float64, device=dev)
        torch.distributed.all_reduce(t, op=torch.distributed.ReduceOp.MAX)
        t_ms = float(t.item())
    ms_per_step = t_ms / args.steps
    value = world * N * args.steps / (t_ms * 1e-3)

    # ---- end to end through the public API with host buffers (pinned), copies inside
    h_off = torch.as_tensor(wl.system.atom_off, dtype=torch.int64).pin_memory()
    h_pos = torch.as_tensor(wl.system.pos, dtype=torch.float64).pin_memory()
    h_spec = torch.as_tensor(wl.system.species, dtype=torch.int32).pin_memory()
    h_cell = torch.as_tensor(wl.system.cell, dtype=torch.float64).pin_memory()
    h_pbc = torch.as_tensor(wl.system.pbc, dtype=torch.uint8).pin_memory()
    h_er = torch.as_tensor(wl.e_ref, dtype=torch.float64).pin_memory()
    h_fr = torch.as_tensor(wl.f_ref, dtype=torch.float32).pin_memory()
    h_loss = torch.empty(1, dtype=torch.float64).pin_memory()
    d_in = [torch.empty_like(t, device=dev) for t in (h_off, h_pos, h_spec, h_cell, h_pbc, h_er, h_fr)]
    h2d = sum(t.numel() * t.element_size() for t in (h_off, h_pos, h_spec, h_cell, h_pbc, h_er, h_fr))
    d2h = h_loss.numel() * h_loss.element_size()
    sys_e2e = P.DeviceSystem.from_tensors(d_in[0], d_in[1], d_in[2], d_in[3], d_in[4])

    def e2e_step():
        for h, d in zip((h_off, h_pos, h_spec, h_cell, h_pbc, h_er, h_fr), d_in):
            d.copy_(h, non_blocking=True)
        P.panna_loss_grad(pot.ctx, sys_e2e, theta, d_in[5], d_in[6], wl.w_force, loss, grad)
        if world > 1:
            torch.distributed.all_reduce(grad)
            torch.distributed.all_reduce(loss)
        h_loss.copy_(loss, non_blocking=True)
        torch.cuda.current_stream().synchronize()

    for _ in range(2):
        e2e_step()
    if world > 1:
        torch.distributed.barrier()
    t0 = time.perf_counter()
    for _ in range(args.steps):
        e2e_step()
    e2e_s = time.perf_counter() - t0
    if world > 1:
        t = torch.tensor([e2e_s], dtype=torch.float64, device=dev)
        torch.distributed.all_reduce(t, op=torch.distributed.ReduceOp.MAX)
        e2e_s = float(t.item())
    e2e_value = world * N * args.steps / e2e_s

    if rank != 0:
        if world > 1:
            torch.distributed.barrier()
        return 0

    # ---- roofline of the dominant kernel.  The descriptor, adjoint and JVP stages are one
    # kernel launch each (FP32 CUDA-core arithmetic, "alu"); algorithmic FLOPs per unit are
    # minimal operation counts (geometry, 8 zeta-powers by 7 multiplies, 8 Gaussians, the
    # 64-term outer product per pair of an 8 x 8 tile).  The network stages are several kernels
    # each and are listed per stage only.
    peaks, peak_kind = load_peaks()
    clock_mhz = peaks.get("sm_max_mhz", 2070.0)
    alu_peak = N_SM * FP32_LANES * 2 * clock_mhz * 1e6 / 1e12     # TFLOP/s FP32 FMA
    counts = [int((wl.system.species == s).sum()) for s in range(wl.desc.n_species)]
    mlp_fwd = sum(2 * counts[s] * sum(a.widths[l] * a.widths[l + 1] for l in range(a.n_layers))
                  for s, a in enumerate(wl.archs))
    off, _, _ = pot.neighbors(sysd)
    nb = torch.diff(off).double()
    n_entries = float(nb.sum().item())
    n_pairs = float((nb * (nb - 1) / 2).sum().item())
    d = wl.desc
    nbins = d.n_theta * d.n_ang_r
    per_pair = {"descriptor": 265.0 * nbins / 64, "adjoint": 495.0 * nbins / 64, "jvp": 450.0 * nbins / 64}
    per_entry = {"descriptor": 6.0 * d.n_rad, "adjoint": 8.0 * d.n_rad, "jvp": 8.0 * d.n_rad}
    stage_flops = {s: per_pair[s] * n_pairs + per_entry[s] * n_entries for s in per_pair}
    stage_flops["mlp"] = 2 * mlp_fwd          # forward + input gradient
    stage_flops["mlp_grad"] = 3 * mlp_fwd     # tangent forward + two weight-gradient passes
    per_step = {s: stage_ms[s] / args.steps for s in stages}
    kernels = [k for k in ("descriptor", "adjoint", "jvp") if per_step.get(k, 0) > 0]
    roof = None
    if kernels:
        dom = max(kernels, key=per_step.get)
        ach = stage_flops[dom] / (per_step[dom] * 1e-3) / 1e12
        traffic = measured_traffic(dom)
        roof = {"bound": "alu", "kernel": dom, "achieved": ach, "peak": alu_peak,
                "unit": "TFLOP/s", "frac": ach / alu_peak, "traffic": traffic,
                "peak_source": "derived: 152 SMs x 128 FP32 lanes x 2 flop x %.0f MHz (%s sm_max_mhz)" % (
                    clock_mhz, peak_kind),
                "ms_per_launch": per_step[dom],
                "traffic_source": TRAFFIC_FILE if traffic is not None else None,
                "all_stages_tflops": {s: round(stage_flops[s] / (per_step[s] * 1e-3) / 1e12, 2)
                                      for s in stage_flops if per_step.get(s, 0) > 0},
                "pairs_per_step": n_pairs, "neighbour_entries_per_step": n_entries}
    cpu = cpu_baseline(wl, args.cpu_seconds) if args.cpu_seconds > 0 else None
    out = {"metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
           "warmup": args.warmup, "ms_per_step": ms_per_step, "higher_is_better": True, "scaling": "weak",
           "vs_baseline": None, "dtype": "fp32", "data": "synthetic",
           "config": {"workload": workload_desc(wl), "atoms_per_gpu": N, "configs_per_gpu": C,
                      "parallelism": "dp%d" % world, "l2": "flushed between steps (256 MiB write)",
                      "stage_ms_per_step": {k: round(v, 4) for k, v in per_step.items()}},
           "roofline": roof, "cpu_baseline": cpu,
           "e2e": {"value": e2e_value, "unit": UNIT, "h2d_bytes_per_step": h2d, "d2h_bytes_per_step": d2h},
           "gpu_launches": launches_per_step * args.steps, "clocks": clk}
    print(json.dumps(out))
    if world > 1:
        torch.distributed.barrier()
    return 0


def run_ragged(args):
    """Ragged batch of 4096 periodic boxes (32..4096 atoms), BF16 networks: the whole batch as
    one captured CUDA graph versus the same configurations launched one call at a time."""
    import numpy as np
    import torch
    from paper_2305_11805_gb300 import build
    build.build()
    from paper_2305_11805_gb300 import panna as P
    from paper_2305_11805_gb300 import workloads as W
    torch.cuda.set_device(dist_env()[2])
    wl = W.make("ragged4096", seed=args.seed)
    s = wl.system
    N, C = s.n_atoms, s.n_cfg
    pot = P.Potential(wl.desc, wl.archs)
    sysd = P.DeviceSystem(s)
    theta = torch.as_tensor(wl.theta.astype(np.float32), device="cuda")
    prec = P.PANNA_MLP_BF16
    E = torch.empty(C, dtype=torch.float64, device="cuda")
    Ea = torch.empty(N, dtype=torch.float32, device="cuda")
    F = torch.empty((N, 3), dtype=torch.float32, device="cuda")
    V = torch.empty((C, 3, 3), dtype=torch.float64, device="cuda")
    P.panna_capture(pot.ctx, sysd, theta, prec, E, Ea, F, V)
    stream = torch.cuda.current_stream()
    for _ in range(args.warmup):
        P.panna_replay(pot.ctx, stream)
    P.panna_check(pot.ctx, stream)
    ev = [torch.cuda.Event(enable_timing=True) for _ in range(2)]
    clocks = ClockSampler(0)
    clocks.start()
    time.sleep(0.3)
    ev[0].record(stream)
    for _ in range(args.steps):
        P.panna_replay(pot.ctx, stream)
    ev[1].record(stream)
    torch.cuda.synchronize()
    clk = clocks.stop()
    P.panna_check(pot.ctx, stream)
    t_graph = ev[0].elapsed_time(ev[1]) / args.steps
    # the same configurations, one call each
    off = torch.zeros((C, 2), dtype=torch.int64, device="cuda")
    off[:, 1] = torch.as_tensor(np.diff(s.atom_off), device="cuda")
    pot1 = P.Potential(wl.desc, wl.archs)
    views = []
    for c in range(C):
        a0 = int(s.atom_off[c])
        views.append(P.DeviceSystem.from_tensors(off[c], sysd.pos[a0:int(s.atom_off[c + 1])],
                                                 sysd.species[a0:int(s.atom_off[c + 1])], sysd.cell[c:c + 1],
                                                 sysd.pbc[c:c + 1]))
    out1 = [torch.empty(1, dtype=torch.float64, device="cuda"), None]
    P.panna_set_tuning(pot1.ctx, "autotune", 0)   # no per-size measurement inside the loop
    big = int(np.argmax(np.diff(s.atom_off)))
    for v in [views[big]] + views[:16]:
        n = v.n_atoms
        P.panna_energy_forces(pot1.ctx, v, theta, prec, out1[0], None, F[:n], None)
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    for v in views:
        P.panna_energy_forces(pot1.ctx, v, theta, prec, out1[0], None, F[:v.n_atoms], None)
    torch.cuda.synchronize()
    t_one = time.perf_counter() - t0
    out = {"metric": METRIC, "value": N / (t_graph * 1e-3), "unit": UNIT, "n_gpus": 1, "steps": args.steps,
           "warmup": args.warmup, "ms_per_step": t_graph, "higher_is_better": True, "scaling": "weak",
           "vs_baseline": None, "dtype": "bf16 (hi+lo operands), fp32 descriptors", "data": "synthetic",
           "config": {"workload": "4096 periodic cubic boxes, N log-uniform 32..4096 (%d atoms), 3 species, "
                                  "0.05 atoms/A^3, rc 5.5, D=480, networks 480-128-32-1, energy+forces" % N,
                      "mode": "one captured CUDA graph per step (replay)",
                      "one_config_per_call_atoms_per_s": N / t_one,
                      "one_config_per_call_s": t_one,
                      "graph_kernels_per_replay": P.panna_last_launch_count(pot.ctx),
                      "l2": "working set (several GB) larger than L2"},
           "clocks": clk}
    print(json.dumps(out))
    return 0


def run_stored(args):
    """The same training step (molecules1024) from precomputed descriptors with stored
    Jacobians (Sec. II.A): neighbour search, descriptors and the angular adjoint / JVP
    arithmetic are done once when the store is built; each step streams the stored
    Jacobians twice (forces, and the tangent of the weight gradient).  The on-the-fly step
    is timed in the same process for the trade-off."""
    import numpy as np
    import torch
    from paper_2305_11805_gb300 import build
    build.build()
    from paper_2305_11805_gb300 import panna as P
    from paper_2305_11805_gb300 import workloads as W
    torch.cuda.set_device(dist_env()[2])
    wl = W.make(WORKLOAD, seed=args.seed)
    N, C = wl.system.n_atoms, wl.system.n_cfg
    pot = P.Potential(wl.desc, wl.archs)
    sysd = P.DeviceSystem(wl.system)
    theta = torch.as_tensor(wl.theta.astype(np.float32), device="cuda")
    E_ref = torch.as_tensor(wl.e_ref, dtype=torch.float64, device="cuda")
    F_ref = torch.as_tensor(wl.f_ref, dtype=torch.float32, device="cuda")
    loss = torch.empty(1, dtype=torch.float64, device="cuda")
    grad = torch.empty(pot.P, dtype=torch.float32, device="cuda")
    stream = torch.cuda.current_stream()
    flush = torch.empty(256 * 1024 * 1024 // 4, dtype=torch.float32, device="cuda")

    # one-time build, timed (plan + build; the second build is the one reported)
    st = P.Store(pot, sysd)
    ev = [torch.cuda.Event(enable_timing=True) for _ in range(2)]
    ev[0].record(stream)
    P.panna_store_build(pot.ctx, sysd, st.info, st.buf)
    ev[1].record(stream)
    torch.cuda.synchronize()
    build_ms = ev[0].elapsed_time(ev[1])

    def timed(fn, profile):
        for _ in range(args.warmup):
            fn()
        torch.cuda.synchronize()
        launches = P.panna_last_launch_count(pot.ctx)
        stages = ["mlp", "adjoint", "forces", "loss", "jvp", "mlp_grad", "neighbors", "descriptor"]
        sm = {k: 0.0 for k in stages}
        P.panna_set_profiling(pot.ctx, profile)
        starts = [torch.cuda.Event(enable_timing=True) for _ in range(args.steps)]
        ends = [torch.cuda.Event(enable_timing=True) for _ in range(args.steps)]
        torch.cuda.synchronize()
        for k in range(args.steps):
            flush.fill_(float(k))
            starts[k].record(stream)
            fn()
            ends[k].record(stream)
            if profile:
                for q in stages:
                    v = P.panna_stage_ms(pot.ctx, q)
                    if v > 0:
                        sm[q] += v
        torch.cuda.synchronize()
        P.panna_set_profiling(pot.ctx, False)
        t = sum(a.elapsed_time(b) for a, b in zip(starts, ends))
        return t / args.steps, {k: v / args.steps for k, v in sm.items() if v > 0}, launches

    clocks = ClockSampler(0)
    clocks.start()
    time.sleep(0.3)
    ms, stage, launches = timed(lambda: P.panna_store_loss_grad(pot.ctx, sysd, st.info, st.buf, theta, E_ref, F_ref,
                                                                wl.w_force, loss, grad), True)
    clk = clocks.stop()
    otf_ms, _, _ = timed(lambda: P.panna_loss_grad(pot.ctx, sysd, theta, E_ref, F_ref, wl.w_force, loss, grad),
                         False)
    value = N / (ms * 1e-3)

    # end to end: labels from pinned host memory each step, loss read back; the store is the
    # resident dataset
    h_er = torch.as_tensor(wl.e_ref, dtype=torch.float64).pin_memory()
    h_fr = torch.as_tensor(wl.f_ref, dtype=torch.float32).pin_memory()
    h_loss = torch.empty(1, dtype=torch.float64).pin_memory()

    def e2e_step():
        E_ref.copy_(h_er, non_blocking=True)
        F_ref.copy_(h_fr, non_blocking=True)
        P.panna_store_loss_grad(pot.ctx, sysd, st.info, st.buf, theta, E_ref, F_ref, wl.w_force, loss, grad)
        h_loss.copy_(loss, non_blocking=True)
        torch.cuda.current_stream().synchronize()

    for _ in range(2):
        e2e_step()
    t0 = time.perf_counter()
    for _ in range(args.steps):
        e2e_step()
    e2e_value = N * args.steps / (time.perf_counter() - t0)

    # roofline: the two store kernels stream the Jacobians (HBM bound); algorithmic bytes per
    # launch = Jacobian + entry records + the per-atom rows they read and write
    peaks, peak_kind = load_peaks()
    P_e, W_c, D = int(st.info.n_entries), int(st.info.width), wl.desc.D
    jac_bytes = P_e * 3 * W_c * 4
    bytes_ = {"adjoint": jac_bytes + P_e * 8 + N * D * 4 + N * 12 * 2 + P_e * 12,
              "jvp": jac_bytes + P_e * 8 + N * 12 + P_e * 12 + N * D * 4}
    dom = max(("adjoint", "jvp"), key=lambda k: stage.get(k, 0.0))
    ach = bytes_[dom] / (stage[dom] * 1e-3) / 1e9
    traffic = measured_traffic(dom, STORE_TRAFFIC_FILE)
    out = {"metric": METRIC, "value": value, "unit": UNIT, "n_gpus": 1, "steps": args.steps,
           "warmup": args.warmup, "ms_per_step": ms, "higher_is_better": True, "scaling": "weak",
           "vs_baseline": None, "dtype": "fp32", "data": "synthetic",
           "config": {"workload": "stored descriptors + Jacobians: " + workload_desc(wl), "atoms": N,
                      "configs": C, "store_bytes": st.nbytes, "neighbour_entries": P_e,
                      "jacobian_columns_per_entry": W_c, "store_build_ms": build_ms,
                      "on_the_fly_ms_per_step": otf_ms, "l2": "flushed between steps (256 MiB write)",
                      "stage_ms_per_step": {k: round(v, 4) for k, v in stage.items()}},
           "roofline": {"bound": "hbm", "kernel": dom, "achieved": ach, "peak": peaks["hbm_gbs"], "unit": "GB/s",
                        "frac": ach / peaks["hbm_gbs"], "traffic": traffic,
                        "traffic_source": STORE_TRAFFIC_FILE if traffic is not None else None,
                        "peak_source": "%s hbm_gbs" % peak_kind, "algorithmic_bytes_per_launch": bytes_[dom],
                        "ms_per_launch": stage[dom]},
           "e2e": {"value": e2e_value, "unit": UNIT, "h2d_bytes_per_step": h_er.numel() * 8 + h_fr.numel() * 4,
                   "d2h_bytes_per_step": 8},
           "gpu_launches": launches * args.steps, "clocks": clk}
    print(json.dumps(out))
    return 0


def run_qeq(args):
    """Charge equilibration (Sec. II.B) on 4096 charged NaCl clusters (Na9Cl8+ and Na8Cl8+
    alternating, the shapes of Sec. III.C): neighbour search, size-45 descriptors, 45-15-15-3
    networks, one FP64 constrained linear solve per cluster, pair forces, network input
    gradients and the descriptor adjoint, per call."""
    import numpy as np
    import torch
    from paper_2305_11805_gb300 import build
    build.build()
    from paper_2305_11805_gb300 import panna as P
    from paper_2305_11805_gb300 import workloads as W
    torch.cuda.set_device(dist_env()[2])
    wl = W.make("nacl4096", seed=args.seed)
    N, C = wl.system.n_atoms, wl.system.n_cfg
    pot = P.Potential(wl.desc, wl.archs)
    P.panna_set_qeq(pot.ctx, wl.qeq["sigma"], wl.qeq["chi0"], wl.qeq["hard0"])
    sysd = P.DeviceSystem(wl.system)
    theta = torch.as_tensor(wl.theta.astype(np.float32), device="cuda")
    Q = torch.as_tensor(wl.charge, dtype=torch.float64, device="cuda")
    E = torch.empty(C, dtype=torch.float64, device="cuda")
    q = torch.empty(N, dtype=torch.float64, device="cuda")
    F = torch.empty((N, 3), dtype=torch.float32, device="cuda")
    stream = torch.cuda.current_stream()
    flush = torch.empty(256 * 1024 * 1024 // 4, dtype=torch.float32, device="cuda")

    def step():
        P.panna_qeq_energy_forces(pot.ctx, sysd, theta, Q, E, None, q, F)

    for _ in range(args.warmup):
        step()
    torch.cuda.synchronize()
    launches = P.panna_last_launch_count(pot.ctx)
    stages = ["neighbors", "descriptor", "mlp", "forces", "adjoint", "loss"]
    sm = {k: 0.0 for k in stages}
    P.panna_set_profiling(pot.ctx, True)
    starts = [torch.cuda.Event(enable_timing=True) for _ in range(args.steps)]
    ends = [torch.cuda.Event(enable_timing=True) for _ in range(args.steps)]
    clocks = ClockSampler(0)
    clocks.start()
    time.sleep(0.3)
    for k in range(args.steps):
        flush.fill_(float(k))
        starts[k].record(stream)
        step()
        ends[k].record(stream)
        for st in stages:
            v = P.panna_stage_ms(pot.ctx, st)
            if v > 0:
                sm[st] += v
    torch.cuda.synchronize()
    clk = clocks.stop()
    P.panna_set_profiling(pot.ctx, False)
    ms = sum(a.elapsed_time(b) for a, b in zip(starts, ends)) / args.steps
    stage = {k: round(v / args.steps, 4) for k, v in sm.items() if v > 0}

    # training step through the charge layer (energy + force loss and its gradient), timed the
    # same way and reported beside the evaluation
    rng = np.random.default_rng(args.seed)
    e_ref = torch.as_tensor(rng.normal(0, 1, C), dtype=torch.float64, device="cuda") + E
    f_ref = F + torch.as_tensor(rng.normal(0, 0.2, (N, 3)), dtype=torch.float32, device="cuda")
    loss = torch.empty(1, dtype=torch.float64, device="cuda")
    grad = torch.empty(pot.P, dtype=torch.float32, device="cuda")

    def train_step():
        P.panna_qeq_loss_grad(pot.ctx, sysd, theta, Q, e_ref, f_ref, 0.1, None, 0.0, loss, grad)

    for _ in range(args.warmup):
        train_step()
    torch.cuda.synchronize()
    t0e, t1e = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    t0e.record(stream)
    for k in range(args.steps):
        train_step()
    t1e.record(stream)
    torch.cuda.synchronize()
    train_ms = t0e.elapsed_time(t1e) / args.steps

    # end to end: positions, species, offsets and total charges from pinned host memory,
    # energies and charges read back
    hs = [torch.as_tensor(a).pin_memory() for a in (wl.system.atom_off, wl.system.pos, wl.system.species,
                                                     wl.system.cell, wl.system.pbc, wl.charge)]
    ds = [torch.empty_like(t, device="cuda") for t in hs]
    sys_e2e = P.DeviceSystem.from_tensors(ds[0], ds[1], ds[2], ds[3], ds[4])
    hE = torch.empty(C, dtype=torch.float64).pin_memory()
    hq = torch.empty(N, dtype=torch.float64).pin_memory()

    def e2e_step():
        for h, d in zip(hs, ds):
            d.copy_(h, non_blocking=True)
        P.panna_qeq_energy_forces(pot.ctx, sys_e2e, theta, ds[5], E, None, q, F)
        hE.copy_(E, non_blocking=True)
        hq.copy_(q, non_blocking=True)
        torch.cuda.current_stream().synchronize()

    for _ in range(2):
        e2e_step()
    t0 = time.perf_counter()
    for _ in range(args.steps):
        e2e_step()
    e2e = N * args.steps / (time.perf_counter() - t0)
    out = {"metric": "charge-equilibrated energy+force atoms/sec (NaCl clusters)", "value": N / (ms * 1e-3),
           "unit": UNIT, "n_gpus": 1, "steps": args.steps, "warmup": args.warmup, "ms_per_step": ms,
           "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "fp32 networks, fp64 solve",
           "data": "synthetic",
           "config": {"workload": "4096 NaCl clusters (Na9Cl8+ / Na8Cl8+ alternating, +1 e each), %d atoms; "
                                  "descriptor D=%d, networks 45-15-15-3, Gaussian charges (sigma Na 1.0, Cl 1.2 A)"
                                  % (N, wl.desc.D), "l2": "flushed between steps (256 MiB write)",
                      "stage_ms_per_step": stage, "training_step_ms": train_ms,
                      "training_atoms_per_s": N / (train_ms * 1e-3)},
           "e2e": {"value": e2e, "unit": UNIT,
                   "h2d_bytes_per_step": sum(t.numel() * t.element_size() for t in hs),
                   "d2h_bytes_per_step": hE.numel() * 8 + hq.numel() * 8},
           "gpu_launches": launches * args.steps, "clocks": clk}
    print(json.dumps(out))
    return 0


def run_md(args):
    """Langevin dynamics (BAOAB, 300 K, dt 0.5 fs, friction 0.01 / fs, skin 0.5 A) of the
    16-atom carbon cell the paper times (Sec. III.B, Table II: 0.78 ms per step per atom,
    one A100 through ASE, context only), and of 4096 independent copies of it in one batch."""
    import numpy as np
    import torch
    from paper_2305_11805_gb300 import build
    build.build()
    from paper_2305_11805_gb300 import panna as P
    from paper_2305_11805_gb300 import workloads as W
    torch.cuda.set_device(dist_env()[2])
    mass, T, dt, gam, skin = [12.011], 300.0, 0.5, 0.01, 0.5
    out = {"metric": "Langevin MD time per step per atom", "unit": "ms", "higher_is_better": False,
           "n_gpus": 1, "dtype": "fp32", "data": "synthetic",
           "paper_context": {"value": 0.78, "unit": "ms per step per atom",
                             "hardware": "1x A100, TensorFlow through ASE, PANNA small, 16-atom carbon cell"}}
    clocks = ClockSampler(0)
    clocks.start()
    time.sleep(0.3)
    for name, n_steps in (("carbon16", 1000), ("carbon16x4096", 200)):
        wl = W.make(name, seed=args.seed)
        pot = P.Potential(wl.desc, wl.archs)
        sysd = P.DeviceSystem(wl.system)
        theta = torch.as_tensor(wl.theta.astype(np.float32), device="cuda")
        rng = np.random.default_rng(args.seed)
        v = rng.normal(0.0, np.sqrt(8.617333262e-5 * T * 9.648533212e-3 / mass[0]), size=(wl.system.n_atoms, 3))
        vel = torch.as_tensor(v, dtype=torch.float64, device="cuda")
        F = torch.zeros((wl.system.n_atoms, 3), dtype=torch.float32, device="cuda")
        E = torch.zeros(wl.system.n_cfg, dtype=torch.float64, device="cuda")
        P.panna_md_run(pot.ctx, sysd, vel, theta, P.PANNA_MLP_FP32, dt, T, gam, skin, mass, 1, 0, 20, F, False, E)
        ev = [torch.cuda.Event(enable_timing=True) for _ in range(2)]
        torch.cuda.synchronize()
        ev[0].record()
        builds = P.panna_md_run(pot.ctx, sysd, vel, theta, P.PANNA_MLP_FP32, dt, T, gam, skin, mass, 1, 20,
                                n_steps, F, True, E)
        ev[1].record()
        torch.cuda.synchronize()
        ms = ev[0].elapsed_time(ev[1]) / n_steps
        N = wl.system.n_atoms
        out[name] = {"atoms": N, "steps": n_steps, "ms_per_step": ms, "ms_per_step_per_atom": ms / N,
                     "atom_steps_per_s": N / (ms * 1e-3), "neighbour_searches": builds}
    out["clocks"] = clocks.stop()
    out["value"] = out["carbon16"]["ms_per_step_per_atom"]
    out["config"] = {"workload": "carbon16: diamond carbon 2x1x1 cells (16 atoms), D=152 (24 radial + 8 R x 16 "
                                 "theta), network 152-64-32-1; BAOAB 300 K, dt 0.5 fs, friction 0.01/fs, "
                                 "skin 0.5 A; carbon16x4096: 4096 independent copies in one batch"}
    print(json.dumps(out))
    return 0


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=20)
    ap.add_argument("--warmup", type=int, default=5)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--seed", type=int, default=0)
    ap.add_argument("--cpu-seconds", type=float, default=12.0)
    ap.add_argument("--ref-molecules", type=int, default=24)
    ap.add_argument("--workload", default=WORKLOAD, choices=[WORKLOAD, "ragged4096", "md", "stored", "qeq"])
    args = ap.parse_args()
    if args.workload != WORKLOAD and args.impl == "ours":
        # the secondary workloads are single-GPU measurements: under torchrun rank 0 runs on
        # its own device and prints the line, the other ranks exit without work
        rank, world, local = dist_env()
        if rank != 0:
            return 0
        import torch
        torch.cuda.set_device(local)
    if args.workload == "ragged4096" and args.impl == "ours":
        return run_ragged(args)
    if args.workload == "md" and args.impl == "ours":
        return run_md(args)
    if args.workload == "stored" and args.impl == "ours":
        return run_stored(args)
    if args.workload == "qeq" and args.impl == "ours":
        return run_qeq(args)
    if args.impl == "reference":
        return run_reference(args)
    return run_ours(args)


if __name__ == "__main__":
    sys.exit(main())
