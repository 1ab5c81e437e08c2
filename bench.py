"""Benchmark of the PANNA energy + force potential (arXiv 2305.11805) on one GB300 per rank.

Default workload ragged4096: energies and forces of a ragged batch of 4096 periodic cubic
boxes of 32..4096 atoms (log-uniform; 3.37 M atoms; 3 species in Dirichlet(1,1,1) proportions;
0.05 atoms/A^3; rc 5.5 A), descriptor D = 480 (32 radial shells per species, 8 x 8 angular
bins per species pair), per-species networks 480-128-32-1 (Gaussian), BF16 networks with FP32
accumulation, FP32 descriptors and adjoint, FP64 energy sums.  One step = neighbour search,
descriptors, networks, energies, forces, run as one captured CUDA graph.  Metric: atoms/s,
stated with the measured force error against the FP64 oracle.

    python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]
                    [--workload ragged4096|fcc1m|water32k|diamond64|molecules1024|stored|qeq|md]

Other workloads: fcc1m (1,048,576-atom FCC box, 64 radial + 16 x 8 angular, 192-128-64-1, BF16),
water32k (32,768-atom O/H box, rc 6, 256-256-128-1, BF16), diamond64 (64-atom diamond cell,
96-256-128-32-1, FP32), molecules1024 (the training step: loss and its parameter gradient over
1024 molecules, FP32), stored / qeq / md (precomputed descriptors, charge equilibration,
Langevin dynamics).

Every line carries the roofline of the dominant kernel, the FP64 oracle timed on the host's
cores as `cpu_baseline` (one core and all cores), `e2e` through the C ABI with host buffers,
and, for the inference workloads, the force error against the oracle on a stated sample.
--impl reference times the oracle itself (all host cores) on a bounded sample of the workload.
Under torchrun every rank evaluates its own batch (seed + rank; weak scaling); the inference
workloads need no collective, the training step sums its gradient with one all-reduce.
"""
from __future__ import annotations

import argparse
import json
import math
import os
import platform
import statistics
import subprocess
import sys
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

METRIC = "energy+force atoms/sec at stated force error vs FP64; % HBM/tensor roofline"
UNIT = "atoms/s"
INFER = ("ragged4096", "fcc1m", "water32k", "diamond64")
TRAIN = "molecules1024"
DEFAULT_WORKLOAD = "ragged4096"
PEAKS_FILE = os.path.join(ROOT, "MEASURED_PEAKS.json")
N_SM, FP32_LANES = 152, 128
TOL_F = {"fp32": 1e-5, "bf16": 1e-2}   # max |dF| / RMS(F) against the FP64 oracle


def workload_desc(wl):
    return ("%d isolated molecules (5-29 atoms, H/C/N/O .5/.3/.1/.1, bonded chains, no PBC, rc %.1f A), "
            "%d atoms; descriptor D=%d (32 radial x 4 species + 8x8 angular x 10 species pairs); "
            "networks %s per species, Gaussian; training step: energy+force loss (w_F=%.1f) and "
            "weight gradient" % (wl.system.n_cfg, wl.desc.rc, wl.system.n_atoms, wl.desc.D,
                                 "-".join(str(w) for w in wl.archs[0].widths), wl.w_force))


INFER_DESC = {
    "ragged4096": "4096 periodic cubic boxes, N log-uniform 32..4096 (%d atoms), 3 species (Dirichlet(1,1,1) "
                  "proportions), 0.05 atoms/A^3, rc 5.5 A, D=480 (32 radial + 8x8 angular), networks "
                  "480-128-32-1 per species; energies + forces",
    "fcc1m": "periodic FCC box 64^3 cells (%d atoms), a=4.05 A, sigma 0.05 A, rc 5.0 A, D=192 (64 radial + "
             "16 theta x 8 R), network 192-128-64-1; energies + forces",
    "water32k": "periodic O/H box (%d atoms, O:H 1:2, 0.1003 atoms/A^3, min sep 0.9 A), rc 6.0 A, D=256, "
                "networks 256-256-128-1 per species; energies + forces",
    "diamond64": "periodic diamond cell 2x2x2 (%d atoms), a=5.43 A, sigma 0.1 A, rc 4.6 A, D=96, network "
                 "96-256-128-32-1; energies + forces",
}


def dist_env():
    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return rank, world, local


TRAFFIC_FILE = "profiles/geometry_kernels_molecules1024.md"
STORE_TRAFFIC_FILE = "profiles/store_kernels_molecules1024.md"
RAGGED_TRAFFIC_FILE = "profiles/angular_kernels_ragged256.md"


def measured_traffic(kernel, path=TRAFFIC_FILE, atoms=None):
    """DRAM bytes per launch of `kernel` from a committed ncu summary, or None when there is
    none or the kernel source has changed since the counters were taken.  With `atoms`, the
    summary's figure (captured on a smaller batch of the same recipe, `atoms=` in its line) is
    scaled to that many atoms: the angular kernels read each atom's neighbour slots and its
    descriptor or gradient row once, so their traffic grows with the atoms processed."""
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
    if v is None:
        return None
    if atoms is not None:
        if "atoms" not in kv:
            return None
        return int(round(int(v) * atoms / int(kv["atoms"])))
    return int(v)


def load_peaks():
    try:
        with open(PEAKS_FILE) as f:
            return json.load(f), "measured"
    except Exception:
        return {"hbm_gbs": 6800.0, "bf16_tflops": 1900.0, "sm_max_mhz": 2070.0}, "fallback"


def host_info():
    """Host cores available to this process and the CPU model (for the oracle baselines)."""
    try:
        cores = len(os.sched_getaffinity(0))
    except AttributeError:
        cores = os.cpu_count() or 1
    model = None
    try:
        out = subprocess.run(["lscpu"], capture_output=True, text=True, timeout=10).stdout
        for line in out.splitlines():
            if line.lower().startswith("model name"):
                model = line.split(":", 1)[1].strip()
                break
    except Exception:
        pass
    return cores, "%s (%s)" % (model or platform.processor() or "unknown", platform.machine())


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


# ------------------------------------------------------------------ the oracle on the host cores
#
# The oracle runs as it stands (FP64, one thread per call).  "All cores" runs independent
# calls side by side in a process pool started with `spawn` (no process is forked after the
# GPU is in use); the pool is warmed up first so that interpreter start-up is not timed.

def _orc_batch_job(job):
    """One oracle call in a worker: (system, desc, archs, theta) -> (atoms, seconds, E_cfg, F)."""
    from oracle import oracle as O
    system, desc, archs, theta = job
    t0 = time.perf_counter()
    r = O.batch(system, desc, archs, theta)
    return system.n_atoms, time.perf_counter() - t0, r["E_cfg"], r["F"]


def _orc_sampled_job(job):
    from oracle import oracle as O
    system, cfg, desc, archs, theta, samples = job
    r = O.sampled(system, cfg, desc, archs, theta, samples)
    return samples, r["F"], r["E"]


def _orc_ping(_):
    from oracle import oracle as O
    O.lib()
    return os.getpid()


class OraclePool:
    def __init__(self, workers: int):
        import concurrent.futures as cf
        import multiprocessing as mp
        self.workers = workers
        self.ex = cf.ProcessPoolExecutor(max_workers=workers, mp_context=mp.get_context("spawn"))
        list(self.ex.map(_orc_ping, range(4 * workers)))

    def map(self, fn, jobs):
        return list(self.ex.map(fn, jobs))

    def close(self):
        self.ex.shutdown(wait=True)


def oracle_samples(name, wl, seed):
    """The bounded samples the oracle runs on, per workload: (one-core jobs, all-core jobs,
    description).  Each job is one oracle call (system, desc, archs, theta)."""
    import numpy as np
    from paper_2305_11805_gb300 import workloads as W
    th = wl.theta.astype(np.float32).astype(np.float64)
    if name == "ragged4096":
        jobs = [(wl.system.subset([c]), wl.desc, wl.archs, th) for c in range(64)]
        return jobs, jobs, "configurations 0..63 of the batch (%d atoms)" % sum(j[0].n_atoms for j in jobs)
    if name in ("fcc1m", "water32k", "diamond64"):
        mk = {"fcc1m": lambda s: W.fcc(s, 8), "water32k": lambda s: W.water(s, 512),
              "diamond64": lambda s: W.diamond64(s)}[name]
        subs = [mk(seed + 1000 + k) for k in range(64)]
        jobs = [(b.system, wl.desc, wl.archs, th) for b in subs]
        what = {"fcc1m": "periodic FCC boxes of 8^3 cells (2048 atoms) with the fcc1m recipe, descriptor and "
                         "network, other seeds",
                "water32k": "periodic 512-atom boxes with the water32k recipe, descriptor and network, other seeds",
                "diamond64": "64-atom diamond cells (other seeds)"}[name]
        return jobs, jobs, what
    raise ValueError(name)


def cpu_baseline(name, wl, seed, seconds, pool):
    """The oracle timed on one core (calls in turn until `seconds` have passed) and on all cores
    (as many calls as workers x rounds, side by side).  Returns the baseline record and the
    oracle results of the all-core run (for the force error of the GPU result)."""
    one, many, what = oracle_samples(name, wl, seed)
    cores, model = host_info()
    atoms1, t1, k = 0, 0.0, 0
    while k < len(one) and (t1 < seconds or k == 0):
        n, dt, _, _ = _orc_batch_job(one[k])
        atoms1 += n
        t1 += dt
        k += 1
    v1 = atoms1 / t1
    res, v_all, n_all, t_all = None, None, 0, None
    if pool is not None:
        # about `seconds` of wall time on all workers, whole rounds of calls
        per_call = t1 / k
        n_calls = max(pool.workers, min(len(many), int(pool.workers * seconds / max(per_call, 1e-3))))
        n_calls = min(len(many), n_calls)
        t0 = time.perf_counter()
        res = pool.map(_orc_batch_job, many[:n_calls])
        t_all = time.perf_counter() - t0
        n_all = sum(r[0] for r in res)
        v_all = n_all / t_all
    rec = {"value": v_all if v_all else v1, "unit": UNIT, "cores": pool.workers if pool else 1, "kind": "oracle",
           "sample": "%s; energies + forces, FP64" % what,
           "one_core": {"value": v1, "calls": k, "atoms": atoms1, "seconds": round(t1, 2)},
           "all_cores": None if pool is None else {"value": v_all, "cores": pool.workers, "calls": len(res),
                                                   "atoms": n_all, "seconds": round(t_all, 2)},
           "nproc": cores, "cpu_model": model}
    return rec, (many[:len(res)] if res else []), res


def force_error(F, Fo):
    """max |F - Fo| / RMS(Fo) (the tolerance of the FP32 and BF16 paths)."""
    import numpy as np
    rms = float(np.sqrt((Fo ** 2).mean()))
    return float(np.abs(F - Fo).max() / rms) if rms > 0 else float(np.abs(F - Fo).max())


def force_error_sample(name, wl, F_gpu, E_gpu, pool, base_res, base_jobs, seed):
    """Force (and energy) error of the GPU result against the oracle on a stated sample of the
    same batch: whole configurations of the ragged batch (the ones the all-core baseline ran),
    sampled atoms of the big boxes (the oracle evaluates each one by brute force)."""
    import numpy as np
    s = wl.system
    th = wl.theta.astype(np.float32).astype(np.float64)
    if name == "ragged4096":
        n_cfg = len(base_res)
        a1 = int(s.atom_off[n_cfg])
        Fo = np.concatenate([r[3] for r in base_res])
        Eo = np.concatenate([r[2] for r in base_res])
        ferr = force_error(F_gpu[:a1], Fo)
        eerr = float(np.max(np.abs(E_gpu[:n_cfg] - Eo) / np.maximum(np.abs(Eo), 1e-30)))
        return {"max_abs_over_rms": ferr, "energy_rel": eerr, "sample": "configurations 0..%d (%d atoms), "
                "whole-configuration FP64 oracle" % (n_cfg - 1, a1)}
    if name == "diamond64":
        _, _, Eo, Fo = _orc_batch_job((s, wl.desc, wl.archs, th))
        return {"max_abs_over_rms": force_error(F_gpu, Fo),
                "energy_rel": float(abs(E_gpu[0] - Eo[0]) / abs(Eo[0])),
                "sample": "the whole 64-atom cell of the timed run, FP64 oracle"}
    rng = np.random.default_rng(seed + 17)
    n_smp = 32
    smp = sorted(rng.choice(s.n_atoms, n_smp, replace=False).tolist())
    per = max(1, n_smp // (pool.workers if pool else 1))
    jobs = [(s, 0, wl.desc, wl.archs, th, smp[k:k + per]) for k in range(0, n_smp, per)]
    out = pool.map(_orc_sampled_job, jobs) if pool else [_orc_sampled_job(j) for j in jobs]
    idx = np.concatenate([np.asarray(o[0]) for o in out])
    Fo = np.concatenate([o[1] for o in out])
    rms = float(np.sqrt((F_gpu.astype(np.float64) ** 2).mean()))
    ferr = float(np.abs(F_gpu[idx] - Fo).max() / rms)
    return {"max_abs_over_rms": ferr, "sample": "%d random atoms of the box, each evaluated by the FP64 oracle "
            "(brute force over its environment); RMS over all atoms of the GPU result" % n_smp}


def run_infer(args):
    """Energies and forces of one inference workload, the whole pass as one captured CUDA graph."""
    import numpy as np
    import torch
    rank, world, local = dist_env()
    name = args.workload
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl")
    torch.cuda.set_device(local)
    from paper_2305_11805_gb300 import build
    if rank == 0:
        build.build()
    if world > 1:
        torch.distributed.barrier()
    from paper_2305_11805_gb300 import panna as P
    from paper_2305_11805_gb300 import workloads as W
    # the oracle pool first (spawned workers; no fork after the GPU is in use)
    pool = None
    if rank == 0 and args.cpu_seconds > 0:
        from oracle import oracle as O
        O.build()
        pool = OraclePool(max(1, min(host_info()[0], 64)))

    if name == "ragged4096" and args.n_cfg:
        wl = W.ragged(args.seed + rank, args.n_cfg)   # the first n_cfg boxes of the same recipe
    else:
        wl = W.make(name, seed=args.seed + rank)
    s = wl.system
    N, C = s.n_atoms, s.n_cfg
    dev = torch.device("cuda", local)
    bf16 = bool(wl.mlp_bf16)
    prec = P.PANNA_MLP_BF16 if bf16 else P.PANNA_MLP_FP32
    pot = P.Potential(wl.desc, wl.archs)
    sysd = P.DeviceSystem(wl.system)
    theta = torch.as_tensor(wl.theta.astype(np.float32), device=dev)
    E = torch.empty(C, dtype=torch.float64, device=dev)
    F = torch.empty((N, 3), dtype=torch.float32, device=dev)
    stream = torch.cuda.current_stream()
    small = N * wl.desc.D * 4 < 512 * 1024 * 1024     # descriptor rows alone below 4 x L2: flush
    flush = torch.empty(256 * 1024 * 1024 // 4, dtype=torch.float32, device=dev) if small else None

    fp32_tflops, fp32x2_tflops, ex2_gops = P.panna_measure_alu_peaks2()

    # stage times of the same call (direct calls with stage events; the graph has none)
    P.panna_energy_forces(pot.ctx, sysd, theta, prec, E, None, F, None)
    P.panna_set_profiling(pot.ctx, True)
    stages = ["neighbors", "descriptor", "mlp", "adjoint", "forces"]
    stage_ms = {k: 0.0 for k in stages}
    n_prof = 3
    for _ in range(n_prof):
        if flush is not None:
            flush.fill_(1.0)
        P.panna_energy_forces(pot.ctx, sysd, theta, prec, E, None, F, None)
        for k in stages:
            v = P.panna_stage_ms(pot.ctx, k)
            if v > 0:
                stage_ms[k] += v / n_prof
    P.panna_set_profiling(pot.ctx, False)

    # ---- device-timed region: the captured graph, inputs resident in HBM
    P.panna_capture(pot.ctx, sysd, theta, prec, E, None, F, None)
    launches = P.panna_last_launch_count(pot.ctx)
    for _ in range(args.warmup):
        P.panna_replay(pot.ctx, stream)
    P.panna_check(pot.ctx, stream)
    starts = [torch.cuda.Event(enable_timing=True) for _ in range(args.steps)]
    ends = [torch.cuda.Event(enable_timing=True) for _ in range(args.steps)]
    clocks = ClockSampler(local)
    if world > 1:
        torch.distributed.barrier()
    torch.cuda.synchronize()
    clocks.start()
    time.sleep(0.3)
    for k in range(args.steps):
        if flush is not None:
            flush.fill_(float(k))
        starts[k].record(stream)
        P.panna_replay(pot.ctx, stream)
        ends[k].record(stream)
    torch.cuda.synchronize()
    clk = clocks.stop()
    P.panna_check(pot.ctx, stream)
    t_ms = sum(a.elapsed_time(b) for a, b in zip(starts, ends))
    if world > 1:
        t = torch.tensor([t_ms], dtype=torch.float64, device=dev)
        torch.distributed.all_reduce(t, op=torch.distributed.ReduceOp.MAX)
        t_ms = float(t.item())
    ms_per_step = t_ms / args.steps
    value = world * N * args.steps / (t_ms * 1e-3)
    F_host = F.cpu().numpy().astype(np.float64)
    E_host = E.cpu().numpy()

    # ---- end to end through the C ABI with host buffers: inputs copied from pinned host memory
    # into the arrays the graph reads, the graph replayed, energies and forces read back
    hs = [torch.as_tensor(np.ascontiguousarray(a)).pin_memory()
          for a in (s.atom_off, s.pos, s.species.astype(np.int32), s.cell, s.pbc.astype(np.uint8))]
    ds = [sysd.atom_off, sysd.pos, sysd.species, sysd.cell, sysd.pbc]
    hE = torch.empty(C, dtype=torch.float64).pin_memory()
    hF = torch.empty((N, 3), dtype=torch.float32).pin_memory()
    h2d = sum(t.numel() * t.element_size() for t in hs)
    d2h = hE.numel() * 8 + hF.numel() * 4

    def e2e_step():
        for h, d in zip(hs, ds):
            d.copy_(h, non_blocking=True)
        P.panna_replay(pot.ctx, stream)
        hE.copy_(E, non_blocking=True)
        hF.copy_(F, non_blocking=True)
        stream.synchronize()

    for _ in range(2):
        e2e_step()
    if world > 1:
        torch.distributed.barrier()
    t0 = time.perf_counter()
    for _ in range(args.steps):
        e2e_step()
    e2e_s = time.perf_counter() - t0
    P.panna_check(pot.ctx, stream)
    if world > 1:
        t = torch.tensor([e2e_s], dtype=torch.float64, device=dev)
        torch.distributed.all_reduce(t, op=torch.distributed.ReduceOp.MAX)
        e2e_s = float(t.item())
    e2e_value = world * N * args.steps / e2e_s

    # ---- the plain FP32 path on one configuration per call (ragged batch): the comparison the
    # batched BF16 graph is measured against, each with its force error
    comparison = None
    if name == "ragged4096" and rank == 0 and args.compare:
        comparison = compare_single(args, P, wl, pot, sysd, theta, dev)

    if rank != 0:
        if world > 1:
            torch.distributed.barrier()
        return 0

    # ---- roofline of the dominant kernel: the descriptor and adjoint stages are one kernel
    # launch each, bound by the FP32 pipe (hundreds of operations per byte); algorithmic FLOPs
    # per unit are minimal operation counts (geometry, the zeta powers by repeated
    # multiplication, the Gaussians, the outer product per pair of an 8 x 8 tile)
    peaks, peak_kind = load_peaks()
    off, _, _ = pot.neighbors(sysd)
    nb = torch.diff(off).double()
    n_entries = float(nb.sum().item())
    n_pairs = float((nb * (nb - 1) / 2).sum().item())
    d = wl.desc
    nbins = d.n_theta * d.n_ang_r
    per_pair = {"descriptor": 265.0 * nbins / 64, "adjoint": 495.0 * nbins / 64}
    per_entry = {"descriptor": 6.0 * d.n_rad, "adjoint": 8.0 * d.n_rad}
    stage_flops = {k: per_pair[k] * n_pairs + per_entry[k] * n_entries for k in per_pair}
    counts = [int((s.species == q).sum()) for q in range(d.n_species)]
    mlp_fwd = sum(2 * counts[q] * sum(a.widths[l] * a.widths[l + 1] for l in range(a.n_layers))
                  for q, a in enumerate(wl.archs))
    stage_flops["mlp"] = 2 * mlp_fwd      # forward + input gradient (algorithmic, one product each)
    dom = max(("descriptor", "adjoint"), key=lambda k: stage_ms.get(k, 0.0))
    ach = stage_flops[dom] / (stage_ms[dom] * 1e-3) / 1e12
    traffic = measured_traffic(dom, RAGGED_TRAFFIC_FILE, atoms=N) if name == "ragged4096" else None
    roof = {"bound": "alu", "kernel": dom, "achieved": ach, "peak": fp32_tflops, "unit": "TFLOP/s",
            "frac": ach / fp32_tflops, "traffic": traffic,
            "traffic_source": (RAGGED_TRAFFIC_FILE + " (scaled by atoms)") if traffic is not None else None,
            "peak_source": "measured in this run: FP32 FMA microbenchmark (panna_measure_alu_peaks) on all SMs",
            "derived_peak": N_SM * FP32_LANES * 2 * peaks.get("sm_max_mhz", 2070.0) * 1e6 / 1e12,
            "fp32x2_packed_peak": fp32x2_tflops, "ex2_peak_gops": ex2_gops, "ms_per_launch": stage_ms[dom],
            "kernel_variant": {k: P.panna_tuning_choice(pot.ctx, k) for k in ("descriptor", "adjoint")},
            "flop_per_angular_pair": per_pair[dom], "angular_pairs": n_pairs, "neighbour_entries": n_entries,
            "stage_tflops": {k: round(stage_flops[k] / (stage_ms[k] * 1e-3) / 1e12, 3)
                             for k in stage_flops if stage_ms.get(k, 0) > 0},
            "mlp_tensor_frac_of_bf16_peak": (stage_flops["mlp"] / (stage_ms["mlp"] * 1e-3) / 1e12 /
                                             peaks["bf16_tflops"]) if stage_ms.get("mlp", 0) > 0 else None}

    cpu, base_jobs, base_res = (None, [], [])
    ferr = None
    if args.cpu_seconds > 0:
        cpu, base_jobs, base_res = cpu_baseline(name, wl, args.seed, args.cpu_seconds, pool)
        ferr = force_error_sample(name, wl, F_host, E_host, pool, base_res, base_jobs, args.seed)
        ferr["precision"] = "bf16" if bf16 else "fp32"
        ferr["bar"] = TOL_F["bf16" if bf16 else "fp32"]
        if comparison is not None:
            comparison["batched_bf16_graph"]["force_error"] = ferr["max_abs_over_rms"]
            comparison["fp32_one_config_per_call"]["force_error"] = force_error(
                comparison.pop("_F32")[:int(s.atom_off[len(base_res)])],
                np.concatenate([r[3] for r in base_res]))
        pool.close()
    elif comparison is not None:
        comparison.pop("_F32", None)
    dtype = ("bf16 networks (hi+lo operands, FP32 accumulation); fp32 descriptors and adjoint; fp64 sums"
             if bf16 else "fp32 (extended-precision angular terms); fp64 sums")
    out = {"metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
           "warmup": args.warmup, "ms_per_step": ms_per_step, "higher_is_better": True, "scaling": "weak",
           "vs_baseline": None, "dtype": dtype, "data": "synthetic",
           "config": {"workload": name + ": " + (INFER_DESC[name] % N), "atoms_per_gpu": N, "configs_per_gpu": C,
                      "parallelism": "independent batches per rank (dp%d)" % world,
                      "mode": "one captured CUDA graph per step (panna_capture / panna_replay)",
                      "l2": "flushed between steps (256 MiB write)" if small else
                            "working set (GBs) far larger than L2, no flush",
                      "stage_ms_per_step": {k: round(v, 4) for k, v in stage_ms.items()}},
           "force_error": ferr, "roofline": roof, "cpu_baseline": cpu,
           "e2e": {"value": e2e_value, "unit": UNIT, "h2d_bytes_per_step": h2d, "d2h_bytes_per_step": d2h},
           "gpu_launches": launches * args.steps, "clocks": clk}
    if comparison is not None:
        comparison["batched_bf16_graph"]["atoms_per_s"] = value
        comparison["batched_bf16_graph"]["precision"] = "bf16 networks (hi+lo), fp32 descriptors"
        comparison["speedup_batched_bf16_over_fp32_one_config_per_call"] = (
            value / comparison["fp32_one_config_per_call"]["atoms_per_s"])
        out["comparison"] = comparison
    print(json.dumps(out))
    if world > 1:
        torch.distributed.barrier()
    return 0


def compare_single(args, P, wl, pot, sysd, theta, dev):
    """The same batch through the plain FP32 path, one configuration per call (synchronous
    panna_energy_forces per configuration), and the FP32 networks as one batched graph."""
    import numpy as np
    import torch
    s = wl.system
    N, C = s.n_atoms, s.n_cfg
    stream = torch.cuda.current_stream()
    off = torch.zeros((C, 2), dtype=torch.int64, device=dev)
    off[:, 1] = torch.as_tensor(np.diff(s.atom_off), device=dev)
    views = []
    for c in range(C):
        a0, a1 = int(s.atom_off[c]), int(s.atom_off[c + 1])
        views.append(P.DeviceSystem.from_tensors(off[c], sysd.pos[a0:a1], sysd.species[a0:a1], sysd.cell[c:c + 1],
                                                 sysd.pbc[c:c + 1]))
    pot1 = P.Potential(wl.desc, wl.archs)
    P.panna_set_tuning(pot1.ctx, "autotune", 0)   # no per-size measurement inside the loop
    E1 = torch.empty(1, dtype=torch.float64, device=dev)
    F32 = torch.empty((N, 3), dtype=torch.float32, device=dev)
    big = int(np.argmax(np.diff(s.atom_off)))
    for v in [views[big]] + views[:16]:
        P.panna_energy_forces(pot1.ctx, v, theta, P.PANNA_MLP_FP32, E1, None, F32[:v.n_atoms], None)
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    for c, v in enumerate(views):
        a0 = int(s.atom_off[c])
        P.panna_energy_forces(pot1.ctx, v, theta, P.PANNA_MLP_FP32, E1, None, F32[a0:a0 + v.n_atoms], None)
    torch.cuda.synchronize()
    t_one = time.perf_counter() - t0
    pot1.close()
    # FP32 networks, whole batch in one graph (separates batching from precision)
    potb = P.Potential(wl.desc, wl.archs)
    Eb = torch.empty(C, dtype=torch.float64, device=dev)
    Fb = torch.empty((N, 3), dtype=torch.float32, device=dev)
    P.panna_capture(potb.ctx, sysd, theta, P.PANNA_MLP_FP32, Eb, None, Fb, None)
    for _ in range(2):
        P.panna_replay(potb.ctx, stream)
    ev = [torch.cuda.Event(enable_timing=True) for _ in range(2)]
    ev[0].record(stream)
    for _ in range(3):
        P.panna_replay(potb.ctx, stream)
    ev[1].record(stream)
    torch.cuda.synchronize()
    P.panna_check(potb.ctx, stream)
    t_b32 = ev[0].elapsed_time(ev[1]) / 3
    potb.close()
    return {"fp32_one_config_per_call": {"atoms_per_s": N / t_one, "seconds": t_one,
                                         "calls": C, "precision": "fp32 networks, extended angular terms"},
            "fp32_batched_graph": {"atoms_per_s": N / (t_b32 * 1e-3), "ms": t_b32},
            "batched_bf16_graph": {"atoms_per_s": None},
            "_F32": F32.cpu().numpy().astype(np.float64)}


# ------------------------------------------------------------------ reference arm (the oracle)

def run_reference(args):
    rank, world, _ = dist_env()
    if rank != 0:
        return 0
    import numpy as np
    from oracle import oracle as O
    from paper_2305_11805_gb300 import workloads as W
    O.build()
    name = args.workload
    cores, model = host_info()
    if name == TRAIN:
        wl = W.make(TRAIN, seed=args.seed)
        n_mol = args.ref_molecules
        th = wl.theta.astype(np.float32).astype(np.float64)
        sub = wl.system.subset(range(n_mol))

        def step():
            O.batch(sub, wl.desc, wl.archs, th, e_ref=wl.e_ref[:n_mol], f_ref=wl.f_ref[:sub.n_atoms],
                    w_force=wl.w_force, param_grad=True)
        atoms = sub.n_atoms
        used = 1
        sample = "first %d of the 1024 molecules (%d atoms), full training step, FP64 oracle, 1 thread" % (
            n_mol, atoms)
        cfg = workload_desc(wl)
        dtype = "f64"
    elif name in INFER:
        wl = W.make(name, seed=args.seed)
        one, many, what = oracle_samples(name, wl, args.seed)
        pool = OraclePool(max(1, min(cores, 64)))
        used = pool.workers
        n_calls = {"ragged4096": 32, "fcc1m": used, "water32k": used, "diamond64": 4 * used}[name]
        jobs = many[:n_calls]
        atoms = sum(j[0].n_atoms for j in jobs)

        def step():
            pool.map(_orc_batch_job, jobs)
        sample = "%d oracle calls side by side on %d host cores: %s; %d atoms per step" % (
            len(jobs), used, what if name != "ragged4096" else "configurations 0..%d of the batch" % (n_calls - 1),
            atoms)
        cfg = name + ": " + (INFER_DESC[name] % wl.system.n_atoms)
        dtype = "f64"
    else:
        print(json.dumps({"impl": "reference", "unavailable": "no oracle arm for workload %s" % name}))
        return 0
    for _ in range(args.warmup):
        step()
    t0 = time.perf_counter()
    for _ in range(args.steps):
        step()
    dt = time.perf_counter() - t0
    if name in INFER:
        pool.close()
    v = atoms * args.steps / dt
    out = {"impl": "reference", "metric": METRIC, "value": v, "unit": UNIT, "n_gpus": world,
           "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * dt / args.steps,
           "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": dtype,
           "data": "synthetic", "config": {"workload": cfg, "sample": sample},
           "cpu_baseline": {"value": v, "unit": UNIT, "cores": used, "kind": "oracle", "sample": sample,
                            "nproc": cores, "cpu_model": model},
           "e2e": {"value": v, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(out))
    return 0



def _orc_train_job(job):
    """One training-step oracle call in a worker: (system, desc, archs, theta, e_ref, f_ref, w_force)."""
    from oracle import oracle as O
    system, desc, archs, theta, er, fr, wf = job
    t0 = time.perf_counter()
    O.batch(system, desc, archs, theta, e_ref=er, f_ref=fr, w_force=wf, param_grad=True)
    return system.n_atoms, time.perf_counter() - t0


def cpu_baseline_train(wl, seconds, pool):
    """The oracle's training step (loss and parameter gradient) on batches of 32 molecules: one
    core (batches in turn until `seconds` have passed) and all cores (batches side by side)."""
    import numpy as np
    th = wl.theta.astype(np.float32).astype(np.float64)
    s = wl.system
    jobs = []
    for k in range(s.n_cfg // 32):
        a0, a1 = int(s.atom_off[32 * k]), int(s.atom_off[32 * (k + 1)])
        jobs.append((s.subset(range(32 * k, 32 * (k + 1))), wl.desc, wl.archs, th, wl.e_ref[32 * k:32 * (k + 1)],
                     wl.f_ref[a0:a1], wl.w_force))
    cores, model = host_info()
    atoms1, t1, k = 0, 0.0, 0
    while k < len(jobs) and (t1 < seconds or k == 0):
        n, dt = _orc_train_job(jobs[k])
        atoms1 += n
        t1 += dt
        k += 1
    rec = {"value": atoms1 / t1, "unit": UNIT, "cores": 1, "kind": "oracle",
           "sample": "training step (loss + parameter gradient) on batches of 32 molecules, FP64",
           "one_core": {"value": atoms1 / t1, "calls": k, "atoms": atoms1, "seconds": round(t1, 2)},
           "all_cores": None, "nproc": cores, "cpu_model": model}
    if pool is not None:
        n_calls = min(len(jobs), max(pool.workers, int(pool.workers * seconds / max(t1 / k, 1e-3))))
        t0 = time.perf_counter()
        res = pool.map(_orc_train_job, jobs[:n_calls])
        ta = time.perf_counter() - t0
        na = sum(r[0] for r in res)
        rec["all_cores"] = {"value": na / ta, "cores": pool.workers, "calls": n_calls, "atoms": na,
                            "seconds": round(ta, 2)}
        rec["value"] = na / ta
        rec["cores"] = pool.workers
    return rec

# ------------------------------------------------------------------ our arm

def run_training(args):
    import numpy as np
    import torch
    rank, world, local = dist_env()
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl")
    pool = None
    if rank == 0 and args.cpu_seconds > 0:
        from oracle import oracle as O
        O.build()
        pool = OraclePool(max(1, min(host_info()[0], 64)))
    torch.cuda.set_device(local)
    from paper_2305_11805_gb300 import build
    if rank == 0:
        build.build()
    if world > 1:
        dist.barrier()
    from paper_2305_11805_gb300 import panna as P
    from paper_2305_11805_gb300 import workloads as W

    wl = W.make(TRAIN, seed=args.seed + rank)
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

    fp32_tflops, ex2_gops = P.panna_measure_alu_peaks()

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
        roof = {"bound": "alu", "kernel": dom, "achieved": ach, "peak": fp32_tflops,
                "unit": "TFLOP/s", "frac": ach / fp32_tflops, "traffic": traffic,
                "peak_source": "measured in this run: FP32 FMA microbenchmark (panna_measure_alu_peaks) on all SMs",
                "derived_peak": alu_peak, "ex2_peak_gops": ex2_gops,
                "ms_per_launch": per_step[dom],
                "traffic_source": TRAFFIC_FILE if traffic is not None else None,
                "all_stages_tflops": {s: round(stage_flops[s] / (per_step[s] * 1e-3) / 1e12, 2)
                                      for s in stage_flops if per_step.get(s, 0) > 0},
                "pairs_per_step": n_pairs, "neighbour_entries_per_step": n_entries}
    cpu = cpu_baseline_train(wl, args.cpu_seconds, pool) if args.cpu_seconds > 0 else None
    if pool is not None:
        pool.close()
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
    wl = W.make(TRAIN, seed=args.seed)
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
    ap.add_argument("--cpu-seconds", type=float, default=10.0)
    ap.add_argument("--ref-molecules", type=int, default=24)
    ap.add_argument("--no-compare", dest="compare", action="store_false",
                    help="skip the FP32 one-configuration-per-call comparison (ragged4096)")
    ap.add_argument("--workload", default=DEFAULT_WORKLOAD, choices=list(INFER) + [TRAIN, "md", "stored", "qeq"])
    ap.add_argument("--n-cfg", type=int, default=0,
                    help="ragged4096 only: the first N boxes of the batch (small cases for profiling)")
    args = ap.parse_args()
    if args.impl == "reference":
        return run_reference(args)
    if args.workload in INFER:
        return run_infer(args)
    if args.workload == TRAIN:
        return run_training(args)
    # the remaining workloads are single-GPU measurements: under torchrun rank 0 runs on its
    # own device and prints the line, the other ranks exit without work
    rank, world, local = dist_env()
    if rank != 0:
        return 0
    import torch
    torch.cuda.set_device(local)
    return {"md": run_md, "stored": run_stored, "qeq": run_qeq}[args.workload](args)


if __name__ == "__main__":
    sys.exit(main())
