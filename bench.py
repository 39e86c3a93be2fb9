"""Benchmark: Laplace DOF/s and RK4 steps/s of the σ-transformed SEM wave model on GB300.

Workload (one "step"): one classical RK4 step of every tank of the uneven batch — 512
independent periodic tanks from seed 0 (Nx ∈ [16,128], Nz ∈ {1,2,4}, P ∈ {4..8},
kh ∈ [0.5,3], H/L ∈ [0.01,0.09], 3.18 M Laplace unknowns) — each RK4 step being four
σ-geometry updates, four Dirichlet-lifted Laplace solves, four gradient recoveries, four
over-integrated Zakharov right-hand sides, the RK4 combination and the modal filter per tank,
run as one fused launch per RK stage and (order, precision, cluster size) group, the groups on
concurrent streams, all in the library's CUDA kernels; every solve to the C3 configuration's
relative residual of 1e-10 (the strict tolerances are reported beside it).

value   = Laplace DOF/s of the batched plain FP64 path = 4 · Σ unknowns · steps / device time;
          the batched mixed-precision path (FP32 inner, FP64 refinement), the same tanks one
          after another on the plain FP64 single-mesh path, and each path's relative L² error
          against the CPU oracle on a seeded sample of tanks are reported beside it;
e2e     = the same metric through sem_batch_rk4_step_host (packed pinned host buffers, the
          host↔device copies of every tank's (η, φ̃) inside the timed region);
roofline: the fused stage kernel of the batch, FP64-ALU bound (FP64 Krylov work counted);
cpu_baseline: the CPU oracle on a bounded sample of the same tanks, on all host cores.
Extras: the C2 steep wave, the C4 shoal and the C5 request stream (mixed vs FP64, each with
its error against the oracle), and the operator apply on a long tank (HBM roofline).

`--impl reference` times the CPU oracle itself (the reference arm).  Under torchrun each rank
runs an independent replica of the batch (weak scaling, no data-path collective); rank 0
prints the JSON line.
"""
from __future__ import annotations

import argparse
import hashlib
import json
import math
import os
import statistics
import subprocess
import sys
import tempfile
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "Laplace DOF/s (tank RK4 steps/s alongside), batched FP64; mixed precision beside it"
UNIT = "DOF/s"
C3_NAME = ("C3 512 uneven periodic tanks (seed 0): Nx 16-128, Nz 1/2/4, P 4-8, kh 0.5-3, H/L 0.01-0.09; "
           "one RK4 step of every tank per step")
# Algorithmic FP64 work (per-unit figures stated in the design notes):
#   operator apply: 8(P+1)+7 flops per element-local node (gradients, fluxes, transposed sums)
#   Krylov vector updates and dots: 13 flops per unknown and iteration
# The σ-separable preconditioner runs in FP32 in both precisions and is not counted.
FP64_PEAK_TFLOPS = 1.25   # nominal GB300 FP64 rate (vector and tensor alike)


def flops_per_apply(wl) -> float:
    P = wl.P
    return wl.Nx * wl.Nz * (P + 1) ** 2 * (8 * (P + 1) + 7)


def fp64_solver_flops(wl, solves: int, iterations: int, refinements: int, mixed: bool) -> float:
    """FP64 algorithmic flops of `solves` Laplace solves: one apply per solve for the initial
    residual 𝓛[x; φ̃] (the lifted right-hand side enters only through its norm, taken with an FP32
    apply), one per Krylov iteration with its vector work (plain FP64), or one per refinement
    (mixed: its inner iterations run in FP32)."""
    if mixed:
        return (solves + refinements) * flops_per_apply(wl)
    return (solves + iterations) * flops_per_apply(wl) + iterations * 13 * wl.n_unknowns


def max_over_ranks(value: float, device=None) -> float:
    """Max of a per-rank scalar over all ranks (identity without torch.distributed)."""
    import torch
    import torch.distributed as dist
    if not (dist.is_available() and dist.is_initialized()) or dist.get_world_size() == 1:
        return float(value)
    t = torch.tensor([float(value)], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def job_throughput(world: int, steps: int, units_per_step: float, t_max_ms: float) -> float:
    """Whole-job units/s: every rank runs `steps` steps of its own replica; the job takes the
    slowest rank's time (weak scaling, no data-path collective)."""
    return world * steps * units_per_step / (t_max_ms / 1e3)


def dist_env():
    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return rank, world, local


class ClockSampler:
    """nvidia-smi sampling of SM clocks and throttle reasons during the timed region."""

    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index: int):
        self.gpu = gpu_index
        self.proc = None
        # the samples are read back by this process only; SEM_CLOCKS_DIR keeps them elsewhere
        self.path = os.path.join(os.environ.get("SEM_CLOCKS_DIR", tempfile.gettempdir()),
                                 f"sem_clocks_rank{gpu_index}_{os.getpid()}.csv")

    def start(self):
        try:
            os.makedirs(os.path.dirname(self.path), exist_ok=True)
            self.f = open(self.path, "w")
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", str(self.gpu), f"--query-gpu={self.FIELDS}", "--format=csv,noheader",
                 "-lms", "200"], stdout=self.f, stderr=subprocess.DEVNULL)
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
        self.f.close()
        sm, smax, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for line in open(self.path):
            parts = [p.strip() for p in line.split(",")]
            if len(parts) < 9:
                continue
            try:
                sm.append(float(parts[1].split()[0]))
                smax.append(float(parts[2].split()[0]))
            except ValueError:
                continue
            for nm, v in zip(names, parts[5:9]):
                if v.lower().startswith("active"):
                    reasons.add(nm)
        if not sm:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["no samples"]}
        return {"sm_mhz": statistics.median(sm), "sm_max_mhz": max(smax), "reasons": sorted(reasons),
                "samples": len(sm)}


STAGE_SOURCES = ("laplace_device.cuh", "surface_device.cuh", "sem_internal.cuh", "mesh_index.cuh")


def kernel_source_hash() -> str:
    """Hash of the device sources the fused stage kernel is compiled from."""
    h = hashlib.sha256()
    for f in STAGE_SOURCES:
        h.update(open(os.path.join(ROOT, "paper_1512_02548_gb300", "csrc", f), "rb").read())
    return h.hexdigest()[:16]


def profiled_traffic(kernel: str):
    """Per-launch DRAM bytes of `kernel` from the committed ncu summary, if still current."""
    path = os.path.join(ROOT, "profiles", "traffic.json")
    try:
        data = json.load(open(path))
    except Exception:
        return None
    ent = data.get(kernel)
    if not ent or ent.get("source_sha256_16") != kernel_source_hash():
        return None
    return ent.get("dram_bytes_per_launch")


# ---------------------------------------------------------------------------------------------
# CPU oracle timing (reference arm and cpu_baseline)
# ---------------------------------------------------------------------------------------------
def _oracle_init():
    """Worker initialiser of the oracle pool (spawned processes, one BLAS thread each)."""
    for k in ("OMP_NUM_THREADS", "OPENBLAS_NUM_THREADS", "MKL_NUM_THREADS", "BLIS_NUM_THREADS"):
        os.environ[k] = "1"


def oracle_job(job):
    """One oracle run in a worker: job = (kind, key, eta0, phis0, nsteps, t0) with kind "c3" (key =
    tank index), "c2" (key = H/L, 0 for the configured 0.08), "c4" or "c5" (key = (rate, count,
    request index)); nsteps = 0 means one Laplace solve (returns Φ), nsteps < 0 the displaced volume
    1ᵀM'η and energy ½Φᵀ(−𝓛)Φ + ½gηᵀM'η of the state.  Returns (key, results, seconds, Laplace
    unknowns solved)."""
    import numpy as np
    from oracle import sem as osem
    from sem_workloads import c2_steep_periodic, c3_instances, c4_shoal, c5_requests, depth_columns
    kind, key, eta, phis, nsteps, t = job
    if kind == "c3":
        wl = c3_instances(512)[key]
    elif kind == "c2":
        wl = c2_steep_periodic()
        if key:                                   # another wave steepness H/L
            import dataclasses
            wl = dataclasses.replace(wl, wave_height=key * wl.length)
    elif kind == "c4":
        wl = c4_shoal()
    else:
        wl = c5_requests(key[0], key[1], 0)[key[2]][2]
    h = depth_columns(wl, column_positions(wl)) if wl.bathymetry == "shoal" else np.full(wl.ncol, wl.depth)
    om = osem.mesh_for(wl, h_col=h)
    t0 = time.perf_counter()
    if nsteps < 0:                                # diagnostics of a state: displaced volume, energy
        out = (om.mass(eta), om.energy(eta, phis))
        dof = wl.n_unknowns
    elif nsteps == 0:
        out = (om.laplace_solve(eta, phis),)
        dof = wl.n_unknowns
    else:
        for _ in range(nsteps):
            eta, phis = om.rk4_step(eta, phis, wl.dt, t)
            t += wl.dt
        out = (eta, phis)
        dof = 4 * nsteps * wl.n_unknowns
    return key, out, time.perf_counter() - t0, dof


def oracle_pool(n: int):
    """A pool of `n` spawned oracle processes (safe after CUDA is initialised in this one)."""
    import multiprocessing as mp
    names = ("CUDA_VISIBLE_DEVICES", "OMP_NUM_THREADS", "OPENBLAS_NUM_THREADS", "MKL_NUM_THREADS", "BLIS_NUM_THREADS")
    env_keep = {k: os.environ.get(k) for k in names}
    for k in names:
        os.environ[k] = "" if k == "CUDA_VISIBLE_DEVICES" else "1"
    try:
        pool = mp.get_context("spawn").Pool(n, initializer=_oracle_init)
    finally:
        for k, v in env_keep.items():
            if v is None:
                os.environ.pop(k, None)
            else:
                os.environ[k] = v
    return pool


def c3_sample(count: int, seed: int = 7):
    """A seeded sample of C3 tank indices (splitmix64 keys, sorted order of the keys)."""
    from sem_workloads import splitmix64
    gen = splitmix64(seed)
    keys = [next(gen) for _ in range(512)]
    return sorted(range(512), key=lambda i: keys[i])[:count]


def c3_unknowns() -> int:
    """Laplace unknowns of the 512-tank C3 batch (one solve of every tank)."""
    from sem_workloads import c3_instances
    return int(sum(wl.n_unknowns for wl in c3_instances(512)))


def c3_initial(i: int):
    import numpy as np
    from sem_workloads import c3_instances, initial_state
    wl = c3_instances(512)[i]
    return initial_state(wl, column_positions(wl), np.full(wl.ncol, wl.depth))


def host_cores() -> int:
    try:
        return len(os.sched_getaffinity(0))
    except Exception:
        return os.cpu_count() or 1


def run_reference(args):
    """Reference arm: the CPU oracle on the headline workload.  One step = one RK4 step of
    `cores` C3 tanks (a seeded rotation through the 512), one tank per host core, each
    single-threaded; value = Laplace unknowns solved (4 per tank and step) / wall time."""
    rank, world, _ = dist_env()
    if rank != 0:
        return 0
    cores = host_cores()
    order = c3_sample(512)
    pool = oracle_pool(cores)
    try:
        def one(k):
            idx = [order[(k * cores + j) % 512] for j in range(cores)]
            jobs = [("c3", i, *c3_initial(i), 1, 0.0) for i in idx]
            t0 = time.perf_counter()
            res = pool.map(oracle_job, jobs, chunksize=1)
            return time.perf_counter() - t0, sum(r[3] for r in res)
        for k in range(args.warmup):
            one(k)
        wall, dof = 0.0, 0
        for k in range(args.warmup, args.warmup + args.steps):
            w, d = one(k)
            wall += w
            dof += d
    finally:
        pool.close()
        pool.join()
    value = dof / wall
    line = {
        "impl": "reference", "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": args.gpus,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * wall / args.steps,
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
        "data": "synthetic",
        "config": {"workload": C3_NAME, "instances": 512, "n_unknowns": c3_unknowns(), "precision": "fp64",
                   "tol": "direct banded-Cholesky solves (the oracle)",
                   "step": f"one RK4 step of {cores} of the tanks (seeded rotation) on the CPU oracle",
                   "parallelism": "single" if args.gpus == 1 else "replicas"},
        "cpu_baseline": {"value": value, "unit": UNIT, "cores": cores, "kind": "oracle",
                         "sample": f"{args.steps} steps of {cores} C3 tanks each, one RK4 step (four "
                                   f"banded-Cholesky Laplace solves) per tank, one process per core, "
                                   f"nproc = {os.cpu_count()}"},
        "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line))
    return 0


# ---------------------------------------------------------------------------------------------
# Supplementary: the operator apply on a long tank (working set above L2)
# ---------------------------------------------------------------------------------------------
def apply_roofline(dev, reps: int = 20, Nx: int = 65536,
                   kernels=("fp64_column", "fp64_tile", "fp32_tile", "fp32_tile_tc")):
    """The operator apply y = 𝓛x on a 65536×4, P=6 periodic tank (9.8 M nodes), four kernels:
    the FP64 tiled kernel (sem_laplace_apply), the FP64 element-column kernel (same call with
    SEM_APPLY_KERNEL=column), the FP32 tiled kernel (sem_laplace_apply_f32) and the tensor-core
    FP32 tiled kernel (same call with SEM_APPLY_F32=tc).

    Algorithmic work per apply: (8(P+1)+7) flops per element-local node; algorithmic bytes:
    read x + write y, 16 B (FP64) or 8 B (FP32) per node.  Design bytes add the per-column
    geometry (4 values per element-local column).  Each apply is timed alone with CUDA events,
    with L2 flushed (256 MB written) before it; the median of `reps` is reported.
    """
    import numpy as np
    import torch
    import paper_1512_02548_gb300 as sem
    from sem_workloads import roofline_tank
    wl = roofline_tank(Nx=Nx)
    mesh = sem.Mesh.from_workload(wl)
    xcol = column_positions(wl)
    eta = torch.tensor(0.05 * np.cos(2 * np.pi * xcol / wl.length * (Nx // 1024)), device=dev)
    mesh.update_geometry(eta)
    x = torch.randn(mesh.n, dtype=torch.float64, device=dev)
    y = torch.empty_like(x)
    x32 = x.float()
    y32 = torch.empty_like(x32)
    flush = torch.empty(256 * 1024 * 1024 // 4, dtype=torch.float32, device=dev)
    stream = torch.cuda.current_stream()

    def timed(fn):
        for _ in range(3):
            fn()
        ts = []
        for _ in range(reps):
            flush.zero_()
            e0 = torch.cuda.Event(enable_timing=True)
            e1 = torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            fn()
            e1.record(stream)
            e1.synchronize()
            ts.append(e0.elapsed_time(e1))
        return float(np.median(ts))

    def with_env(key, value, fn):
        old = os.environ.get(key)
        os.environ[key] = value
        try:
            fn()
        finally:
            if old is None:
                del os.environ[key]
            else:
                os.environ[key] = old

    def column64():
        with_env("SEM_APPLY_KERNEL", "column", lambda: mesh.laplace_apply(x, y))

    y32t = torch.empty_like(x32)

    def tc32():
        with_env("SEM_APPLY_F32", "tc", lambda: mesh.laplace_apply_f32(x32, y32t))

    P = wl.P
    flops = wl.Nx * wl.Nz * (P + 1) ** 2 * (8 * (P + 1) + 7)
    geo_cols = wl.Nx * (P + 1)
    peaks = measured_peaks()
    hbm = peaks.get("hbm_gbs")
    out = {"workload": wl.name, "n_nodes": mesh.n, "flops_per_apply": flops, "l2_flushed": True}
    for name, fn, elem in (("fp64_column", column64, 8), ("fp64_tile", lambda: mesh.laplace_apply(x, y), 8),
                           ("fp32_tile", lambda: mesh.laplace_apply_f32(x32, y32), 4),
                           ("fp32_tile_tc", tc32, 4)):
        if name not in kernels:
            continue
        ms = timed(fn)
        alg = 2 * elem * mesh.n
        design = alg + 4 * elem * geo_cols
        out[name] = {"ms_per_apply": ms, "tflops": flops / ms / 1e9,
                     "algorithmic_bytes": alg, "hbm_gbs": alg / ms / 1e6, "hbm_frac": alg / ms / 1e6 / hbm,
                     "design_bytes": design, "design_hbm_frac": design / ms / 1e6 / hbm}
        if elem == 8:
            out[name]["fp64_frac"] = flops / ms / 1e9 / FP64_PEAK_TFLOPS
    out["hbm_peak"] = hbm
    out["fp64_peak"] = FP64_PEAK_TFLOPS
    if "fp32_tile" in kernels and "fp64_tile" in kernels:
        out["fp32_vs_fp64_rel_l2"] = float(torch.linalg.norm(y32.double() - y) / torch.linalg.norm(y))
    if "fp32_tile_tc" in kernels and "fp64_tile" in kernels:
        out["fp32_tc_vs_fp64_rel_l2"] = float(torch.linalg.norm(y32t.double() - y) / torch.linalg.norm(y))
    mesh.close()
    return out


def rel_l2(a, b) -> float:
    import numpy as np
    return float(np.linalg.norm(np.asarray(a) - np.asarray(b)) / max(np.linalg.norm(np.asarray(b)), 1e-300))


C3_TOL = 1e-10                     # the C3 configuration's refined residual
STRICT_TOL = {"fp64": 1e-13, "mixed": 1e-12}


def c3_run(dev, prec: str, wls, init, steps: int, warmup: int, keep=(), flush=None, timing=False, clocks=None,
           world: int = 1, tol: float = C3_TOL):
    """C3 batch in one precision: `warmup` untimed steps (the state after the first is kept for the
    tanks in `keep`), then `steps` steps, each timed alone with CUDA events on the stream, L2
    flushed before each (clocks sampled and library launches counted over the timed steps).
    Returns (figures, kept states, per-tank counters, stage-launch timing, final states)."""
    import torch
    import paper_1512_02548_gb300 as sem
    meshes = [sem.Mesh.from_workload(wl, precision=prec, tol=tol) for wl in wls]
    batch = sem.Batch(meshes)
    etas = [torch.tensor(e, device=dev) for e, _ in init]
    phis = [torch.tensor(p, device=dev) for _, p in init]
    dts = [wl.dt for wl in wls]
    kept = {}
    for k in range(max(1, warmup)):
        batch.rk4_step(etas, phis, dts, 1)
        if k == 0:
            kept = {i: (etas[i].cpu().numpy(), phis[i].cpu().numpy()) for i in keep}
    torch.cuda.synchronize()
    for m in meshes:
        m.reset_counters()
    batch.timing()
    batch.enable_timing(timing)
    stream = torch.cuda.current_stream()
    total = 0.0
    if world > 1:
        import torch.distributed as dist
        dist.barrier()
    torch.cuda.synchronize()
    if clocks is not None:
        clocks.start()
    launches0 = sem.launch_count()
    per_step = []
    for _ in range(steps):
        if flush is not None:
            flush.zero_()
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        batch.rk4_step(etas, phis, dts, 1)                 # synchronises (status check)
        e1.record(stream)
        e1.synchronize()
        per_step.append(e0.elapsed_time(e1))
        total += per_step[-1]
    torch.cuda.synchronize()
    launches = sem.launch_count() - launches0
    if world > 1:
        dist.barrier()
    clk = clocks.stop() if clocks is not None else None
    batch.enable_timing(False)
    tm = batch.timing()
    cnt = [m.counters() for m in meshes]
    info = batch.info()
    dof_step = 4 * sum(wl.n_unknowns for wl in wls)
    ms = total / steps
    srt = sorted(per_step)
    fig = {"ms_per_rk4_step": ms, "laplace_dof_per_s": dof_step / ms * 1e3,
           "step_ms": {"min": srt[0], "median": srt[len(srt) // 2], "max": srt[-1]},
           "tank_steps_per_s": len(wls) / ms * 1e3, **info, "total_ms": total, "launches": launches,
           "clocks": clk,
           "iterations_per_solve": sum(c.iterations for c in cnt) / max(1, sum(c.solves for c in cnt)),
           "refinements_per_solve": sum(c.refinements for c in cnt) / max(1, sum(c.solves for c in cnt)),
           "max_rel_residual": max(c.max_rel_residual for c in cnt)}
    final = [(e.cpu().numpy(), p.cpu().numpy()) for e, p in zip(etas, phis)]
    batch.close()
    for m in meshes:
        m.close()
    return fig, kept, cnt, tm, final


def c3_e2e(dev, wls, init, steps: int, warmup: int):
    """The batched FP64 step through sem_batch_rk4_step_host: every step copies all tanks' (η, φ̃)
    from packed pinned host buffers to the device and back (inside the timed region)."""
    import numpy as np
    import torch
    import paper_1512_02548_gb300 as sem
    meshes = [sem.Mesh.from_workload(wl, tol=C3_TOL) for wl in wls]
    batch = sem.Batch(meshes)
    eta_h = torch.tensor(np.concatenate([e for e, _ in init])).pin_memory()
    phis_h = torch.tensor(np.concatenate([p for _, p in init])).pin_memory()
    dts = [wl.dt for wl in wls]
    for _ in range(max(1, warmup)):
        batch.rk4_step_host(eta_h, phis_h, dts, 1)
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    for _ in range(steps):
        batch.rk4_step_host(eta_h, phis_h, dts, 1)
    wall = time.perf_counter() - t0
    batch.close()
    for m in meshes:
        m.close()
    return wall, 2 * 8 * int(eta_h.numel())


def c3_sequential(dev, wls, init, steps: int):
    """The same tanks one after another on the plain FP64 single-mesh path (sem_rk4_step)."""
    import torch
    import paper_1512_02548_gb300 as sem
    meshes = [sem.Mesh.from_workload(wl, tol=C3_TOL) for wl in wls]
    etas = [torch.tensor(e, device=dev) for e, _ in init]
    phis = [torch.tensor(p, device=dev) for _, p in init]
    for m, e, p, wl in zip(meshes, etas, phis, wls):
        m.rk4_step(e, p, wl.dt, 1)
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    for m, e, p, wl in zip(meshes, etas, phis, wls):
        m.rk4_step(e, p, wl.dt, steps)
    torch.cuda.synchronize()
    ms = (time.perf_counter() - t0) * 1e3 / steps
    for m in meshes:
        m.close()
    return {"ms_per_rk4_step": ms, "laplace_dof_per_s": 4 * sum(wl.n_unknowns for wl in wls) / ms * 1e3}


def c2_run(dev, steps: int, warmup: int, flush):
    """C2 steep periodic wave (64×4, P=6, P_f=9, filter (36,12,5), dt=T/200) on the single-mesh
    fused path, FP64 and mixed: `steps` RK4 steps each timed with CUDA events (L2 flushed before
    each), and the state after one step from the initial state for the oracle check."""
    import numpy as np
    import torch
    import paper_1512_02548_gb300 as sem
    from sem_workloads import c2_steep_periodic, initial_state
    wl = c2_steep_periodic()
    h = np.full(wl.ncol, wl.depth)
    e0, p0 = initial_state(wl, column_positions(wl), h)
    out = {"workload": wl.name, "unknowns": wl.n_unknowns, "dt": wl.dt}
    one = {}
    stream = torch.cuda.current_stream()
    for prec in ("fp64", "mixed"):
        m = sem.Mesh.from_workload(wl, h=h, precision=prec)
        eta, phis = torch.tensor(e0, device=dev), torch.tensor(p0, device=dev)
        m.rk4_step(eta, phis, wl.dt, 1)
        one[prec] = (eta.cpu().numpy(), phis.cpu().numpy())
        for _ in range(warmup - 1):
            m.rk4_step(eta, phis, wl.dt, 1)
        torch.cuda.synchronize()
        m.reset_counters()
        total = 0.0
        for _ in range(steps):
            flush.zero_()
            a = torch.cuda.Event(enable_timing=True)
            b = torch.cuda.Event(enable_timing=True)
            a.record(stream)
            m.rk4_step(eta, phis, wl.dt, 1)
            b.record(stream)
            b.synchronize()
            total += a.elapsed_time(b)
        c = m.counters()
        ms = total / steps
        out[prec] = {"ms_per_rk4_step": ms, "rk4_steps_per_s": 1e3 / ms,
                     "laplace_dof_per_s": 4 * wl.n_unknowns / ms * 1e3,
                     "iterations_per_solve": c.iterations / max(c.solves, 1),
                     "refinements_per_solve": c.refinements / max(c.solves, 1)}
        m.close()
    out["mixed_over_fp64"] = out["mixed"]["laplace_dof_per_s"] / out["fp64"]["laplace_dof_per_s"]
    return out, (e0, p0), one


def c4_shoal_run(dev, spinup: int = 600, steps: int = 100):
    """C4: JONSWAP waves generated over the synthetic shoal (2048×2, P=6, walls, relaxation
    zones), FP64 and mixed precision.  `spinup` untimed steps from rest let the generated
    waves fill the first part of the tank; then `steps` RK4 steps are timed with CUDA events.
    For the oracle check, one more step of each precision starts from the FP64 spun-up state."""
    import torch
    import paper_1512_02548_gb300 as sem
    from sem_workloads import c4_shoal, depth_columns
    wl = c4_shoal()
    h = depth_columns(wl, column_positions(wl))
    out = {"workload": wl.name, "unknowns": wl.n_unknowns, "dt": wl.dt, "spinup_steps": spinup, "steps": steps}
    res = {}
    start = None
    for prec in ("fp64", "mixed"):
        m = sem.Mesh.from_workload(wl, h=h, precision=prec, tol=1e-13 if prec == "fp64" else 1e-12)
        eta = torch.zeros(wl.ncol, dtype=torch.float64, device=dev)
        phis = torch.zeros_like(eta)
        t = m.rk4_step(eta, phis, wl.dt, spinup, t=0.0)
        if prec == "fp64":
            start = (eta.cpu().numpy(), phis.cpu().numpy(), t)
        m.reset_counters()
        torch.cuda.synchronize()
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record()
        m.rk4_step(eta, phis, wl.dt, steps, t=t)
        e1.record()
        e1.synchronize()
        ms = e0.elapsed_time(e1) / steps
        c = m.counters()
        out[prec] = {"ms_per_rk4_step": ms, "rk4_steps_per_s": 1e3 / ms,
                     "laplace_dof_per_s": 4 * wl.n_unknowns / ms * 1e3,
                     "iterations_per_solve": c.iterations / max(c.solves, 1),
                     "refinements_per_solve": c.refinements / max(c.solves, 1)}
        res[prec] = (eta, phis)
        m.close()
    out["mixed_vs_fp64_rel_l2"] = max(float(torch.linalg.norm(a - b) / torch.linalg.norm(b))
                                      for a, b in zip(res["mixed"], res["fp64"]))
    out["mixed_over_fp64"] = out["mixed"]["rk4_steps_per_s"] / out["fp64"]["rk4_steps_per_s"]
    out["max_abs_eta"] = float(res["fp64"][0].abs().max())
    one = {}
    for prec in ("fp64", "mixed"):
        m = sem.Mesh.from_workload(wl, h=h, precision=prec, tol=1e-13 if prec == "fp64" else 1e-12)
        eta = torch.tensor(start[0], device=dev)
        phis = torch.tensor(start[1], device=dev)
        m.rk4_step(eta, phis, wl.dt, 1, t=start[2])
        one[prec] = (eta.cpu().numpy(), phis.cpu().numpy())
        m.close()
    return out, start, one


def c5_serving(rates=(100.0, 1000.0), count: int = 1000, sample: int = 4, steps_per_tick: int = 1):
    """C5: Poisson streams of Laplace solves and 10-step RK4 runs (seed 0) served by the
    continuous-batching loop in mixed precision (150 GB admission budget; `steps_per_tick` > 1 lets
    a tick run several RK4 steps while nothing waits), against the same requests run one after
    another on the plain FP64 single-instance path.  Before either arm the host tables of the
    stream's (order, layers, over-integration, filter) combinations are built, as a server does
    at start-up.  Wall-clock from the first arrival; latency = completion − arrival.  The served
    results of a seeded sample of small requests at the first rate are kept for the oracle
    check."""
    import numpy as np
    from paper_1512_02548_gb300.serve import GpuExecutor, Request, Server, sequential
    from sem_workloads import c5_requests, initial_state, splitmix64
    keys = ("p50_ms", "p99_ms", "laplace_dof_per_s", "rk4_steps_per_s", "requests_per_s", "wall_s", "completed",
            "failed")
    out = {"requests_per_rate": count, "budget_gb": 150}
    warm = True
    checks = []
    for ri, rate in enumerate(rates):
        stream = c5_requests(rate, count, 0)
        base = []
        for i, (kind, t, wl, ns) in enumerate(stream):
            e0, p0 = initial_state(wl, column_positions(wl), np.full(wl.ncol, wl.depth))
            base.append(Request(i, kind, wl, e0, p0, ns, t))

        def fresh():
            return [Request(r.rid, r.kind, r.wl, r.eta0, r.phis0, r.nsteps, r.arrival) for r in base]

        keep = set()
        if ri == 0:
            gen = splitmix64(11)
            small = sorted((r.rid for r in base if r.wl.n_nodes <= 12000), key=lambda i: next(gen))
            lap = [i for i in small if base[i].kind == "laplace"][: sample // 2]
            rk = [i for i in small if base[i].kind == "rk4"][: sample - len(lap)]
            keep = set(lap + rk)
        if warm:
            Server(GpuExecutor("mixed"), 150 << 30).run(fresh()[:8])      # warm-up (module loading)
            warm = False
        # both arms start with the host tables of the stream's combinations built (the sequential
        # arm runs second and would otherwise find them built by the served arm)
        ent_warm = GpuExecutor("mixed").warm(base)
        ent = {"laplace_share": sum(r.kind == "laplace" for r in base) / count,
               "nodes_total": int(sum(r.wl.n_nodes for r in base)), "table_combinations_warmed": ent_warm}
        def slowest(rs, n=10):
            done = [r for r in rs if r.error is None and r.finished is not None]
            done.sort(key=lambda r: r.finished - r.arrival, reverse=True)
            return [{"kind": r.kind, "nodes": r.wl.n_nodes, "P": r.wl.P, "latency_ms": 1e3 * (r.finished - r.arrival),
                     "wait_ms": (1e3 * (r.admitted - r.arrival)) if r.admitted is not None else None}
                    for r in done[:n]]

        reqs = fresh()
        s = Server(GpuExecutor("mixed"), 150 << 30, keep_results=keep, max_steps_per_tick=steps_per_tick).run(reqs)
        ent["served_mixed"] = {k: s[k] for k in keys + ("ticks", "peak_active", "host_phases")}
        ent["served_mixed"]["slowest"] = slowest(reqs)
        for r in reqs:
            if r.rid in keep and r.error is None:
                checks.append((rate, count, r.rid, r.kind, r.eta0, r.phis0, r.nsteps, r.result))
        reqs = fresh()
        s = sequential(reqs, "fp64")
        ent["sequential_fp64"] = {k: s[k] for k in keys}
        ent["sequential_fp64"]["slowest"] = slowest(reqs)
        ent["served_mixed_dof_speedup_vs_sequential_fp64"] = (ent["served_mixed"]["laplace_dof_per_s"] /
                                                              ent["sequential_fp64"]["laplace_dof_per_s"])
        out[f"rate_{int(rate)}_per_s"] = ent
    return out, checks


def long_runs(dev, cores: int):
    """The full-length runs of C2 and C4 with their conservation diagnostics, computed by the oracle
    (all host cores) from GPU states:
      * C2 as configured (H/L = 0.08): FP64 steps until the library reports that the state is no
        longer regular (the wave, started from linear theory at this steepness, breaks), with the
        displaced volume and energy every 10 steps up to there;
      * C2 at H/L = 0.055, the steepest of the same family of initial states that runs 100 periods
        (20 000 steps, FP64 and mixed): volume and energy every 5 periods, and the drift;
      * C4 (5 000 steps, FP64 and mixed): volume and energy every 500 steps (the zones generate and
        absorb waves, so neither is conserved there).
    Returns a dict of series and summaries."""
    import numpy as np
    import torch
    import paper_1512_02548_gb300 as sem
    from sem_workloads import c2_steep_periodic, c4_shoal, depth_columns, initial_state
    pool = oracle_pool(cores)
    out = {}
    try:
        def diag(kind, key, states):
            futs = [(s, pool.apply_async(oracle_job, ((kind, key, e, p, -1, 0.0),))) for s, e, p in states]
            rows = [(s,) + tuple(f.get()[1]) for s, f in futs]
            return [{"step": s, "mass": m, "energy": en} for s, m, en in rows]

        # C2 as configured, until it stops
        wl = c2_steep_periodic()
        h = np.full(wl.ncol, wl.depth)
        e0, p0 = initial_state(wl, column_positions(wl), h)
        m = sem.Mesh.from_workload(wl, h=h)
        eta, phis = torch.tensor(e0, device=dev), torch.tensor(p0, device=dev)
        states, fail, err = [(0, e0, p0)], None, None
        for step in range(1, wl.nsteps + 1):
            try:
                m.rk4_step(eta, phis, wl.dt, 1)
            except sem.SemError as ex:
                fail, err = step, str(ex)
                break
            if step % 10 == 0:
                states.append((step, eta.cpu().numpy(), phis.cpu().numpy()))
        m.close()
        ser = diag("c2", 0, states)
        out["c2_as_configured"] = {"H_over_L": 0.08, "dt": wl.dt, "failed_at_step": fail, "error": err,
                                   "periods_run": (fail - 1 if fail else wl.nsteps) / 200.0, "series": ser}
        # C2 at H/L = 0.055 for 100 periods
        import dataclasses
        wl = dataclasses.replace(c2_steep_periodic(), wave_height=0.055 * c2_steep_periodic().length)
        e0, p0 = initial_state(wl, column_positions(wl), h)
        finals = {}
        for prec in ("fp64", "mixed"):
            m = sem.Mesh.from_workload(wl, h=h, precision=prec, tol=1e-13 if prec == "fp64" else 1e-12)
            eta, phis = torch.tensor(e0, device=dev), torch.tensor(p0, device=dev)
            states = [(0, e0, p0)]
            t0 = time.perf_counter()
            for k in range(1, 21):
                m.rk4_step(eta, phis, wl.dt, 1000)
                states.append((1000 * k, eta.cpu().numpy(), phis.cpu().numpy()))
            wall = time.perf_counter() - t0
            m.close()
            ser = diag("c2", 0.055, states)
            m0, E0 = ser[0]["mass"], ser[0]["energy"]
            scale = 0.5 * wl.wave_height * wl.length
            out[f"c2_hl0055_{prec}"] = {
                "steps": 20000, "periods": 100, "wall_s": wall, "series": ser,
                "max_abs_mass_drift_rel_to_HL2": max(abs(r["mass"] - m0) for r in ser) / scale,
                "energy_rel_change": (ser[-1]["energy"] - E0) / E0,
                "energy_increases": sum(1 for a, b in zip(ser, ser[1:]) if b["energy"] > a["energy"])}
            finals[prec] = states[-1]
        out["c2_hl0055_mixed_vs_fp64_rel_l2"] = max(rel_l2(finals["mixed"][1], finals["fp64"][1]),
                                                    rel_l2(finals["mixed"][2], finals["fp64"][2]))
        # C4, 5000 steps
        wl = c4_shoal()
        h = depth_columns(wl, column_positions(wl))
        finals = {}
        for prec in ("fp64", "mixed"):
            m = sem.Mesh.from_workload(wl, h=h, precision=prec, tol=1e-13 if prec == "fp64" else 1e-12)
            eta = torch.zeros(wl.ncol, dtype=torch.float64, device=dev)
            phis = torch.zeros_like(eta)
            t, states = 0.0, []
            t0 = time.perf_counter()
            for k in range(1, 11):
                t = m.rk4_step(eta, phis, wl.dt, 500, t=t)
                states.append((500 * k, eta.cpu().numpy(), phis.cpu().numpy()))
            wall = time.perf_counter() - t0
            m.close()
            out[f"c4_{prec}"] = {"steps": wl.nsteps, "wall_s": wall, "series": diag("c4", 0, states),
                                 "max_abs_eta": float(np.abs(states[-1][1]).max())}
            finals[prec] = states[-1]
        out["c4_mixed_vs_fp64_rel_l2"] = max(rel_l2(finals["mixed"][1], finals["fp64"][1]),
                                             rel_l2(finals["mixed"][2], finals["fp64"][2]))
    finally:
        pool.close()
        pool.join()
    return out


def measured_peaks() -> dict:
    try:
        return json.load(open(os.path.join(ROOT, "MEASURED_PEAKS.json")))
    except Exception:
        return {"hbm_gbs": 6800.0, "bf16_tflops": 1900.0}


# ---------------------------------------------------------------------------------------------
# GPU arm
# ---------------------------------------------------------------------------------------------
def run_gpu(args):
    import numpy as np
    import torch

    import paper_1512_02548_gb300 as sem
    from sem_workloads import c3_instances

    rank, world, local = dist_env()
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl" if torch.cuda.is_available() else "gloo")
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    sem.load_library()
    lead = rank == 0
    check = lead and world == 1 and not args.no_oracle

    wls = c3_instances(512)
    init = [c3_initial(i) for i in range(512)]
    flush = torch.empty(256 * 1024 * 1024 // 4, dtype=torch.float32, device=dev)   # > 129 MB L2
    sample = c3_sample(max(args.oracle_tanks, 2 * host_cores())) if check else []
    dof_step = 4 * sum(wl.n_unknowns for wl in wls)

    # ---- headline: C3 batched plain FP64 --------------------------------------------------
    clocks = ClockSampler(local)
    f64, kept64, cnt64, tm64, _ = c3_run(dev, "fp64", wls, init, args.steps, args.warmup, keep=sample,
                                         flush=flush, timing=True, clocks=clocks, world=world)
    t_max = max_over_ranks(f64["total_ms"], dev)
    value = job_throughput(world, args.steps, dof_step, t_max)
    tank_steps = job_throughput(world, args.steps, len(wls), t_max)
    mix, keptmx, cntmx, tmmx, _ = c3_run(dev, "mixed", wls, init, args.steps, args.warmup, keep=sample,
                                         flush=flush, timing=True, world=world)
    seq = c3_sequential(dev, wls, init, max(1, min(2, args.steps))) if lead else None
    # both paths again at the strict tolerances of the other configurations (1e-13 FP64, 1e-12 mixed)
    strict = {}
    for prec in ("fp64", "mixed"):
        fig, kept, _, _, _ = c3_run(dev, prec, wls, init, max(1, min(5, args.steps)), args.warmup, keep=sample,
                                    flush=flush, world=world, tol=STRICT_TOL[prec])
        strict[prec] = ({k: v for k, v in fig.items() if k not in ("total_ms", "clocks", "launches")}, kept)

    # roofline of the batched fused stage kernel.  The launches of the (order, precision, cluster
    # size) groups run at the same time on their own streams, so the unit is the whole step: FP64
    # Krylov work of all timed steps / their event-timed device time (the stage launches fill it)
    flops = sum(fp64_solver_flops(wl, c.solves, c.iterations, c.refinements, False) for wl, c in zip(wls, cnt64))
    launches = max(tm64.krylov_launches, 1)
    avg_launch_ms = tm64.krylov_ms / launches
    achieved = flops / (f64["total_ms"] / 1e3) / 1e12
    flops_mx = sum(fp64_solver_flops(wl, c.solves, c.iterations, c.refinements, True) for wl, c in zip(wls, cntmx))

    # end to end through the host-buffer batch call
    e2e_wall, e2e_bytes = c3_e2e(dev, wls, init, args.steps, args.warmup)
    e2e_s = max_over_ranks(e2e_wall, dev)
    e2e = {"value": job_throughput(world, args.steps, dof_step, 1e3 * e2e_s), "unit": UNIT,
           "h2d_bytes_per_step": e2e_bytes, "d2h_bytes_per_step": e2e_bytes,
           "call": "sem_batch_rk4_step_host (packed pinned host buffers)"}

    c3 = {"instances": len(wls), "unknowns": dof_step // 4,
          "batched_fp64": {k: v for k, v in f64.items() if k not in ("total_ms", "clocks")},
          "batched_mixed": {k: v for k, v in mix.items() if k not in ("total_ms", "clocks")},
          "sequential_fp64": seq,
          "mixed_over_batched_fp64": mix["laplace_dof_per_s"] / f64["laplace_dof_per_s"],
          "mixed_over_sequential_fp64": (mix["laplace_dof_per_s"] / seq["laplace_dof_per_s"]) if seq else None,
          "batched_fp64_over_sequential_fp64": (f64["laplace_dof_per_s"] / seq["laplace_dof_per_s"]) if seq else None,
          "at_strict_tol": {"fp64": strict["fp64"][0], "mixed": strict["mixed"][0],
                            "mixed_over_fp64": strict["mixed"][0]["laplace_dof_per_s"] /
                            strict["fp64"][0]["laplace_dof_per_s"],
                            "note": "relative residual 1e-13 (FP64) and 1e-12 with refinement (mixed); errors "
                                    "against the oracle in oracle_check"},
          "fp64_work_per_step_gflop": {"fp64": flops / args.steps / 1e9, "mixed": flops_mx / args.steps / 1e9},
          "stage_launch_ms": {"fp64": avg_launch_ms, "mixed": tmmx.krylov_ms / max(tmmx.krylov_launches, 1)}}

    line = {
        "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": t_max / args.steps, "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
        "config": {"workload": C3_NAME, "instances": len(wls), "n_unknowns": dof_step // 4, "precision": "fp64",
                   "tol": "relative residual 1e-10 (FP64 PCG; mixed: refined FP64 residual), the C3 configuration's",
                   "l2": "flushed between timed steps (256 MB write, untimed); working set above L2",
                   "parallelism": "replicas" if world > 1 else "single"},
        "rk4_steps_per_s": tank_steps,
        "mixed": {"value": mix["laplace_dof_per_s"] * world, "dtype": "f32+f64",
                  "over_batched_fp64": c3["mixed_over_batched_fp64"],
                  "over_sequential_fp64": c3["mixed_over_sequential_fp64"],
                  "tank_steps_per_s": mix["tank_steps_per_s"] * world},
        "c3_uneven_batch": c3,
        "roofline": {"bound": "alu", "kernel": "k_stage, batched fused RK stage with cluster teams, all "
                                               "concurrent launches of a step (FP64 Krylov work counted: applies "
                                               "and vector updates; the FP32 preconditioner left out)",
                     "achieved": achieved, "peak": FP64_PEAK_TFLOPS, "unit": "TFLOP/s",
                     "frac": achieved / FP64_PEAK_TFLOPS,
                     "peak_source": "nominal GB300 FP64 rate, 1.25 TFLOP/s (no measured FP64 peak)",
                     "unit_of_time": "event-timed device time of the timed steps",
                     "launches": tm64.krylov_launches, "avg_launch_ms": avg_launch_ms,
                     "flops_per_step": flops / args.steps,
                     # the unit of `achieved` is a whole step (all concurrent launches); the committed
                     # capture measured one group's launch alone, so it is reported beside, not as, traffic
                     "traffic": None,
                     "dram_bytes_per_group_launch_profiled": profiled_traffic("k_stage_batch")},
        "e2e": e2e,
        "gpu_launches": f64["launches"],
        "clocks": f64["clocks"],
    }

    extras = {}
    if lead and not args.no_c2:
        c2, c2_init, c2_one = c2_run(dev, args.steps, args.warmup, flush)
        line["c2_steep_wave"] = c2
        extras["c2"] = (c2_init, c2_one)
    if lead and not args.no_c4:
        c4, c4_start, c4_one = c4_shoal_run(dev)
        line["c4_shoal"] = c4
        extras["c4"] = (c4_start, c4_one)
    if lead and not args.no_c5:
        c5, c5_checks = c5_serving(tuple(args.c5_rates), args.c5_requests, steps_per_tick=args.c5_steps_per_tick)
        line["c5_serving"] = c5
        extras["c5"] = c5_checks
    if lead and not args.no_apply_roofline:
        line["apply_long_tank"] = apply_roofline(dev)

    if check:
        extras["c3_strict"] = {p: strict[p][1] for p in strict}
        oracle_checks(line, sample, init, kept64, keptmx, extras)
    if world > 1:
        dist.barrier()
    if lead:
        print(json.dumps(line))
    if world > 1:
        dist.destroy_process_group()
    return 0


def oracle_checks(line, sample, init, kept64, keptmx, extras):
    """The CPU oracle on all host cores: one RK4 step of each sampled C3 tank (timed: the
    cpu_baseline), then the oracle runs behind the C2, C4 and C5 error figures.  Each GPU
    result's relative L² error against the oracle is added to its section."""
    import numpy as np
    cores = host_cores()
    pool = oracle_pool(cores)
    try:
        jobs = [("c3", i, init[i][0], init[i][1], 1, 0.0) for i in sample]
        t0 = time.perf_counter()
        res = pool.map(oracle_job, jobs, chunksize=1)
        wall = time.perf_counter() - t0
        dof = sum(r[3] for r in res)
        cpu_s = sum(r[2] for r in res)
        err64 = max(max(rel_l2(kept64[i][0], r[1][0]), rel_l2(kept64[i][1], r[1][1])) for i, r in zip(sample, res))
        errmx = max(max(rel_l2(keptmx[i][0], r[1][0]), rel_l2(keptmx[i][1], r[1][1])) for i, r in zip(sample, res))
        line["cpu_baseline"] = {"value": dof / wall, "unit": UNIT, "cores": cores, "kind": "oracle",
                                "sample": f"one RK4 step (four banded-Cholesky Laplace solves) of each of {len(sample)} "
                                          f"seeded C3 tanks, one process per core on {cores} cores (nproc = "
                                          f"{os.cpu_count()}): {wall:.1f} s wall, {cpu_s:.1f} s of CPU work"}
        c3 = line["c3_uneven_batch"]
        c3["oracle_check"] = {"tanks": list(sample), "steps": 1, "fp64_max_rel_l2": err64, "mixed_max_rel_l2": errmx,
                              "tolerance": {"fp64": 1e-10, "mixed": 1e-8}}
        for prec, kept in extras.get("c3_strict", {}).items():
            c3["oracle_check"][f"{prec}_at_strict_tol_max_rel_l2"] = max(
                max(rel_l2(kept[i][0], r[1][0]), rel_l2(kept[i][1], r[1][1])) for i, r in zip(sample, res))
        line["mixed"]["max_rel_l2_vs_oracle"] = errmx
        line["max_rel_l2_vs_oracle"] = err64
        pending = []
        if "c2" in extras:
            (e0, p0), one = extras["c2"]
            pending.append(("c2", pool.apply_async(oracle_job, (("c2", 0, e0, p0, 1, 0.0),)), one))
        if "c4" in extras:
            (e0, p0, t), one = extras["c4"]
            pending.append(("c4", pool.apply_async(oracle_job, (("c4", 0, e0, p0, 1, t),)), one))
        for rate, count, rid, kind, e0, p0, ns, result in extras.get("c5", []):
            pending.append((("c5", kind, rid),
                            pool.apply_async(oracle_job, (("c5", (rate, count, rid), e0, p0, ns, 0.0),)), result))
        c5err = []
        for tag, fut, gpu in pending:
            _, ref, _, _ = fut.get()
            if tag == "c2":
                sec = line["c2_steep_wave"]
                for prec in ("fp64", "mixed"):
                    sec[prec]["rel_l2_vs_oracle_one_step"] = max(rel_l2(gpu[prec][0], ref[0]), rel_l2(gpu[prec][1], ref[1]))
            elif tag == "c4":
                sec = line["c4_shoal"]
                for prec in ("fp64", "mixed"):
                    sec[prec]["rel_l2_vs_oracle_one_step"] = max(rel_l2(gpu[prec][0], ref[0]), rel_l2(gpu[prec][1], ref[1]))
                sec["oracle_check"] = "one RK4 step from the FP64 state after the spin-up"
            else:
                err = rel_l2(gpu["Phi"], ref[0]) if tag[1] == "laplace" else \
                    max(rel_l2(gpu["eta"], ref[0]), rel_l2(gpu["phis"], ref[1]))
                c5err.append({"request": tag[2], "kind": tag[1], "rel_l2_vs_oracle": err})
        if c5err:
            line["c5_serving"]["oracle_check"] = {"served_mixed": c5err,
                                                  "max_rel_l2": max(e["rel_l2_vs_oracle"] for e in c5err)}
    finally:
        pool.close()
        pool.join()


def column_positions(wl):
    """Column x positions from the GLL nodes of order P (Newton on P'_P; input generation only)."""
    import numpy as np
    P = wl.P
    r = -np.cos(np.pi * np.arange(P + 1) / P)
    for _ in range(100):
        x = r[1:-1]
        p0, p1 = np.ones_like(x), x.copy()
        dp0, dp1 = np.zeros_like(x), np.ones_like(x)
        for k in range(1, P):
            p0, p1 = p1, ((2 * k + 1) * x * p1 - k * p0) / (k + 1)
            dp0, dp1 = dp1, dp0 + (2 * k + 1) * p0
        d2 = (2 * x * dp1 - P * (P + 1) * p1) / (1 - x * x)
        r[1:-1] = x - dp1 / d2
    from sem_workloads import column_x
    return column_x(wl, r)


def main():
    # one hardware work queue per stream of the batch's group launches (15 for the 512-tank batch;
    # CUDA's default of 8 makes streams share queues, where a launch waits behind another stream's);
    # read when the CUDA context is created, so before anything touches the GPU
    os.environ.setdefault("CUDA_DEVICE_MAX_CONNECTIONS", "32")
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=20)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="gb300", choices=["gb300", "reference"])
    ap.add_argument("--oracle-tanks", type=int, default=16, help="C3 tanks checked against the oracle (at least)")
    ap.add_argument("--no-oracle", action="store_true", help="skip the oracle checks and the cpu_baseline")
    ap.add_argument("--no-apply-roofline", action="store_true")
    ap.add_argument("--no-c2", action="store_true")
    ap.add_argument("--no-c4", action="store_true")
    ap.add_argument("--no-c5", action="store_true")
    ap.add_argument("--c5-rates", type=float, nargs="+", default=[100.0, 1000.0])
    ap.add_argument("--c5-requests", type=int, default=1000)
    ap.add_argument("--c5-steps-per-tick", type=int, default=1)
    ap.add_argument("--c5-sweep", action="store_true",
                    help="only the serving sweep: rates 10, 30, 100, 300, 1000, 2000 per s, 2000 requests each")
    ap.add_argument("--long-runs", action="store_true",
                    help="only the full-length C2 and C4 runs with the oracle's volume and energy diagnostics")
    ap.add_argument("--apply-only", default=None,
                    help="comma list of fp64_column,fp64_tile,fp32_tile,fp32_tile_tc: time only these applies")
    ap.add_argument("--apply-nx", type=int, default=65536)
    ap.add_argument("--apply-reps", type=int, default=20)
    args = ap.parse_args()
    if args.apply_only:
        import torch
        print(json.dumps(apply_roofline(torch.device("cuda", 0), args.apply_reps, args.apply_nx,
                                        tuple(args.apply_only.split(",")))))
        return 0
    if args.c5_sweep:
        import paper_1512_02548_gb300 as sem
        sem.load_library()
        out, _ = c5_serving((10.0, 30.0, 100.0, 300.0, 1000.0, 2000.0), 2000, steps_per_tick=args.c5_steps_per_tick)
        print(json.dumps({"c5_sweep": out}))
        return 0
    if args.long_runs:
        import torch
        import paper_1512_02548_gb300 as sem
        sem.load_library()
        print(json.dumps({"long_runs": long_runs(torch.device("cuda", 0), host_cores())}))
        return 0
    if args.warmup < 3:
        args.warmup = 3
    if args.impl == "reference":
        return run_reference(args)
    return run_gpu(args)


if __name__ == "__main__":
    sys.exit(main())
