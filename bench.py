"""Benchmark: Laplace DOF/s and RK4 steps/s of the σ-transformed SEM wave model on GB300.

Workload (one "step"): one classical RK4 step of the steep periodic nonlinear wave
(64×4 elements, P=6, P_f=9, filter (36,12,P-1), kh=1, H/L=0.08, dt=T/200) —
four σ-geometry updates, four Dirichlet-lifted Laplace solves (persistent PCG),
four gradient recoveries, four over-integrated Zakharov right-hand sides, the RK4
combination and the modal filter, all in the library's CUDA kernels.

value   = Laplace DOF/s = 4 · n_unknowns · steps / device time (FP64 path);
e2e     = the same metric through sem_rk4_step_host (pinned host buffers,
          host↔device copies of (η, φ̃) inside the timed region);
roofline: dominant kernel = the persistent Krylov kernel, FP64-ALU bound;
cpu_baseline: the CPU oracle on a bounded sample of the same workload.

`--impl reference` times the CPU oracle itself (the reference arm).  Under
torchrun each rank runs an independent replica of the tank (weak scaling, no
data-path collective); rank 0 prints the JSON line.
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

METRIC = "Laplace DOF/s (RK4 steps/s alongside)"
UNIT = "DOF/s"
# Algorithmic FP64 work of one Krylov iteration (per-unit figures stated in the design notes):
#   operator apply: 8(P+1)+7 flops per element-local node (gradients, fluxes, transposed sums)
#   vector updates and dots: 13 flops per unknown
#   σ-separable preconditioner: see flops_per_precond
FP64_PEAK_TFLOPS = 1.25   # nominal GB300 FP64 rate (vector and tensor alike)


def workload():
    from sem_workloads import c2_steep_periodic
    return c2_steep_periodic()


def flops_per_precond(wl) -> float:
    """σ-separable preconditioner: two σ-transforms (nr² FMAs per column each), per-(mode,
    element) condensation and back-substitution ((P−1)² + 4(P−1) FMAs), interface solve."""
    P, nr = wl.P, wl.nrow - 1
    nif = wl.Nx if wl.periodic else wl.Nx + 1
    return 4 * wl.ncol * nr * nr + 2 * nr * wl.Nx * ((P - 1) ** 2 + 4 * (P - 1)) + 6 * nr * nif


def flops_per_iteration(wl) -> float:
    P = wl.P
    return (wl.Nx * wl.Nz * (P + 1) ** 2 * (8 * (P + 1) + 7) + 13 * wl.n_unknowns
            + flops_per_precond(wl))


def flops_per_apply(wl) -> float:
    P = wl.P
    return wl.Nx * wl.Nz * (P + 1) ** 2 * (8 * (P + 1) + 7)


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
def oracle_stage_sample(n_stages: int):
    """Run n_stages RK4 stages of the oracle on the bench workload; returns (seconds, DOF)."""
    import numpy as np
    from oracle import sem as osem
    from sem_workloads import initial_state
    wl = workload()
    om = osem.mesh_for(wl)
    eta, phis = initial_state(wl, om.xcol, om.h)
    om.surface_mass()
    om.mass2d()
    om.laplace_solve(eta, phis)          # RCM ordering and mass factors are set-up, not timed
    t0 = time.perf_counter()
    for _ in range(n_stages):
        de, dp = om.zakharov_rhs(eta, phis)
        eta = eta + 0.5 * wl.dt * de
        phis = phis + 0.5 * wl.dt * dp
    dt = time.perf_counter() - t0
    assert np.all(np.isfinite(eta))
    return dt, n_stages * wl.n_unknowns


def oracle_subprocess(n_stages: int) -> dict:
    env = dict(os.environ)
    for k in ("OMP_NUM_THREADS", "OPENBLAS_NUM_THREADS", "MKL_NUM_THREADS", "BLIS_NUM_THREADS"):
        env[k] = "1"
    env["CUDA_VISIBLE_DEVICES"] = ""
    code = ("import json,sys; sys.path.insert(0, %r); import bench; "
            "t, dof = bench.oracle_stage_sample(%d); print(json.dumps({'t': t, 'dof': dof}))" % (ROOT, n_stages))
    out = subprocess.run([sys.executable, "-c", code], env=env, capture_output=True, text=True, timeout=900)
    if out.returncode != 0:
        raise RuntimeError(out.stderr[-2000:])
    return json.loads(out.stdout.strip().splitlines()[-1])


def run_reference(args):
    rank, world, _ = dist_env()
    if rank != 0:
        return 0
    wl = workload()
    # warm-up stages, then K timed stages: one "step" = one RK4 stage (one Laplace solve)
    oracle_subprocess(max(1, min(args.warmup, 1)))
    res = oracle_subprocess(args.steps)
    value = res["dof"] / res["t"]
    line = {
        "impl": "reference", "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": args.gpus,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * res["t"] / args.steps,
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
        "data": "synthetic",
        "config": {"workload": wl.name, "Nx": wl.Nx, "Nz": wl.Nz, "P": wl.P, "Pf": wl.Pf,
                   "n_unknowns": wl.n_unknowns, "step": "one RK4 stage of the CPU oracle",
                   "parallelism": "replicas"},
        "cpu_baseline": {"value": value, "unit": UNIT, "cores": 1, "kind": "oracle",
                         "sample": f"{args.steps} RK4 stages of the C2 tank (one banded-Cholesky "
                                   f"Laplace solve each), single thread"},
        "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line))
    return 0


# ---------------------------------------------------------------------------------------------
# Supplementary: the operator apply on a long tank (working set above L2)
# ---------------------------------------------------------------------------------------------
def apply_roofline(dev, reps: int = 20, Nx: int = 65536, kernels=("fp64_column", "fp64_tile", "fp32_tile")):
    """The operator apply y = 𝓛x on a 65536×4, P=6 periodic tank (9.8 M nodes), three kernels:
    the FP64 tiled kernel (sem_laplace_apply), the FP64 element-column kernel (same call with
    SEM_APPLY_KERNEL=column) and the FP32 tiled kernel of the mixed path (sem_laplace_apply_f32).

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

    def column64():
        old = os.environ.get("SEM_APPLY_KERNEL")
        os.environ["SEM_APPLY_KERNEL"] = "column"
        try:
            mesh.laplace_apply(x, y)
        finally:
            if old is None:
                del os.environ["SEM_APPLY_KERNEL"]
            else:
                os.environ["SEM_APPLY_KERNEL"] = old

    P = wl.P
    flops = wl.Nx * wl.Nz * (P + 1) ** 2 * (8 * (P + 1) + 7)
    geo_cols = wl.Nx * (P + 1)
    peaks = measured_peaks()
    hbm = peaks.get("hbm_gbs")
    out = {"workload": wl.name, "n_nodes": mesh.n, "flops_per_apply": flops, "l2_flushed": True}
    for name, fn, elem in (("fp64_column", column64, 8), ("fp64_tile", lambda: mesh.laplace_apply(x, y), 8),
                           ("fp32_tile", lambda: mesh.laplace_apply_f32(x32, y32), 4)):
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
    if "fp32_tile" in kernels and len(kernels) > 1:
        out["fp32_vs_fp64_rel_l2"] = float(torch.linalg.norm(y32.double() - y) / torch.linalg.norm(y))
    mesh.close()
    return out


def c3_batch(dev, count: int = 512, steps: int = 3):
    """C3: uneven periodic tanks (seed 0) stepped together, mixed precision and FP64, against the
    same tanks stepped one after another on the plain FP64 path.  Laplace DOF/s = 4·Σ unknowns
    per RK4 step / time; the mixed path is checked against the FP64 batch (≤1e-8 rel)."""
    import numpy as np
    import torch
    import paper_1512_02548_gb300 as sem
    from sem_workloads import c3_instances, initial_state
    wls = c3_instances(count)
    out = {"instances": count, "unknowns": int(sum(w.n_unknowns for w in wls))}
    dof_step = 4 * out["unknowns"]
    init = []
    for wl in wls:
        xcol = column_positions(wl)
        init.append(initial_state(wl, xcol, np.full(wl.ncol, wl.depth)))
    dts = [wl.dt for wl in wls]
    results = {}
    for prec in ("fp64", "mixed"):
        meshes = [sem.Mesh.from_workload(wl, precision=prec, tol=1e-13 if prec == "fp64" else 1e-12) for wl in wls]
        batch = sem.Batch(meshes)
        etas = [torch.tensor(e, device=dev) for e, _ in init]
        phis = [torch.tensor(p, device=dev) for _, p in init]
        batch.rk4_step(etas, phis, dts, 1)                       # warm-up step
        torch.cuda.synchronize()
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record()
        batch.rk4_step(etas, phis, dts, steps)
        e1.record()
        e1.synchronize()
        ms = e0.elapsed_time(e1) / steps
        info = batch.info()
        results[prec] = (etas, phis)
        out[f"batched_{prec}"] = {"ms_per_rk4_step": ms, "laplace_dof_per_s": dof_step / ms * 1e3,
                                  "tank_steps_per_s": count / ms * 1e3, **info}
        batch.close()
        for m in meshes:
            m.close()
    err = max(float(torch.linalg.norm(a - b) / torch.linalg.norm(b))
              for a, b in zip(results["mixed"][0] + results["mixed"][1], results["fp64"][0] + results["fp64"][1]))
    out["mixed_vs_fp64_max_rel_l2"] = err
    # sequential plain FP64: one mesh after another, same steps
    meshes = [sem.Mesh.from_workload(wl) for wl in wls]
    etas = [torch.tensor(e, device=dev) for e, _ in init]
    phis = [torch.tensor(p, device=dev) for _, p in init]
    for m, e, p, dt in zip(meshes, etas, phis, dts):
        m.rk4_step(e, p, dt, 1)
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    for m, e, p, dt in zip(meshes, etas, phis, dts):
        m.rk4_step(e, p, dt, steps)
    torch.cuda.synchronize()
    ms = (time.perf_counter() - t0) * 1e3 / steps
    out["sequential_fp64"] = {"ms_per_rk4_step": ms, "laplace_dof_per_s": dof_step / ms * 1e3}
    for m in meshes:
        m.close()
    out["mixed_batched_speedup_vs_sequential_fp64"] = out["sequential_fp64"]["ms_per_rk4_step"] / \
        out["batched_mixed"]["ms_per_rk4_step"]
    return out


def c4_shoal_run(dev, spinup: int = 600, steps: int = 100):
    """C4: JONSWAP waves generated over the synthetic shoal (2048×2, P=6, walls, relaxation
    zones), FP64 and mixed precision.  `spinup` untimed steps from rest let the generated
    waves fill the first part of the tank; then `steps` RK4 steps are timed with CUDA events.
    The two precisions are compared at the end (relative L2 of η and φ̃)."""
    import numpy as np
    import torch
    import paper_1512_02548_gb300 as sem
    from sem_workloads import c4_shoal, depth_columns
    wl = c4_shoal()
    h = depth_columns(wl, column_positions(wl))
    out = {"workload": wl.name, "unknowns": wl.n_unknowns, "dt": wl.dt, "spinup_steps": spinup, "steps": steps}
    res = {}
    for prec in ("fp64", "mixed"):
        m = sem.Mesh.from_workload(wl, h=h, precision=prec, tol=1e-13 if prec == "fp64" else 1e-12)
        eta = torch.zeros(wl.ncol, dtype=torch.float64, device=dev)
        phis = torch.zeros_like(eta)
        t = m.rk4_step(eta, phis, wl.dt, spinup, t=0.0)
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
    out["max_abs_eta"] = float(res["fp64"][0].abs().max())
    return out


def c5_serving(rates=(100.0, 1000.0), count: int = 300):
    """C5: Poisson streams of Laplace solves and 10-step RK4 runs (seed 0) served by the
    continuous-batching loop in mixed precision (150 GB admission budget), against the same
    requests run one after another on the plain FP64 single-instance path.  Wall-clock from
    the first arrival; latency = completion − arrival.  One rate below the loop's capacity and
    one above it."""
    import numpy as np
    from paper_1512_02548_gb300.serve import GpuExecutor, Request, Server, sequential
    from sem_workloads import c5_requests, initial_state
    keys = ("p50_ms", "p99_ms", "laplace_dof_per_s", "rk4_steps_per_s", "requests_per_s", "wall_s", "completed",
            "failed")
    out = {"requests_per_rate": count, "budget_gb": 150}
    warm = True
    for rate in rates:
        base = []
        for i, (kind, t, wl, ns) in enumerate(c5_requests(rate, count, 0)):
            e0, p0 = initial_state(wl, column_positions(wl), np.full(wl.ncol, wl.depth))
            base.append(Request(i, kind, wl, e0, p0, ns, t))

        def fresh():
            return [Request(r.rid, r.kind, r.wl, r.eta0, r.phis0, r.nsteps, r.arrival) for r in base]

        if warm:
            Server(GpuExecutor("mixed"), 150 << 30).run(fresh()[:8])      # warm-up (module loading)
            warm = False
        ent = {"laplace_share": sum(r.kind == "laplace" for r in base) / count,
               "nodes_total": int(sum(r.wl.n_nodes for r in base))}
        s = Server(GpuExecutor("mixed"), 150 << 30, keep_results=False).run(fresh())
        ent["served_mixed"] = {k: s[k] for k in keys + ("ticks", "peak_active")}
        s = sequential(fresh(), "fp64")
        ent["sequential_fp64"] = {k: s[k] for k in keys}
        ent["served_mixed_dof_speedup_vs_sequential_fp64"] = (ent["served_mixed"]["laplace_dof_per_s"] /
                                                              ent["sequential_fp64"]["laplace_dof_per_s"])
        out[f"rate_{int(rate)}_per_s"] = ent
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
    from sem_workloads import initial_state

    rank, world, local = dist_env()
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl" if torch.cuda.is_available() else "gloo")
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    sem.load_library()

    wl = workload()
    # column positions need GLL nodes; take them from a throw-away oracle-free formula:
    # the library only needs edges and depth, initial data are sampled at the columns.
    h = np.full(wl.ncol, wl.depth)
    mesh = sem.Mesh.from_workload(wl, h=h, precision=args.precision)
    xcol = column_positions(wl)
    eta0, phis0 = initial_state(wl, xcol, h)
    eta = torch.tensor(eta0, device=dev)
    phis = torch.tensor(phis0, device=dev)
    flush = torch.empty(256 * 1024 * 1024 // 4, dtype=torch.float32, device=dev)   # > 129 MB L2
    stream = torch.cuda.current_stream()

    for _ in range(args.warmup):
        mesh.rk4_step(eta, phis, wl.dt, 1)
    torch.cuda.synchronize()
    mesh.reset_counters()
    mesh.timing()                                   # discard
    mesh.enable_timing(True)
    launches0 = sem.launch_count()
    clocks = ClockSampler(local)
    clocks.start()
    if world > 1:
        dist.barrier()
    torch.cuda.synchronize()
    total_ms = 0.0
    for _ in range(args.steps):
        flush.zero_()                               # evict L2 between timed steps (not timed)
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        mesh.rk4_step(eta, phis, wl.dt, 1)          # synchronises at its end (status check)
        e1.record(stream)
        e1.synchronize()
        total_ms += e0.elapsed_time(e1)
    torch.cuda.synchronize()
    if world > 1:
        dist.barrier()
    clk = clocks.stop()
    gpu_launches = sem.launch_count() - launches0
    mesh.enable_timing(False)
    tm = mesh.timing()
    cnt = mesh.counters()
    t_max = max_over_ranks(total_ms, dev)
    dof_per_step = 4 * wl.n_unknowns
    value = job_throughput(world, args.steps, dof_per_step, t_max)
    steps_per_s = job_throughput(world, args.steps, 1, t_max)

    # roofline of the dominant kernel: the fused RK-stage kernel (Laplace solve inside), FP64 ALU
    # bound; its algorithmic work is counted from the Krylov part only (a lower bound)
    solves = max(cnt.solves, 1)
    # per solve: 2 FP64 applies for r0 and b, one preconditioner application per start
    # (1 in FP64, one per refinement in mixed), one FP64 apply per refinement
    extra_applies = 2 * cnt.solves + cnt.refinements
    starts = cnt.refinements if args.precision == "mixed" else cnt.solves
    flops = (cnt.iterations * flops_per_iteration(wl) + extra_applies * flops_per_apply(wl)
             + starts * flops_per_precond(wl))
    avg_launch_ms = tm.krylov_ms / max(tm.krylov_launches, 1)
    flops_per_launch = flops / max(tm.krylov_launches, 1)
    achieved = flops_per_launch / (avg_launch_ms / 1e3) / 1e12
    krylov_share = tm.krylov_ms / total_ms if total_ms > 0 else None

    # end to end through the host-buffer entry point
    he = torch.tensor(eta0).pin_memory().numpy()
    hp = torch.tensor(phis0).pin_memory().numpy()
    for _ in range(2):
        mesh.rk4_step_host(he, hp, wl.dt, 1)
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    for _ in range(args.steps):
        mesh.rk4_step_host(he, hp, wl.dt, 1)
    e2e_s = max_over_ranks(time.perf_counter() - t0, dev)
    e2e = {"value": job_throughput(world, args.steps, dof_per_step, 1e3 * e2e_s), "unit": UNIT,
           "h2d_bytes_per_step": 2 * 8 * wl.ncol, "d2h_bytes_per_step": 2 * 8 * wl.ncol}

    line = {
        "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": t_max / args.steps, "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "f64" if args.precision == "fp64" else "f32+f64",
        "data": "synthetic",
        "config": {"workload": wl.name, "Nx": wl.Nx, "Nz": wl.Nz, "P": wl.P, "Pf": wl.Pf,
                   "n_unknowns": wl.n_unknowns, "dt": wl.dt, "precision": args.precision,
                   "l2": "flushed between timed steps (256 MB write, untimed)",
                   "parallelism": "replicas" if world > 1 else "single"},
        "rk4_steps_per_s": steps_per_s,
        "krylov": {"solves": cnt.solves, "iterations_per_solve": cnt.iterations / solves,
                   "refinements": cnt.refinements, "max_rel_residual": cnt.max_rel_residual,
                   "stage_kernel_share_of_step_time": krylov_share},
        "roofline": {"bound": "alu", "kernel": "k_stage (fused RK stage, Krylov work counted)",
                     "achieved": achieved,
                     "peak": FP64_PEAK_TFLOPS, "unit": "TFLOP/s", "frac": achieved / FP64_PEAK_TFLOPS,
                     "peak_source": "nominal GB300 FP64 rate, 1.25 TFLOP/s",
                     "traffic": profiled_traffic("k_stage")},
        "e2e": e2e,
        "gpu_launches": gpu_launches,
        "clocks": clk,
    }
    if not args.no_apply_roofline:
        line["apply_long_tank"] = apply_roofline(dev)
    if not args.no_c3:
        line["c3_uneven_batch"] = c3_batch(dev)
    if not args.no_c4:
        line["c4_shoal"] = c4_shoal_run(dev)
    if not args.no_c5:
        line["c5_serving"] = c5_serving(tuple(args.c5_rates), args.c5_requests)
    if rank == 0 and not args.no_cpu_baseline:
        try:
            res = oracle_subprocess(args.cpu_stages)
            line["cpu_baseline"] = {"value": res["dof"] / res["t"], "unit": UNIT, "cores": 1, "kind": "oracle",
                                    "sample": f"{args.cpu_stages} RK4 stages of the same tank (one banded-"
                                              f"Cholesky Laplace solve each), single thread, "
                                              f"{res['t']:.1f} s"}
        except Exception as e:  # the GPU number stands on its own
            line["cpu_baseline"] = {"value": None, "unit": UNIT, "cores": 1, "kind": "oracle",
                                    "sample": f"failed: {str(e)[-200:]}"}
    if rank == 0:
        print(json.dumps(line))
    mesh.close()
    if world > 1:
        dist.destroy_process_group()
    return 0


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
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=20)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="gb300", choices=["gb300", "reference"])
    ap.add_argument("--precision", default="fp64", choices=["fp64", "mixed"])
    ap.add_argument("--cpu-stages", type=int, default=8)
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-apply-roofline", action="store_true")
    ap.add_argument("--no-c3", action="store_true")
    ap.add_argument("--no-c4", action="store_true")
    ap.add_argument("--no-c5", action="store_true")
    ap.add_argument("--c5-rates", type=float, nargs="+", default=[100.0, 1000.0])
    ap.add_argument("--c5-requests", type=int, default=300)
    ap.add_argument("--apply-only", default=None,
                    help="comma list of fp64_column,fp64_tile,fp32_tile: time only these applies (for profiling)")
    ap.add_argument("--apply-nx", type=int, default=65536)
    ap.add_argument("--apply-reps", type=int, default=20)
    args = ap.parse_args()
    if args.apply_only:
        import torch
        print(json.dumps(apply_roofline(torch.device("cuda", 0), args.apply_reps, args.apply_nx,
                                        tuple(args.apply_only.split(",")))))
        return 0
    if args.warmup < 3:
        args.warmup = 3
    if args.impl == "reference":
        return run_reference(args)
    return run_gpu(args)


if __name__ == "__main__":
    sys.exit(main())
