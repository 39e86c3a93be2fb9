"""Autotuner: measured batch planning parameters and tiled-apply widths for this GPU.

Run on the GPU:

    python -m paper_1512_02548_gb300.autotune [--out PATH] [--quick]

It measures, with CUDA events on the launching stream,

* the batched RK4 step (FP64 and mixed precision) of a seeded set of uneven periodic tanks drawn
  like the 512-tank batch but from another seed (so the benchmark's own tanks are not what is
  tuned on), for every candidate of the batch planning parameters of ``sem_set_batch_tuning``:
  the cluster team share, the largest cluster and the group size up to which the one-CTA-per-SM
  build is used; the candidate with the smallest summed step time wins;
* the FP32 tiled apply on a long periodic tank of about 9.8 M nodes (above the L2, flushed before
  each timed apply) for every order P = 2..12, layer count Nz = 1, 2, 4 and tile width E = 1..16
  that fits in shared memory; the fastest width per (P, Nz) wins (the FP64 apply keeps its rule);

and writes the winners with every measurement to ``tuning.json`` next to this file (or PATH);
``--apply-only`` re-measures the tile widths alone and keeps the file's batch section.
:func:`apply_tuning` reads that file and hands the winners to the library, if it was measured on
a GPU of the same name, each part once per process: ``Batch`` applies the batch parameters before
its first batch and ``Mesh`` the tile widths when the first mesh is created.  Results do
not depend on the tuning (team sizes and tile widths change only the summation order within each
team's reductions), which ``tests/test_gpu_autotune.py`` checks.
"""
from __future__ import annotations

import argparse
import itertools
import json
import os
import time

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
TUNING_PATH = os.path.join(HERE, "tuning.json")
_applied: set = set()


def apply_tuning(path: str = TUNING_PATH, batch: bool = True, tiles: bool = True) -> dict | None:
    """Hand the measured winners in `path` to the library: the batch planning parameters and/or
    the tile widths, each at most once per process; None if there is no file or it was measured on
    another GPU."""
    parts = [p for p, on in (("batch", batch), ("tiles", tiles)) if on and p not in _applied]
    if not parts:
        return None
    _applied.update(parts)
    if not os.path.exists(path):
        return None
    import torch
    from . import set_apply_tile_width, set_batch_tuning
    data = json.load(open(path))
    if not torch.cuda.is_available() or data.get("device") != torch.cuda.get_device_name(0):
        return None
    if "batch" in parts:
        b = data["batch"]
        set_batch_tuning(cluster_share=b["cluster_share"], max_cluster=b["max_cluster"],
                         narrow_max=b["narrow_max"], plan=b["plan"])
    if "tiles" in parts:
        for key, E in data.get("apply_tile_width", {}).items():
            P, Nz = (int(v) for v in key.split(","))
            set_apply_tile_width(P, Nz, E)
    return data


def _column_x(wl):
    # column positions: GLL nodes of order P by Newton on P'_P (inputs only)
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


def time_batch(wls, init, precision: str, steps: int, dev) -> float:
    """ms per batched RK4 step of the tanks `wls` from `init`, after one untimed step."""
    import torch
    from . import Batch, Mesh
    meshes = [Mesh.from_workload(wl, precision=precision, tol=1e-13 if precision == "fp64" else 1e-12)
              for wl in wls]
    batch = Batch(meshes, tuned=False)
    etas = [torch.tensor(e, device=dev) for e, _ in init]
    phis = [torch.tensor(p, device=dev) for _, p in init]
    dts = [wl.dt for wl in wls]
    batch.rk4_step(etas, phis, dts, 1)
    torch.cuda.synchronize()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record()
    batch.rk4_step(etas, phis, dts, steps)
    e1.record()
    e1.synchronize()
    batch.close()
    for m in meshes:
        m.close()
    return e0.elapsed_time(e1) / steps


def tune_batch(dev, count: int = 512, seed: int = 1, steps: int = 3, quick: bool = False):
    from sem_workloads import c3_instances, initial_state
    from . import set_batch_tuning
    wls = c3_instances(count, seed=seed)
    init = [initial_state(wl, _column_x(wl), np.full(wl.ncol, wl.depth)) for wl in wls]
    shares = (0.25, 0.5, 1.0) if quick else (0.125, 0.25, 0.5, 1.0, 2.0)
    clusters = (8, 16) if quick else (4, 8, 16)
    narrows = (8,) if quick else (8, 1 << 20)
    rows = []
    for share, mc, nm in itertools.product(shares, clusters, narrows):
        set_batch_tuning(cluster_share=share, max_cluster=mc, narrow_max=nm, plan=-1, reset=True)
        ms = {p: time_batch(wls, init, p, steps, dev) for p in ("fp64", "mixed")}
        rows.append({"cluster_share": share, "max_cluster": mc, "narrow_max": nm, "plan": -1,
                     "fp64_ms": ms["fp64"], "mixed_ms": ms["mixed"]})
    set_batch_tuning(reset=True, plan=0)
    ms = {p: time_batch(wls, init, p, steps, dev) for p in ("fp64", "mixed")}
    rows.append({"cluster_share": 0.5, "max_cluster": 16, "narrow_max": 8, "plan": 0,
                 "fp64_ms": ms["fp64"], "mixed_ms": ms["mixed"]})
    set_batch_tuning(reset=True)
    best = min(rows, key=lambda r: r["fp64_ms"] + r["mixed_ms"])
    return {k: best[k] for k in ("cluster_share", "max_cluster", "narrow_max", "plan")}, rows


def tune_apply(dev, nodes: float = 9.8e6, reps: int = 7, quick: bool = False):
    """FP32 tile widths on long tanks of about `nodes` nodes (x and y above the L2), the L2 flushed
    before each timed apply, median of `reps`."""
    import torch
    from . import Mesh, set_apply_tile_width
    from sem_workloads import roofline_tank
    winners, rows = {}, []
    flush = torch.empty(64 << 20, dtype=torch.float32, device=dev)   # 256 MB, above the L2
    orders = (4, 6, 8) if quick else range(2, 13)
    for P in orders:
        for Nz in (1, 2, 4):
            Nx = max(64, int(nodes / (P * (Nz * P + 1))))
            wl = roofline_tank(Nx=Nx, Nz=Nz, P=P)
            mesh = Mesh.from_workload(wl)
            mesh.update_geometry(torch.zeros(wl.ncol, dtype=torch.float64, device=dev))
            x = torch.randn(mesh.n, dtype=torch.float32, device=dev)
            y = torch.empty_like(x)
            best = None
            for E in range(1, 17):
                set_apply_tile_width(P, Nz, E)
                try:
                    for _ in range(2):
                        mesh.laplace_apply_f32(x, y)
                except Exception:
                    continue
                torch.cuda.synchronize()
                ts = []
                for _ in range(reps):
                    flush.zero_()
                    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
                    e0.record()
                    mesh.laplace_apply_f32(x, y)
                    e1.record()
                    e1.synchronize()
                    ts.append(e0.elapsed_time(e1))
                ms = float(np.median(ts))
                rows.append({"P": P, "Nz": Nz, "E": E, "ms": ms, "nodes": mesh.n})
                if best is None or ms < best[1]:
                    best = (E, ms)
            set_apply_tile_width(P, Nz, 0)
            mesh.close()
            if best:
                winners[f"{P},{Nz}"] = best[0]
    return winners, rows


def main():
    import torch
    from . import load_library
    ap = argparse.ArgumentParser()
    ap.add_argument("--out", default=TUNING_PATH)
    ap.add_argument("--quick", action="store_true", help="fewer candidates (for tests)")
    ap.add_argument("--apply-only", action="store_true",
                    help="re-measure the tile widths only; keep the batch section of the existing file")
    args = ap.parse_args()
    load_library()
    dev = torch.device("cuda", 0)
    t0 = time.time()
    if args.apply_only:
        old = json.load(open(args.out))
        batch, batch_rows = old["batch"], old["measured"]["batch"]
    else:
        batch, batch_rows = tune_batch(dev, quick=args.quick)
    tiles, tile_rows = tune_apply(dev, quick=args.quick)
    out = {"device": torch.cuda.get_device_name(0), "when": time.strftime("%Y-%m-%dT%H:%M:%SZ", time.gmtime()),
           "batch": batch, "apply_tile_width": tiles,
           "measured": {"batch": batch_rows, "apply_tile": tile_rows,
                        "batch_workload": "512 uneven periodic tanks, seed 1, drawn like the benchmark batch (seed 0)",
                        "seconds": time.time() - t0}}
    with open(args.out, "w") as f:
        json.dump(out, f, indent=1)
    print(json.dumps({"batch": batch, "apply_tile_width": tiles, "seconds": out["measured"]["seconds"]}))


if __name__ == "__main__":
    main()
