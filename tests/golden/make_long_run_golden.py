"""Writes the oracle trajectories that the long-run GPU parity tests compare against.

Calls only the CPU oracle (``oracle/``) and the seeded input generators (``sem_workloads``);
nothing here runs on or reads from the CUDA library.  Run from the repository root:

    python tests/golden/make_long_run_golden.py [c2] [c4] [c5big]

Files (numpy .npz, FP64):
  c2_window.npz     C2 steep periodic wave (64×4, P=6, P_f=9, filter (36,12,5), dt=T/200) from its
                    initial state: η, φ̃ after 1, 25, 50 and 75 RK4 steps (all 384 columns), the
                    displaced volume 1ᵀM'η and energy ½Φᵀ(−𝓛)Φ + ½gηᵀM'η every 5 steps (§3.1.1 RK4,
                    §3.4 filter; the diagnostics of the paper's stability study, §4.3), and the first
                    step at which the oracle fails: the wave started from linear theory at this
                    steepness keeps steepening, and within about half a period its state stops being
                    finite, or the depth positive, or the σ-Laplace matrix definite.
  c4_window.npz     C4 JONSWAP waves over the shoal (2048×2, P=6, walls, relaxation zones of §2.2)
                    from rest: η, φ̃ at every 4th column after 1, 10, 25 and 50 RK4 steps.
  c5_big_tank.npz   The 192 k-node periodic request of the C5 stream at 100 req/s (5352×2, P=4):
                    η, φ̃ at every 4th column after one RK4 step from its initial state.
Each step of the 50-step C4 window takes about a minute of oracle time (four banded-Cholesky
solves of 147 k unknowns), so the C4 file takes most of an hour to write.
"""
from __future__ import annotations

import os
import sys
import time

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(os.path.dirname(HERE))
sys.path.insert(0, ROOT)

from oracle import sem as osem  # noqa: E402
from sem_workloads import c2_steep_periodic, c4_shoal, c5_requests, initial_state  # noqa: E402

STRIDE = 4   # column stride of the sampled checkpoints of the large tanks


def c2_window(path):
    wl = c2_steep_periodic()
    om = osem.mesh_for(wl)
    e, p = initial_state(wl, om.xcol, om.h)
    keep = (1, 25, 50, 75)
    out = {"steps": np.array(keep), "diag_steps": np.arange(0, 76, 5)}
    mass, energy = [om.mass(e)], [om.energy(e, p)]
    t0 = time.time()
    for s in range(1, 76):
        e, p = om.rk4_step(e, p, wl.dt)
        if s in keep:
            out[f"eta_{s}"] = e.copy()
            out[f"phis_{s}"] = p.copy()
        if s % 5 == 0:
            mass.append(om.mass(e))
            energy.append(om.energy(e, p))
            print(f"c2 step {s}: mass {mass[-1]:.16e} energy {energy[-1]:.16e} ({time.time() - t0:.0f} s)",
                  flush=True)
    out["mass"] = np.array(mass)
    out["energy"] = np.array(energy)
    # the wave goes on steepening until its state is no longer finite, the depth no longer positive
    # or the σ-transformed Laplace matrix no longer definite: the first step that fails
    s, fail = 75, 0
    while s < 400 and not fail:
        try:
            e, p = om.rk4_step(e, p, wl.dt)
            s += 1
            if not np.all(np.isfinite(e)) or np.any(e + om.h <= 0):
                fail = s
        except np.linalg.LinAlgError:
            fail = s + 1
    out["fail_step"] = np.array(fail)
    print(f"c2: oracle fails at step {fail}", flush=True)
    np.savez_compressed(path, **out)


def c4_window(path):
    wl = c4_shoal()
    om = osem.mesh_for(wl)
    e, p = initial_state(wl, om.xcol, om.h)
    keep = (1, 10, 25, 50)
    out = {"steps": np.array(keep), "stride": np.array(STRIDE)}
    t, t0 = 0.0, time.time()
    for s in range(1, 51):
        e, p = om.rk4_step(e, p, wl.dt, t)
        t += wl.dt
        if s in keep:
            out[f"eta_{s}"] = e[::STRIDE].copy()
            out[f"phis_{s}"] = p[::STRIDE].copy()
        print(f"c4 step {s}: max|eta| {np.abs(e).max():.6e} ({time.time() - t0:.0f} s)", flush=True)
    np.savez_compressed(path, **out)


def c5_big_tank(path):
    wl = c5_requests(100.0, 300, 0)[91][2]
    om = osem.mesh_for(wl)
    e, p = initial_state(wl, om.xcol, om.h)
    e, p = om.rk4_step(e, p, wl.dt)
    np.savez_compressed(path, stride=np.array(STRIDE), eta_1=e[::STRIDE].copy(), phis_1=p[::STRIDE].copy())


def main():
    which = sys.argv[1:] or ["c2", "c4", "c5big"]
    jobs = {"c2": (c2_window, "c2_window.npz"), "c4": (c4_window, "c4_window.npz"),
            "c5big": (c5_big_tank, "c5_big_tank.npz")}
    for name in which:
        fn, fname = jobs[name]
        t0 = time.time()
        fn(os.path.join(HERE, fname))
        print(f"{fname}: {time.time() - t0:.0f} s", flush=True)


if __name__ == "__main__":
    main()
