"""Parity windows of the full-size runs against stored oracle trajectories.

The oracle's trajectories are written by ``tests/golden/make_long_run_golden.py``, which calls
only the CPU oracle: the C2 steep wave over its first 75 RK4 steps (full state at steps 1, 25,
50 and 75) and the step at which the oracle's run fails (the wave, started from linear theory
at H/L = 0.08, steepens until its state is no longer regular, about half a period in), the C4
shoal from rest over its first 50 steps (every 4th column at steps 1, 10, 25 and 50) and one
step of the 192 k-node periodic tank of the C5 stream.  The GPU runs the same steps through the
C ABI, in FP64 and in mixed precision, and each checkpoint must agree with the oracle in
relative L² within 1e-10 (FP64) and 1e-8 (mixed); the GPU run of C2 must fail, reporting a
non-finite state or a non-positive depth, within a few steps of the oracle's.
"""
import os

import numpy as np
import pytest

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():
    pytest.skip("needs a CUDA GPU", allow_module_level=True)

import paper_1512_02548_gb300 as sem  # noqa: E402
from oracle import sem as osem  # noqa: E402
from sem_workloads import c2_steep_periodic, c4_shoal, c5_requests, initial_state  # noqa: E402

pytestmark = [pytest.mark.gpu, pytest.mark.slow]
DEV = torch.device("cuda:0")
GOLDEN = os.path.join(os.path.dirname(os.path.abspath(__file__)), "golden")
TOLS = {"fp64": 1e-10, "mixed": 1e-8}


def T(x):
    return torch.tensor(np.ascontiguousarray(x), dtype=torch.float64, device=DEV)


def rel(a, b):
    return float(np.linalg.norm(a - b) / np.linalg.norm(b))


def golden(name):
    path = os.path.join(GOLDEN, name)
    if not os.path.exists(path):
        pytest.fail(f"{name} is missing: run tests/golden/make_long_run_golden.py")
    return np.load(path)


@pytest.mark.parametrize("precision", ["fp64", "mixed"])
def test_c2_window_matches_the_oracle_and_fails_where_it_fails(precision):
    g = golden("c2_window.npz")
    wl = c2_steep_periodic()
    om = osem.mesh_for(wl)
    gm = sem.Mesh.from_workload(wl, h=om.h, precision=precision)
    e0, p0 = initial_state(wl, om.xcol, om.h)
    eta, phis = T(e0), T(p0)
    done = 0
    for s in g["steps"]:
        gm.rk4_step(eta, phis, wl.dt, int(s) - done)
        done = int(s)
        err = max(rel(eta.cpu().numpy(), g[f"eta_{s}"]), rel(phis.cpu().numpy(), g[f"phis_{s}"]))
        assert err < TOLS[precision], (precision, int(s), err)
    fail = int(g["fail_step"])
    assert fail > done
    failed_at = None
    while done < fail + 10:
        try:
            gm.rk4_step(eta, phis, wl.dt, 1)
        except sem.SemError as ex:
            assert ex.code in (sem.SEM_ERR_NONFINITE, sem.SEM_ERR_NOT_CONVERGED), ex
            failed_at = done + 1
            break
        done += 1
    assert failed_at is not None and abs(failed_at - fail) <= 3, (failed_at, fail)
    gm.close()


@pytest.mark.parametrize("precision", ["fp64", "mixed"])
def test_c4_first_50_steps_match_the_oracle(precision):
    g = golden("c4_window.npz")
    k = int(g["stride"])
    wl = c4_shoal()
    om = osem.mesh_for(wl)
    gm = sem.Mesh.from_workload(wl, h=om.h, precision=precision)
    eta = torch.zeros(wl.ncol, dtype=torch.float64, device=DEV)
    phis = torch.zeros_like(eta)
    done, t = 0, 0.0
    for s in g["steps"]:
        t = gm.rk4_step(eta, phis, wl.dt, int(s) - done, t=t)
        done = int(s)
        err = max(rel(eta.cpu().numpy()[::k], g[f"eta_{s}"]), rel(phis.cpu().numpy()[::k], g[f"phis_{s}"]))
        assert err < TOLS[precision], (precision, int(s), err)
    gm.close()


@pytest.mark.parametrize("precision", ["fp64", "mixed"])
def test_c5_largest_periodic_tank_one_step_matches_the_oracle(precision):
    g = golden("c5_big_tank.npz")
    k = int(g["stride"])
    wl = c5_requests(100.0, 300, 0)[91][2]
    assert (wl.P, wl.Nx, wl.Nz, wl.periodic) == (4, 5352, 2, True)
    om = osem.mesh_for(wl)
    e0, p0 = initial_state(wl, om.xcol, om.h)
    gm = sem.Mesh.from_workload(wl, h=om.h, precision=precision)
    eta, phis = T(e0), T(p0)
    gm.rk4_step(eta, phis, wl.dt, 1)
    err = max(rel(eta.cpu().numpy()[::k], g["eta_1"]), rel(phis.cpu().numpy()[::k], g["phis_1"]))
    assert err < TOLS[precision], (precision, err)
    gm.close()
