"""Initial guesses of the fused RK stage from earlier stage potentials.

Stages 2, 3 and 4 start their Laplace solves from extrapolations of kept stage potentials; stages 2
and 3 use the last step's, but only when the call continues the last fused call's trajectory (the
same state buffers and dt).  The guesses change the starting point only, so:
  * N steps in one call and N calls of one step give the same result (1e-12 apart; both within
    1e-10 of the oracle) and, with the history carried across calls, about the same iterations;
  * new data written into the same buffers (a history that no longer fits) still converges to the
    oracle's step, at the usual 1e-10;
  * a failed step (non-finite surface) clears the history, so the next step of a valid state is
    not started from non-finite guesses.
"""
import numpy as np
import pytest

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():
    pytest.skip("needs a CUDA GPU", allow_module_level=True)

import paper_1512_02548_gb300 as sem  # noqa: E402
from oracle import sem as osem  # noqa: E402
from sem_workloads import small_case  # noqa: E402

pytestmark = pytest.mark.gpu
DEV = torch.device("cuda:0")


def rel(a, b):
    a = a.detach().cpu().numpy() if hasattr(a, "detach") else np.asarray(a)
    return np.linalg.norm(a - b) / max(np.linalg.norm(b), 1e-300)


def T(x):
    return torch.tensor(np.ascontiguousarray(x), dtype=torch.float64, device=DEV)


def setup(P=5, Nx=7, Nz=2, periodic=True, precision="fp64"):
    wl = small_case(P=P, Nx=Nx, Nz=Nz, periodic=periodic)
    om = osem.mesh_for(wl)
    gm = sem.Mesh.from_workload(wl, h=om.h, precision=precision, tol=1e-13 if precision == "fp64" else 1e-12)
    x = om.xcol
    eta = 0.08 * np.cos(2 * np.pi * x / wl.length) + 0.02 * np.sin(4 * np.pi * x / wl.length)
    phis = 0.3 * np.sin(2 * np.pi * x / wl.length)
    return wl, om, gm, eta, phis


def oracle_steps(om, e, p, dt, n):
    for _ in range(n):
        e, p = om.rk4_step(e, p, dt)
    return e, p


@pytest.mark.parametrize("precision", ["fp64", "mixed"])
def test_one_call_equals_separate_calls(precision):
    wl, om, gm, e0, p0 = setup(precision=precision)
    _, _, gm2, _, _ = setup(precision=precision)
    n = 4
    ea, pa = T(e0), T(p0)
    gm.reset_counters()
    gm.rk4_step(ea, pa, wl.dt, n)
    ca = gm.counters()
    eb, pb = T(e0), T(p0)
    gm2.reset_counters()
    for _ in range(n):
        gm2.rk4_step(eb, pb, wl.dt, 1)
    cb = gm2.counters()
    assert rel(eb, ea.cpu().numpy()) < 1e-12 and rel(pb, pa.cpu().numpy()) < 1e-12
    e, p = oracle_steps(om, e0, p0, wl.dt, n)
    tol = 1e-10 if precision == "fp64" else 1e-8
    assert rel(ea, e) < tol and rel(pa, p) < tol
    # the separate calls carried the history: no more iterations than one call, up to rounding
    assert ca.solves == cb.solves == 4 * n
    assert abs(cb.iterations - ca.iterations) <= 2


def test_history_that_no_longer_fits_still_converges():
    wl, om, gm, e0, p0 = setup(P=6, Nx=5, Nz=2, periodic=False)
    eta, phis = T(e0), T(p0)
    gm.rk4_step(eta, phis, wl.dt, 3)
    # other data in the same buffers, same dt: the kept potentials belong to another trajectory
    e1 = 0.05 * np.cos(np.pi * om.xcol / om.xcol[-1]) + 0.01
    p1 = -0.2 * np.cos(2 * np.pi * om.xcol / om.xcol[-1])
    eta.copy_(T(e1))
    phis.copy_(T(p1))
    gm.rk4_step(eta, phis, wl.dt, 2)
    e, p = oracle_steps(om, e1, p1, wl.dt, 2)
    assert rel(eta, e) < 1e-10 and rel(phis, p) < 1e-10


def test_failed_step_clears_history():
    wl, om, gm, e0, p0 = setup()
    eta, phis = T(e0), T(p0)
    gm.rk4_step(eta, phis, wl.dt, 2)
    bad = e0.copy()
    bad[2] = np.nan
    eta.copy_(T(bad))
    with pytest.raises(sem.SemError) as ei:
        gm.rk4_step(eta, phis, wl.dt, 1)
    assert ei.value.code in (4, 5)
    # a valid state in the same buffers, same dt: steps from scratch and matches the oracle
    eta.copy_(T(e0))
    phis.copy_(T(p0))
    gm.rk4_step(eta, phis, wl.dt, 2)
    e, p = oracle_steps(om, e0, p0, wl.dt, 2)
    assert rel(eta, e) < 1e-10 and rel(phis, p) < 1e-10
