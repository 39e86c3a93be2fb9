"""Bounded team barriers: a CTA that never arrives turns into SEM_ERR_TIMEOUT, not a hang.

The library's Krylov and fused stage kernels synchronise the CTAs of a team with barriers
whose waits are limited in wall-clock time; a wait that runs out sets the team's status word
and every CTA returns.  The testing hook sem_set_barrier_test shortens that limit to a few
milliseconds and makes one CTA of the team return before its first barrier, so the others'
waits run out.  No GPU fault, trap or endless wait is involved: every CTA ends its launch.
The tests check the error code, that it comes back within milliseconds rather than seconds,
that one failing member of a batch leaves the others' results alone, and that the mesh solves
normally once the hook is off.
"""
import time

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
TOL_FP64 = 1e-10
LIMIT_MS = 5.0


def T(x):
    return torch.tensor(np.ascontiguousarray(x), dtype=torch.float64, device=DEV)


def rel(a, b):
    a = a.detach().cpu().numpy() if hasattr(a, "detach") else np.asarray(a)
    return np.linalg.norm(a - b) / np.linalg.norm(b)


def surface(om):
    x = om.xcol
    return 0.05 * np.cos(x) + 0.01 * np.sin(2 * x), 0.3 * np.sin(x) + 0.05 * np.cos(3 * x)


def tank():
    wl = small_case(P=4, Nx=64, Nz=2)
    om = osem.mesh_for(wl)
    gm = sem.Mesh.from_workload(wl, h=om.h)
    assert gm.info.grid_ctas >= 2 and gm.info.stage_ctas >= 2   # a team with barriers to miss
    return wl, om, gm


def test_missing_cta_times_out_in_the_solve_and_the_mesh_recovers():
    wl, om, gm = tank()
    eta0, phis0 = surface(om)
    gm.update_geometry(T(eta0))
    Phi = torch.zeros(om.n, dtype=torch.float64, device=DEV)
    gm.set_barrier_test(drop_rank=1, timeout_ms=LIMIT_MS)
    t0 = time.perf_counter()
    with pytest.raises(sem.SemError) as ei:
        gm.laplace_solve(T(phis0), Phi)
    elapsed = time.perf_counter() - t0
    assert ei.value.code == sem.SEM_ERR_TIMEOUT
    assert elapsed < 0.5, elapsed            # the 5 ms limit, not the default 2 s
    gm.set_barrier_test(-1, 0.0)
    Phi.zero_()
    st = gm.laplace_solve(T(phis0), Phi)
    assert st.rel_residual <= 1e-13
    Phi_ref = om.laplace_solve(eta0, phis0)
    assert rel(Phi, Phi_ref) < TOL_FP64


def test_missing_cta_times_out_in_the_fused_stage_and_the_mesh_recovers():
    wl, om, gm = tank()
    eta0, phis0 = surface(om)
    eta, phis = T(eta0), T(phis0)
    gm.set_barrier_test(drop_rank=gm.info.stage_ctas - 1, timeout_ms=LIMIT_MS)
    t0 = time.perf_counter()
    with pytest.raises(sem.SemError) as ei:
        gm.rk4_step(eta, phis, wl.dt, 1)
    assert ei.value.code == sem.SEM_ERR_TIMEOUT
    assert time.perf_counter() - t0 < 0.5
    gm.set_barrier_test(-1, 0.0)
    eta, phis = T(eta0), T(phis0)
    gm.rk4_step(eta, phis, wl.dt, 1)
    e, p = om.rk4_step(eta0, phis0, wl.dt)
    assert rel(eta, e) < TOL_FP64 and rel(phis, p) < TOL_FP64


def test_timeout_stays_with_its_batch_member():
    wl, om, gm_bad = tank()
    gm_ok = sem.Mesh.from_workload(wl, h=om.h)
    batch = sem.Batch([gm_bad, gm_ok])
    eta0, phis0 = surface(om)
    etas, phises = [T(eta0), T(eta0)], [T(phis0), T(phis0)]
    gm_bad.set_barrier_test(drop_rank=0, timeout_ms=LIMIT_MS)
    with pytest.raises(sem.SemError) as ei:
        batch.rk4_step(etas, phises, [wl.dt, wl.dt], 1)
    assert ei.value.code == sem.SEM_ERR_TIMEOUT
    assert batch.status() == [sem.SEM_ERR_TIMEOUT, sem.SEM_OK]
    e, p = om.rk4_step(eta0, phis0, wl.dt)
    assert rel(etas[1], e) < TOL_FP64 and rel(phises[1], p) < TOL_FP64
    gm_bad.set_barrier_test(-1, 0.0)
    etas[0], phises[0] = T(eta0), T(phis0)
    batch.rk4_step(etas[:1] + [T(eta0)], phises[:1] + [T(phis0)], [wl.dt, wl.dt], 1)
    assert batch.status() == [sem.SEM_OK, sem.SEM_OK]
    assert rel(etas[0], e) < TOL_FP64 and rel(phises[0], p) < TOL_FP64
    batch.close()


def test_hook_rejects_bad_arguments():
    wl, om, gm = tank()
    with pytest.raises(sem.SemError):
        gm.set_barrier_test(-2, 0.0)
    with pytest.raises(sem.SemError):
        gm.set_barrier_test(1, 5000.0)
