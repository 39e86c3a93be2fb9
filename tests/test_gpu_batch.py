"""Fused RK stage and batched instances on the GPU.

* The fused per-stage kernel (one cooperative launch per RK stage) gives the same steps as
  the multi-kernel path (SEM_FUSED_STAGE=0) and as the oracle.
* A batch of uneven instances (different orders, element counts, layers, ends, relaxation,
  precision) stepped together equals each instance stepped alone, within the stated
  tolerances (1e-10 FP64, 1e-8 mixed), and an FP64 member equals the oracle; with the plan the
  batch estimates faster, with cluster teams (SEM_BATCH_CLUSTER=1) and with cooperative launches
  (SEM_BATCH_CLUSTER=0), and with either build of the stage kernel for the batch's groups
  (SEM_BATCH_WIDE) or the default choice by group size.
"""
import math
import os

import numpy as np
import pytest

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():
    pytest.skip("needs a CUDA GPU", allow_module_level=True)

import paper_1512_02548_gb300 as sem  # noqa: E402
from oracle import sem as osem  # noqa: E402
from sem_workloads import Workload, small_case, c3_instances, initial_state  # noqa: E402

pytestmark = pytest.mark.gpu
DEV = torch.device("cuda:0")


def T(x):
    return torch.tensor(np.ascontiguousarray(x), dtype=torch.float64, device=DEV)


def rel(a, b):
    a = a.detach().cpu().numpy() if hasattr(a, "detach") else np.asarray(a)
    b = b.detach().cpu().numpy() if hasattr(b, "detach") else np.asarray(b)
    return np.linalg.norm(a - b) / max(np.linalg.norm(b), 1e-300)


def state(wl, om, seed):
    x = om.xcol
    rng = np.random.default_rng(seed)
    ph = rng.uniform(0, 2 * np.pi, 2)
    if wl.periodic:
        k = 2 * np.pi / wl.length
        return 0.03 * np.cos(k * x + ph[0]), 0.2 * np.sin(k * x + ph[1])
    return 0.02 * np.cos(np.pi * x / x[-1]) + 0.005, 0.1 * np.cos(np.pi * x / x[-1])


def mesh_for(wl, om, precision="fp64"):
    return sem.Mesh.from_workload(wl, h=om.h, precision=precision, tol=1e-13 if precision == "fp64" else 1e-12)


def test_fused_stage_equals_multikernel_path():
    wl = small_case(P=5, Nx=9, Nz=2)
    om = osem.mesh_for(wl)
    e0, p0 = state(wl, om, 1)
    fused = mesh_for(wl, om)
    old = os.environ.get("SEM_FUSED_STAGE")
    os.environ["SEM_FUSED_STAGE"] = "0"
    try:
        multi = mesh_for(wl, om)
    finally:
        if old is None:
            del os.environ["SEM_FUSED_STAGE"]
        else:
            os.environ["SEM_FUSED_STAGE"] = old
    ea, pa = T(e0), T(p0)
    eb, pb = T(e0), T(p0)
    fused.rk4_step(ea, pa, wl.dt, 3)
    multi.rk4_step(eb, pb, wl.dt, 3)
    assert rel(ea, eb) < 1e-12 and rel(pa, pb) < 1e-12
    e, p = e0, p0
    for _ in range(3):
        e, p = om.rk4_step(e, p, wl.dt)
    assert rel(ea, e) < 1e-10 and rel(pa, p) < 1e-10


def _uneven_instances():
    wave = (np.array([0.015]), np.array([2.9]), np.array([0.86]), np.array([0.4]))
    cases = [
        (small_case(P=3, Nx=12, Nz=1), "fp64"),
        (small_case(P=4, Nx=7, Nz=2, periodic=False), "fp64"),
        (small_case(P=5, Nx=9, Nz=2), "fp64"),
        (small_case(P=6, Nx=5, Nz=3), "fp64"),
        (small_case(P=4, Nx=20, Nz=1), "mixed"),
        (small_case(P=6, Nx=6, Nz=2), "mixed"),
        (Workload(name="zones", P=5, Nx=10, Nz=2, length=4 * math.pi, periodic=False, depth=1.0, Pf=8,
                  filter_alpha=36.0, filter_s=12.0, filter_ic=4, dt=0.04, init="rest", bathymetry="bar",
                  relax_left=2.5, relax_right=3.0, wave=wave), "fp64"),
        (small_case(P=3, Nx=31, Nz=2), "fp64"),
    ]
    return cases


BUILDS = {
    "plan-by-estimate": {},
    "clusters-build-by-size": {"SEM_BATCH_CLUSTER": "1"},
    "clusters-one-cta-per-sm": {"SEM_BATCH_CLUSTER": "1", "SEM_BATCH_WIDE": "0"},
    "clusters-two-ctas-per-sm": {"SEM_BATCH_CLUSTER": "1", "SEM_BATCH_WIDE": "1"},
    "cooperative-build-by-size": {"SEM_BATCH_CLUSTER": "0"},
    "cooperative-two-ctas-per-sm": {"SEM_BATCH_CLUSTER": "0", "SEM_BATCH_WIDE": "1"},
}


@pytest.fixture(params=list(BUILDS), ids=list(BUILDS))
def batch_build(request):
    """SEM_BATCH_CLUSTER (cluster teams on streams, or one cooperative launch per stage and
    group) and SEM_BATCH_WIDE (build of the stage kernel) for the batches created in the test;
    both are read by sem_batch_create."""
    names = ("SEM_BATCH_WIDE", "SEM_BATCH_CLUSTER")
    old = {k: os.environ.get(k) for k in names}
    for k in names:
        os.environ.pop(k, None)
    os.environ.update(BUILDS[request.param])
    yield request.param
    for k, v in old.items():
        if v is None:
            os.environ.pop(k, None)
        else:
            os.environ[k] = v


def test_batch_equals_instances_alone(batch_build):
    cases = _uneven_instances()
    oms = [osem.mesh_for(wl) for wl, _ in cases]
    states = [state(wl, om, i) for i, ((wl, _), om) in enumerate(zip(cases, oms))]
    # alone
    alone = []
    for (wl, prec), om, (e0, p0) in zip(cases, oms, states):
        m = mesh_for(wl, om, prec)
        e, p = T(e0), T(p0)
        m.rk4_step(e, p, wl.dt, 2, t=0.25)
        alone.append((e, p))
        m.close()
    # together
    meshes = [mesh_for(wl, om, prec) for (wl, prec), om in zip(cases, oms)]
    batch = sem.Batch(meshes)
    assert batch.info()["launches_per_stage"] >= 4
    etas = [T(e0) for e0, _ in states]
    phis = [T(p0) for _, p0 in states]
    ts = batch.rk4_step(etas, phis, [wl.dt for wl, _ in cases], 2, ts=[0.25] * len(cases))
    for k, ((wl, prec), (ea, pa)) in enumerate(zip(cases, alone)):
        tol = 1e-10 if prec == "fp64" else 1e-8
        assert rel(etas[k], ea) < tol and rel(phis[k], pa) < tol, (k, wl.name)
        assert ts[k] == pytest.approx(0.25 + 2 * wl.dt)
    # an FP64 member against the oracle
    wl, _ = cases[2]
    e, p = states[2]
    for s in range(2):
        e, p = oms[2].rk4_step(e, p, wl.dt, t=0.25 + s * wl.dt)
    assert rel(etas[2], e) < 1e-10 and rel(phis[2], p) < 1e-10
    batch.close()


@pytest.mark.slow
def test_c3_batch_runs_and_matches_alone_on_a_sample():
    wls = c3_instances(64)
    meshes, etas, phis, dts = [], [], [], []
    for i, wl in enumerate(wls):
        m = sem.Mesh.from_workload(wl, precision="mixed", tol=1e-12)
        om = osem.mesh_for(wl)
        e0, p0 = initial_state(wl, om.xcol, om.h)
        meshes.append(m)
        etas.append(T(e0))
        phis.append(T(p0))
        dts.append(wl.dt)
    batch = sem.Batch(meshes)
    ref = [(e.clone(), p.clone()) for e, p in zip(etas, phis)]
    batch.rk4_step(etas, phis, dts, 1)
    for k in (0, 17, 63):
        m2 = sem.Mesh.from_workload(wls[k], precision="mixed", tol=1e-12)
        e, p = ref[k]
        m2.rk4_step(e, p, dts[k], 1)
        assert rel(etas[k], e) < 1e-8 and rel(phis[k], p) < 1e-8
    batch.close()


def test_batch_laplace_solve_equals_alone_and_oracle():
    cases = _uneven_instances()
    oms = [osem.mesh_for(wl) for wl, _ in cases]
    states = [state(wl, om, 10 + i) for i, ((wl, _), om) in enumerate(zip(cases, oms))]
    meshes = [mesh_for(wl, om, prec) for (wl, prec), om in zip(cases, oms)]
    batch = sem.Batch(meshes)
    Phis = [torch.zeros(om.n, dtype=torch.float64, device=DEV) for om in oms]
    batch.laplace_solve([T(e) for e, _ in states], [T(p) for _, p in states], Phis)
    assert batch.status() == [0] * len(cases)
    for k, ((wl, prec), om, (e0, p0)) in enumerate(zip(cases, oms, states)):
        tol = 1e-10 if prec == "fp64" else 1e-8
        m = mesh_for(wl, om, prec)
        m.update_geometry(T(e0))
        Phi = torch.zeros(om.n, dtype=torch.float64, device=DEV)
        m.laplace_solve(T(p0), Phi)
        m.close()
        assert rel(Phis[k], Phi) < tol, (k, wl.name)
        assert rel(Phis[k], om.laplace_solve(e0, p0)) < tol, (k, wl.name)
    # the batched solve leaves each mesh's geometry at the given surface: a recovery call
    # that follows sees the same σ-geometry as after sem_update_geometry
    wl, _ = cases[2]
    om, (e0, p0) = oms[2], states[2]
    w, ex, px = (torch.zeros(om.ncol, dtype=torch.float64, device=DEV) for _ in range(3))
    meshes[2].recover_gradient(Phis[2], T(e0), T(p0), w, ex, px)
    assert rel(w, om.w_surface(e0, om.laplace_solve(e0, p0))) < 1e-10
    batch.close()


def test_batch_failure_stays_with_its_instance():
    """A non-finite surface in one instance fails that instance only; the others are
    stepped exactly as without it."""
    cases = _uneven_instances()[:4]
    oms = [osem.mesh_for(wl) for wl, _ in cases]
    states = [state(wl, om, 20 + i) for i, ((wl, _), om) in enumerate(zip(cases, oms))]
    bad = 1
    meshes = [mesh_for(wl, om, prec) for (wl, prec), om in zip(cases, oms)]
    batch = sem.Batch(meshes)
    etas = [T(e) for e, _ in states]
    phis = [T(p) for _, p in states]
    etas[bad][3] = float("nan")
    with pytest.raises(sem.SemError) as ei:
        batch.rk4_step(etas, phis, [wl.dt for wl, _ in cases], 1)
    assert ei.value.code == sem.SEM_ERR_NONFINITE and f"instance {bad}" in str(ei.value)
    codes = batch.status()
    assert codes[bad] == sem.SEM_ERR_NONFINITE
    assert all(c == 0 for k, c in enumerate(codes) if k != bad)
    for k, ((wl, prec), om, (e0, p0)) in enumerate(zip(cases, oms, states)):
        if k == bad:
            continue
        e, p = om.rk4_step(e0, p0, wl.dt)
        assert rel(etas[k], e) < 1e-10 and rel(phis[k], p) < 1e-10, k
    # the failed instance's mesh is usable again afterwards
    e0, p0 = states[bad]
    ea, pa = T(e0), T(p0)
    batch.rk4_step([T(s[0]) if k != bad else ea for k, s in enumerate(states)],
                   [T(s[1]) if k != bad else pa for k, s in enumerate(states)],
                   [wl.dt for wl, _ in cases], 1)
    assert batch.status() == [0] * len(cases)
    e, p = oms[bad].rk4_step(e0, p0, cases[bad][0].dt)
    assert rel(ea, e) < 1e-10 and rel(pa, p) < 1e-10
    batch.close()
