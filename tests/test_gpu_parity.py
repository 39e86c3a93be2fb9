"""GPU parity: the CUDA path through the C ABI against the CPU oracle.

Tolerances (relative L² over canonical-order nodes):
  * index maps: bit-exact;
  * single operator applies, recovery, filter: 1e-12 (FP64 rounding of a few
    hundred terms);
  * Laplace solves, right-hand sides and RK4 steps, FP64 path: 1e-10 (stated
    target; the Krylov tolerance is 1e-13 relative residual);
  * mixed precision (FP32 inner, FP64 refinement): 1e-8.
Cases span several element columns per CTA (SEM_GRID_LIMIT forces uneven
chunks), walls and periodic ends, 1–3 layers, P from 2 to 12, variable depth,
and the degenerate φ̃ ≡ 0 surface.
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
from sem_workloads import (small_case, c1_linear_standing, c2_steep_periodic, initial_state,  # noqa: E402
                           random_field)

pytestmark = pytest.mark.gpu
DEV = torch.device("cuda:0")
TOL_OP = 1e-12
TOL_FP64 = 1e-10
TOL_MIXED = 1e-8


def rel(a, b):
    a = a.detach().cpu().numpy() if hasattr(a, "detach") else np.asarray(a)
    return np.linalg.norm(a - b) / max(np.linalg.norm(b), 1e-300)


def T(x):
    return torch.tensor(np.ascontiguousarray(x), dtype=torch.float64, device=DEV)


def make_pair(P=5, Nx=7, Nz=2, periodic=True, bar=False, Pf=None, filt=True, precision="fp64",
              grid_limit=None, tol=1e-13, precond="separable"):
    wl = small_case(P=P, Nx=Nx, Nz=Nz, periodic=periodic, Pf=Pf, filt=filt)
    om = osem.mesh_for(wl, bar=bar)
    old = os.environ.get("SEM_GRID_LIMIT")
    if grid_limit:
        os.environ["SEM_GRID_LIMIT"] = str(grid_limit)
    try:
        gm = sem.Mesh.from_workload(wl, h=om.h, precision=precision, tol=tol, precond=precond)
    finally:
        if grid_limit:
            if old is None:
                del os.environ["SEM_GRID_LIMIT"]
            else:
                os.environ["SEM_GRID_LIMIT"] = old
    return wl, om, gm


def surface(om, seed=0, amp=0.08):
    x = om.xcol
    rng = np.random.default_rng(seed)
    ph = rng.uniform(0, 2 * np.pi, 3)
    eta = amp * np.cos(x + ph[0]) + 0.3 * amp * np.sin(2 * x + ph[1])
    phis = 0.4 * np.sin(x + ph[2]) + 0.1 * np.cos(3 * x)
    if not om.periodic:
        eta = amp * np.cos(np.pi * x / x[-1]) + 0.01
        phis = 0.3 * np.cos(np.pi * x / x[-1]) + 0.05 * np.cos(2 * np.pi * x / x[-1])
    return eta, phis


CASES = [
    dict(P=5, Nx=7, Nz=2),
    dict(P=2, Nx=9, Nz=3),
    dict(P=8, Nx=4, Nz=1),
    dict(P=6, Nx=5, Nz=2, periodic=False),
    dict(P=4, Nx=11, Nz=2, bar=True, grid_limit=3),
    dict(P=3, Nx=3, Nz=1, periodic=True),
    dict(P=12, Nx=3, Nz=1, periodic=False),
    dict(P=4, Nx=1, Nz=2, periodic=False),
]


@pytest.mark.parametrize("case", CASES, ids=lambda c: "-".join(f"{k}{v}" for k, v in c.items()))
def test_l2g_bit_exact(case):
    wl, om, gm = make_pair(**case)
    out = torch.empty(om.l2g.size, dtype=torch.int32, device=DEV)
    gm.l2g(out)
    assert np.array_equal(out.cpu().numpy(), om.l2g.ravel().astype(np.int32))


@pytest.mark.parametrize("case", CASES, ids=lambda c: "-".join(f"{k}{v}" for k, v in c.items()))
def test_apply_matches_assembled_operator(case):
    wl, om, gm = make_pair(**case)
    eta, _ = surface(om)
    x = random_field(om.n, 11)
    gm.update_geometry(T(eta))
    y = torch.empty(om.n, dtype=torch.float64, device=DEV)
    gm.laplace_apply(T(x), y)
    ref = om.stiffness(eta) @ x
    assert rel(y, ref) < TOL_OP


@pytest.mark.parametrize("case", CASES, ids=lambda c: "-".join(f"{k}{v}" for k, v in c.items()))
def test_laplace_solve_matches_banded_direct(case):
    wl, om, gm = make_pair(**case)
    eta, phis = surface(om, seed=1)
    gm.update_geometry(T(eta))
    Phi = torch.zeros(om.n, dtype=torch.float64, device=DEV)
    st = gm.laplace_solve(T(phis), Phi)
    ref = om.laplace_solve(eta, phis)
    assert st.rel_residual <= 1e-13
    assert rel(Phi, ref) < TOL_FP64
    # warm start from the solution: converges at once to the same answer
    st2 = gm.laplace_solve(T(phis), Phi)
    assert st2.iterations <= 2 and rel(Phi, ref) < TOL_FP64


@pytest.mark.parametrize("case", CASES[:6], ids=lambda c: "-".join(f"{k}{v}" for k, v in c.items()))
@pytest.mark.parametrize("precision", ["fp64", "mixed"])
def test_jacobi_preconditioner_solve(case, precision):
    wl, om, gm = make_pair(precond="jacobi", precision=precision, tol=1e-12 if precision == "mixed" else 1e-13,
                           **case)
    eta, phis = surface(om, seed=9)
    gm.update_geometry(T(eta))
    Phi = torch.zeros(om.n, dtype=torch.float64, device=DEV)
    gm.laplace_solve(T(phis), Phi)
    assert rel(Phi, om.laplace_solve(eta, phis)) < (TOL_MIXED if precision == "mixed" else TOL_FP64)


def test_separable_preconditioner_needs_few_iterations():
    # C2-sized tank: the σ-separable preconditioner converges in tens of iterations where
    # Jacobi needs hundreds
    wl = c2_steep_periodic()
    om = osem.mesh_for(wl)
    e, p = initial_state(wl, om.xcol, om.h)
    its = {}
    for pc in ("separable", "jacobi"):
        gm = sem.Mesh.from_workload(wl, h=om.h, precond=pc)
        gm.update_geometry(T(e))
        Phi = torch.zeros(om.n, dtype=torch.float64, device=DEV)
        its[pc] = gm.laplace_solve(T(p), Phi).iterations
    assert its["separable"] <= 30 and its["jacobi"] > 10 * its["separable"]


def test_laplace_solve_zero_surface_potential():
    wl, om, gm = make_pair(P=4, Nx=5, Nz=2)
    eta, _ = surface(om)
    gm.update_geometry(T(eta))
    Phi = T(random_field(om.n, 3))
    st = gm.laplace_solve(T(np.zeros(om.ncol)), Phi)
    assert st.iterations == 0 and float(Phi.abs().max()) == 0.0


def test_laplace_solve_is_deterministic():
    wl, om, gm = make_pair(P=6, Nx=9, Nz=2, grid_limit=4)
    eta, phis = surface(om, seed=2)
    gm.update_geometry(T(eta))
    a = torch.zeros(om.n, dtype=torch.float64, device=DEV)
    b = torch.zeros(om.n, dtype=torch.float64, device=DEV)
    gm.laplace_solve(T(phis), a)
    gm.laplace_solve(T(phis), b)
    assert torch.equal(a, b)


@pytest.mark.parametrize("case", CASES[:5], ids=lambda c: "-".join(f"{k}{v}" for k, v in c.items()))
def test_mixed_precision_solve(case):
    wl, om, gm = make_pair(precision="mixed", tol=1e-12, **case)
    eta, phis = surface(om, seed=4)
    gm.update_geometry(T(eta))
    Phi = torch.zeros(om.n, dtype=torch.float64, device=DEV)
    st = gm.laplace_solve(T(phis), Phi)
    assert st.rel_residual <= 1e-12 and st.refinements >= 1
    assert rel(Phi, om.laplace_solve(eta, phis)) < TOL_MIXED


@pytest.mark.parametrize("case", CASES, ids=lambda c: "-".join(f"{k}{v}" for k, v in c.items()))
def test_recovery_matches_projections(case):
    wl, om, gm = make_pair(**case)
    eta, phis = surface(om, seed=5)
    Phi = om.laplace_solve(eta, phis)
    w = torch.empty(om.ncol, dtype=torch.float64, device=DEV)
    ex = torch.empty_like(w)
    px = torch.empty_like(w)
    gm.recover_gradient(T(Phi), T(eta), T(phis), w, ex, px)
    assert rel(w, om.w_surface(eta, Phi)) < TOL_OP
    assert rel(ex, om.surface_gradient(eta)) < TOL_OP
    assert rel(px, om.surface_gradient(phis)) < TOL_OP


@pytest.mark.parametrize("case", CASES, ids=lambda c: "-".join(f"{k}{v}" for k, v in c.items()))
def test_zakharov_rhs(case):
    wl, om, gm = make_pair(**case)
    eta, phis = surface(om, seed=6)
    de = torch.empty(om.ncol, dtype=torch.float64, device=DEV)
    dp = torch.empty_like(de)
    gm.zakharov_rhs(T(eta), T(phis), de, dp)
    re, rp = om.zakharov_rhs(eta, phis)
    assert rel(de, re) < TOL_FP64 and rel(dp, rp) < TOL_FP64


@pytest.mark.parametrize("P", [3, 6, 10])
def test_filter(P):
    wl, om, gm = make_pair(P=P, Nx=5, Nz=1)
    q = random_field(om.ncol, P)
    qd = T(q)
    gm.apply_filter(qd)
    assert rel(qd, om.apply_filter(q)) < TOL_OP


@pytest.mark.parametrize("case", [dict(P=5, Nx=7, Nz=2), dict(P=6, Nx=5, Nz=2, periodic=False),
                                  dict(P=4, Nx=11, Nz=2, bar=True, grid_limit=3)],
                         ids=["periodic", "walls", "bar"])
def test_rk4_steps(case):
    wl, om, gm = make_pair(**case)
    eta0, phis0 = surface(om, seed=7)
    eta, phis = T(eta0), T(phis0)
    t = gm.rk4_step(eta, phis, wl.dt, 2)
    e, p = eta0, phis0
    for _ in range(2):
        e, p = om.rk4_step(e, p, wl.dt)
    assert t == pytest.approx(2 * wl.dt)
    assert rel(eta, e) < TOL_FP64 and rel(phis, p) < TOL_FP64


@pytest.mark.parametrize("Nx", [150, 1500])
@pytest.mark.parametrize("periodic", [True, False], ids=["periodic", "walls"])
def test_long_tank_interface_solves(periodic, Nx):
    """More than 128 interface unknowns: the preconditioner's and M''s interface systems are
    solved by a whole CTA (chunks over all its threads) instead of one warp.  Nx = 150 gives one
    value per thread; Nx = 1500 gives chunks of 6, which the single-mesh stage build keeps in
    registers between the passes of the solve."""
    import dataclasses
    # the tank grows with Nx, so that the elements keep the aspect ratio of the Nx = 150 case
    wl = dataclasses.replace(small_case(P=3, Nx=Nx, Nz=1, periodic=periodic), length=2 * math.pi * Nx / 150)
    om = osem.mesh_for(wl)
    gm = sem.Mesh.from_workload(wl, h=om.h)
    eta0, phis0 = surface(om, seed=11)
    eta, phis = T(eta0), T(phis0)
    gm.rk4_step(eta, phis, wl.dt, 2)
    e, p = eta0, phis0
    for _ in range(2):
        e, p = om.rk4_step(e, p, wl.dt)
    assert rel(eta, e) < TOL_FP64 and rel(phis, p) < TOL_FP64


@pytest.mark.slow
def test_long_periodic_tank_fused_equals_multikernel():
    """A 192 k-node periodic tank (5352×2, P=4; request 91 of the C5 stream): the fused stage
    (long-system paths) against the multi-kernel path, two RK4 steps, 1e-10, with every solve
    converging in a normal number of iterations.  Scanned interface pivots had made this tank's
    solves stall (its lowest σ-mode is nearly singular in x)."""
    from sem_workloads import c5_requests
    wl = c5_requests(100.0, 300, 0)[91][2]
    assert (wl.P, wl.Nx, wl.Nz, wl.periodic) == (4, 5352, 2, True)
    x = np.linspace(0.0, wl.length, wl.ncol, endpoint=False)
    h = np.full(wl.ncol, wl.depth)
    e0, p0 = initial_state(wl, x, h)
    res = []
    for fused in ("1", "0"):
        old = os.environ.get("SEM_FUSED_STAGE")
        os.environ["SEM_FUSED_STAGE"] = fused
        try:
            gm = sem.Mesh.from_workload(wl, h=h)
        finally:
            if old is None:
                del os.environ["SEM_FUSED_STAGE"]
            else:
                os.environ["SEM_FUSED_STAGE"] = old
        eta, phis = T(e0), T(p0)
        gm.reset_counters()
        gm.rk4_step(eta, phis, wl.dt, 2)
        c = gm.counters()
        assert c.iterations / c.solves < 20 and c.max_rel_residual <= 1e-13, (fused, c.iterations, c.solves)
        res.append((eta.cpu().numpy(), phis.cpu().numpy()))
        gm.close()
    assert rel(res[0][0], res[1][0]) < TOL_FP64 and rel(res[0][1], res[1][1]) < TOL_FP64


def test_c1_one_period_matches_oracle():
    wl = c1_linear_standing()
    om = osem.mesh_for(wl)
    gm = sem.Mesh.from_workload(wl, h=om.h)
    e, p = initial_state(wl, om.xcol, om.h)
    eta, phis = T(e), T(p)
    gm.rk4_step(eta, phis, wl.dt, wl.nsteps)
    for _ in range(wl.nsteps):
        e, p = om.rk4_step(e, p, wl.dt)
    assert rel(eta, e) < TOL_FP64 and rel(phis, p) < TOL_FP64


def test_host_buffer_step_equals_device_step():
    wl, om, gm = make_pair(P=5, Nx=7, Nz=2)
    e0, p0 = surface(om, seed=8)
    eta, phis = T(e0), T(p0)
    gm.rk4_step(eta, phis, wl.dt, 1)
    he, hp = e0.copy(), p0.copy()
    gm2 = sem.Mesh.from_workload(wl, h=om.h)
    gm2.rk4_step_host(he, hp, wl.dt, 1)
    assert np.array_equal(eta.cpu().numpy(), he) and np.array_equal(phis.cpu().numpy(), hp)


@pytest.mark.slow
def test_c2_full_size_two_steps():
    wl = c2_steep_periodic()
    om = osem.mesh_for(wl)
    gm = sem.Mesh.from_workload(wl, h=om.h)
    e, p = initial_state(wl, om.xcol, om.h)
    eta, phis = T(e), T(p)
    gm.rk4_step(eta, phis, wl.dt, 2)
    for _ in range(2):
        e, p = om.rk4_step(e, p, wl.dt)
    assert rel(eta, e) < TOL_FP64 and rel(phis, p) < TOL_FP64


def test_errors_are_reported():
    wl, om, gm = make_pair(P=4, Nx=5, Nz=2)
    eta, phis = surface(om)
    # negative depth
    gm.update_geometry(T(eta - 5.0))
    Phi = torch.zeros(om.n, dtype=torch.float64, device=DEV)
    with pytest.raises(sem.SemError) as ei:
        gm.laplace_solve(T(phis), Phi)
    assert ei.value.code in (4, 5)
    # iteration cap
    wl2 = small_case(P=6, Nx=8, Nz=2)
    gm2 = sem.Mesh.from_workload(wl2, h=osem.mesh_for(wl2).h, max_iter=3)
    om2 = osem.mesh_for(wl2)
    e2, p2 = surface(om2)
    gm2.update_geometry(T(e2))
    with pytest.raises(sem.SemError) as ei:
        gm2.laplace_solve(T(p2), torch.zeros(om2.n, dtype=torch.float64, device=DEV))
    assert ei.value.code == 4
    # NaN in the surface potential
    gm.update_geometry(T(eta))
    bad = phis.copy()
    bad[3] = np.nan
    with pytest.raises(sem.SemError) as ei:
        gm.laplace_solve(T(bad), Phi)
    assert ei.value.code in (4, 5)
    # the mesh stays usable afterwards
    st = gm.laplace_solve(T(phis), torch.zeros(om.n, dtype=torch.float64, device=DEV))
    assert st.rel_residual <= 1e-13


def test_counters_and_launch_count():
    wl, om, gm = make_pair(P=4, Nx=5, Nz=1)
    eta, phis = surface(om)
    gm.reset_counters()
    n0 = sem.launch_count()
    gm.rk4_step(T(eta), T(phis), wl.dt, 1)
    c = gm.counters()
    assert c.solves == 4 and c.iterations > 0 and c.max_rel_residual <= 1e-13
    # the fused path: one cooperative launch per RK stage
    assert sem.launch_count() - n0 == 4


def _zone_pair(precision="fp64"):
    from sem_workloads import Workload
    wave = (np.array([0.02, 0.01]), np.array([2.7, 3.4]), np.array([0.77, 1.19]), np.array([0.1, 2.0]))
    wl = Workload(name="zones", P=5, Nx=10, Nz=2, length=4 * math.pi, periodic=False, depth=1.0, Pf=8,
                  filter_alpha=36.0, filter_s=12.0, filter_ic=4, dt=0.04, init="rest", bathymetry="bar",
                  relax_left=2.5, relax_right=3.0, relax_tau=0.0, wave=wave)
    om = osem.mesh_for(wl)
    gm = sem.Mesh.from_workload(wl, h=om.h, precision=precision, tol=1e-13 if precision == "fp64" else 1e-12)
    return wl, om, gm


def test_relaxation_zones_rk4_steps():
    wl, om, gm = _zone_pair()
    x = om.xcol
    e0 = 0.01 * np.cos(0.8 * x) + 0.005
    p0 = 0.05 * np.sin(0.8 * x)
    eta, phis = T(e0), T(p0)
    t = gm.rk4_step(eta, phis, wl.dt, 2, t=0.3)
    e, p = e0, p0
    for s in range(2):
        e, p = om.rk4_step(e, p, wl.dt, t=0.3 + s * wl.dt)
    assert t == pytest.approx(0.3 + 2 * wl.dt)
    assert rel(eta, e) < TOL_FP64 and rel(phis, p) < TOL_FP64


def test_zakharov_rhs_with_zones_needs_tau():
    wl, om, gm = _zone_pair()
    de = torch.empty(om.ncol, dtype=torch.float64, device=DEV)
    with pytest.raises(sem.SemError):
        gm.zakharov_rhs(T(np.zeros(om.ncol)), T(np.zeros(om.ncol)), de, torch.empty_like(de), t=0.5)


@pytest.mark.slow
def test_c4_shoal_full_size_two_steps():
    from sem_workloads import c4_shoal
    wl = c4_shoal()
    om = osem.mesh_for(wl)
    for precision, tol in (("fp64", TOL_FP64), ("mixed", TOL_MIXED)):
        gm = sem.Mesh.from_workload(wl, h=om.h, precision=precision, tol=1e-13 if precision == "fp64" else 1e-12)
        e0, p0 = np.zeros(om.ncol), np.zeros(om.ncol)
        eta, phis = T(e0), T(p0)
        gm.rk4_step(eta, phis, wl.dt, 2, t=1.0)
        if precision == "fp64":
            e, p = e0, p0
            for s in range(2):
                e, p = om.rk4_step(e, p, wl.dt, t=1.0 + s * wl.dt)
        assert np.abs(e).max() > 1e-5               # the zone is generating waves
        assert rel(eta, e) < tol and rel(phis, p) < tol


def test_mesh_memory_is_reused_and_trimmed():
    """Destroyed meshes return their device block to the library's cache: creating and destroying
    many meshes of one size does not grow the device memory in use, a reused block gives the same
    results, and sem_trim_cache hands the cached blocks back to CUDA."""
    wl, om, gm = make_pair(P=5, Nx=40, Nz=3)
    eta, phis = surface(om, seed=5)
    ref = om.laplace_solve(eta, phis)
    gm.close()
    torch.cuda.synchronize()
    free0 = torch.cuda.mem_get_info()[0]
    for _ in range(20):
        m = sem.Mesh.from_workload(wl, h=om.h)
        m.update_geometry(T(eta))
        Phi = torch.zeros(om.n, dtype=torch.float64, device=DEV)
        m.laplace_solve(T(phis), Phi)
        assert rel(Phi, ref) < TOL_FP64
        m.close()
    torch.cuda.synchronize()
    block = sem.mesh_footprint(sem.mesh_params(wl.P, wl.Nx, wl.Nz, wl.periodic, wl.Pf, wl.filter_alpha,
                                               wl.filter_s, wl.filter_ic, wl.g), wl.element_edges(), om.h)
    assert free0 - torch.cuda.mem_get_info()[0] <= 2 * block + (4 << 20)
    sem.load_library().sem_trim_cache()
    torch.cuda.synchronize()
    assert torch.cuda.mem_get_info()[0] >= free0 - (4 << 20)
