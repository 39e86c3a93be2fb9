"""Continuous-batching loop on the GPU: each served result equals the same request run alone.

A short Poisson stream of Laplace solves and RK4 runs on uneven periodic tanks is served with
budgeted admission; every result is compared with the request run alone on the plain
single-instance path (1e-10 FP64; 1e-8 for the mixed-precision loop against the FP64 run),
and samples against the oracle.  A budget that admits only a few requests at a time gives the
same results; a request with a non-finite surface fails alone.
"""
import numpy as np
import pytest

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():
    pytest.skip("needs a CUDA GPU", allow_module_level=True)

from oracle import sem as osem  # noqa: E402
from paper_1512_02548_gb300.serve import GpuExecutor, Request, Server, run_alone  # noqa: E402
from sem_workloads import c5_requests, initial_state  # noqa: E402

pytestmark = pytest.mark.gpu


def stream(count=14, seed=3, nsteps=3):
    out = []
    for i, (kind, t, wl, ns) in enumerate(c5_requests(3000.0, count, seed, nmin=1e3, nmax=8e3, nsteps=nsteps)):
        om = osem.mesh_for(wl)
        e0, p0 = initial_state(wl, om.xcol, om.h)
        out.append(Request(i, kind, wl, e0, p0, ns, t))
    return out


def copy(reqs):
    return [Request(r.rid, r.kind, r.wl, r.eta0, r.phis0, r.nsteps, r.arrival) for r in reqs]


def rel(a, b):
    return np.linalg.norm(a - b) / max(np.linalg.norm(b), 1e-300)


def check(served, alone, tol):
    for r in served:
        assert r.error is None, (r.rid, r.error)
        ref = alone[r.rid]
        if r.kind == "laplace":
            assert rel(r.result["Phi"], ref["Phi"]) < tol, r.rid
        else:
            assert rel(r.result["eta"], ref["eta"]) < tol and rel(r.result["phis"], ref["phis"]) < tol, r.rid
            assert r.result["t"] == pytest.approx(ref["t"])


@pytest.fixture(scope="module")
def reqs_and_alone():
    reqs = stream()
    return reqs, {r.rid: run_alone(r, "fp64") for r in reqs}


def test_served_fp64_equals_alone_and_oracle(reqs_and_alone):
    reqs, alone = reqs_and_alone
    served = copy(reqs)
    s = Server(GpuExecutor("fp64"), hbm_budget=8 << 30).run(served)
    assert s["completed"] == len(reqs) and s["peak_active"] > 1
    check(served, alone, 1e-10)
    lap = next(r for r in served if r.kind == "laplace")
    om = osem.mesh_for(lap.wl)
    assert rel(lap.result["Phi"], om.laplace_solve(lap.eta0, lap.phis0)) < 1e-10
    rk = next(r for r in served if r.kind == "rk4")
    om = osem.mesh_for(rk.wl)
    e, p = rk.eta0, rk.phis0
    for k in range(rk.nsteps):
        e, p = om.rk4_step(e, p, rk.wl.dt, t=k * rk.wl.dt)
    assert rel(rk.result["eta"], e) < 1e-10 and rel(rk.result["phis"], p) < 1e-10


def test_served_mixed_precision_within_1e8_of_fp64(reqs_and_alone):
    reqs, alone = reqs_and_alone
    served = copy(reqs)
    s = Server(GpuExecutor("mixed"), hbm_budget=8 << 30).run(served)
    assert s["completed"] == len(reqs)
    check(served, alone, 1e-8)


def test_tight_budget_gives_the_same_results(reqs_and_alone):
    reqs, alone = reqs_and_alone
    ex = GpuExecutor("fp64")
    served = copy(reqs)
    budget = 2 * max(ex.footprint(r) for r in served)
    s = Server(ex, hbm_budget=budget).run(served)
    assert s["completed"] == len(reqs) and s["peak_bytes"] <= budget
    check(served, alone, 1e-10)


def test_nonfinite_request_fails_alone(reqs_and_alone):
    reqs, alone = reqs_and_alone
    served = copy(reqs)
    bad = next(r for r in served if r.kind == "rk4")
    bad.eta0 = bad.eta0.copy()
    bad.eta0[1] = np.nan
    s = Server(GpuExecutor("fp64"), hbm_budget=8 << 30).run(served)
    assert bad.error == "error code 5" and s["failed"] == 1
    check([r for r in served if r is not bad], alone, 1e-10)


@pytest.mark.parametrize("precision,tol", [("fp64", 1e-10), ("mixed", 1e-8)])
def test_requests_run_alone_inside_a_tick_give_the_same_results(reqs_and_alone, precision, tol):
    """With a low solo threshold, each tick runs its larger requests on their own single-mesh path
    and batches the rest: results are those of the requests run alone."""
    reqs, alone = reqs_and_alone
    served = copy(reqs)
    ex = GpuExecutor(precision, solo_nodes=4000)
    assert any(r.wl.n_nodes >= 4000 for r in served) and any(r.wl.n_nodes < 4000 for r in served)
    s = Server(ex, hbm_budget=8 << 30).run(served)
    assert s["completed"] == len(reqs) and s["peak_active"] > 1
    check(served, alone, tol)


def test_nonfinite_request_run_alone_fails_alone(reqs_and_alone):
    reqs, alone = reqs_and_alone
    served = copy(reqs)
    bad = max((r for r in served if r.kind == "rk4"), key=lambda r: r.wl.n_nodes)
    bad.eta0 = bad.eta0.copy()
    bad.eta0[1] = np.nan
    ex = GpuExecutor("fp64", solo_nodes=bad.wl.n_nodes)
    s = Server(ex, hbm_budget=8 << 30).run(served)
    assert bad.error == "error code 5" and s["failed"] == 1
    check([r for r in served if r is not bad], alone, 1e-10)


def test_warm_builds_each_table_combination_once(reqs_and_alone):
    reqs, _ = reqs_and_alone
    combos = {(r.wl.P, r.wl.Nz, r.wl.Pf, r.wl.filter_alpha, r.wl.filter_s, r.wl.filter_ic) for r in reqs}
    assert GpuExecutor("mixed").warm(reqs) == len(combos)
