"""The autotuner's knobs change how a batch is planned, not its results.

The planning parameters (cluster team share, largest cluster, build by group size, plan) and the
tiled apply's tile width are set through the C ABI as the autotuner sets them; an uneven batch and
a long-tank apply then give the same results as with the defaults, within the tolerances of the
other parity tests (1e-10 FP64, 1e-8 mixed, 1e-6 for the FP32 apply).  The committed tuning file
must name a device and hold valid values.
"""
import json
import os

import numpy as np
import pytest

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():
    pytest.skip("needs a CUDA GPU", allow_module_level=True)

import paper_1512_02548_gb300 as sem  # noqa: E402
from paper_1512_02548_gb300.autotune import TUNING_PATH  # noqa: E402
from sem_workloads import c3_instances, initial_state, roofline_tank, random_field  # noqa: E402

pytestmark = pytest.mark.gpu
DEV = torch.device("cuda:0")


def _step(wls, init, precision):
    meshes = [sem.Mesh.from_workload(wl, precision=precision, tol=1e-13 if precision == "fp64" else 1e-12)
              for wl in wls]
    b = sem.Batch(meshes, tuned=False)
    etas = [torch.tensor(e, device=DEV) for e, _ in init]
    phis = [torch.tensor(p, device=DEV) for _, p in init]
    b.rk4_step(etas, phis, [wl.dt for wl in wls], 2)
    out = [(e.cpu().numpy(), p.cpu().numpy()) for e, p in zip(etas, phis)]
    b.close()
    for m in meshes:
        m.close()
    return out


def _rel(a, b):
    return float(np.linalg.norm(a - b) / np.linalg.norm(b))


@pytest.mark.parametrize("precision,tol", [("fp64", 1e-10), ("mixed", 1e-8)])
def test_batch_tuning_changes_the_plan_not_the_results(precision, tol):
    wls = c3_instances(24, seed=3)
    init = []
    for wl in wls:
        x = np.linspace(0.0, wl.length, wl.ncol, endpoint=False)
        init.append(initial_state(wl, x, np.full(wl.ncol, wl.depth)))
    try:
        sem.set_batch_tuning(reset=True)
        ref = _step(wls, init, precision)
        for tune in (dict(cluster_share=0.125, max_cluster=4), dict(cluster_share=2.0, max_cluster=16, narrow_max=0),
                     dict(plan=0), dict(plan=1, max_cluster=8)):
            sem.set_batch_tuning(reset=True, **tune)
            got = _step(wls, init, precision)
            for (e, p), (er, pr) in zip(got, ref):
                assert _rel(e, er) < tol and _rel(p, pr) < tol, tune
    finally:
        sem.set_batch_tuning(reset=True)


def test_apply_tile_width_changes_nothing_but_the_tiling():
    wl = roofline_tank(Nx=300, Nz=2, P=5)
    m = sem.Mesh.from_workload(wl)
    m.update_geometry(torch.tensor(0.05 * np.cos(np.linspace(0, 6 * np.pi, wl.ncol, endpoint=False)), device=DEV))
    x = torch.tensor(random_field(m.n, 5), dtype=torch.float32, device=DEV)
    ref = torch.empty_like(x)
    m.laplace_apply_f32(x, ref)
    try:
        for E in (1, 3, 16):
            sem.set_apply_tile_width(5, 2, E)
            y = torch.full_like(x, float("nan"))
            m.laplace_apply_f32(x, y)
            assert float(torch.linalg.norm(y - ref) / torch.linalg.norm(ref)) < 1e-6, E
    finally:
        sem.set_apply_tile_width(5, 2, 0)


def test_committed_tuning_is_valid():
    if not os.path.exists(TUNING_PATH):
        pytest.skip("no tuning file")
    data = json.load(open(TUNING_PATH))
    b = data["batch"]
    assert data["device"] and 0 < b["cluster_share"] <= 64 and b["max_cluster"] in (1, 2, 4, 8, 16)
    assert b["plan"] in (-1, 0, 1) and b["narrow_max"] >= 0
    for key, E in data["apply_tile_width"].items():
        P, Nz = (int(v) for v in key.split(","))
        assert 2 <= P <= 12 and 1 <= Nz <= 16 and 1 <= E <= 16
