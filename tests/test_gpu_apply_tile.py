"""Tiled operator apply (FP64 through sem_laplace_apply, FP32 through sem_laplace_apply_f32) against
the oracle's assembled operator and the element-column kernel (SEM_APPLY_KERNEL=column).

Tolerances (relative L² over all nodes, random x): FP64 1e-12 as for the element-column kernel;
FP32 2e-6 — unit roundoff 6e-8 times the ≈4(P+1)+10 terms of a node's sum, with random x
there is no cancellation to amplify it.  The cases span several tiles of 16 elements with a
ragged last tile, periodic ends (the first tile's left element is the last element) and walls
(no left element for the first tile, the right-wall column written by the last tile), and
orders 2–12.
"""
import os

import numpy as np
import pytest

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():
    pytest.skip("needs a CUDA GPU", allow_module_level=True)

import paper_1512_02548_gb300 as sem  # noqa: E402
from oracle import sem as osem  # noqa: E402
from sem_workloads import small_case, random_field  # noqa: E402

pytestmark = pytest.mark.gpu
DEV = torch.device("cuda:0")

CASES = [
    dict(P=6, Nx=37, Nz=4),
    dict(P=4, Nx=40, Nz=3, periodic=False),
    dict(P=3, Nx=16, Nz=2, bar=True),
    dict(P=2, Nx=33, Nz=5, periodic=False, bar=True),
    dict(P=8, Nx=19, Nz=2),
    dict(P=12, Nx=5, Nz=1, periodic=False),
    dict(P=5, Nx=1, Nz=3, periodic=False),
    dict(P=7, Nx=3, Nz=2),
]


def rel(a, b):
    a = a.detach().double().cpu().numpy()
    return np.linalg.norm(a - b) / max(np.linalg.norm(b), 1e-300)


def setup(P, Nx, Nz, periodic=True, bar=False):
    wl = small_case(P=P, Nx=Nx, Nz=Nz, periodic=periodic)
    om = osem.mesh_for(wl, bar=bar)
    gm = sem.Mesh.from_workload(wl, h=om.h)
    x = om.xcol
    eta = 0.06 * np.cos(2 * np.pi * x / wl.length * (1 if periodic else 0.5)) + 0.01 * np.sin(5 * x)
    gm.update_geometry(torch.tensor(eta, device=DEV))
    return wl, om, gm, eta


def column_env(fn):
    old = os.environ.get("SEM_APPLY_KERNEL")
    os.environ["SEM_APPLY_KERNEL"] = "column"
    try:
        return fn()
    finally:
        if old is None:
            del os.environ["SEM_APPLY_KERNEL"]
        else:
            os.environ["SEM_APPLY_KERNEL"] = old


@pytest.mark.parametrize("case", CASES, ids=lambda c: "-".join(f"{k}{v}" for k, v in c.items()))
def test_tiled_apply_fp64_and_fp32(case):
    wl, om, gm, eta = setup(**case)
    x = random_field(om.n, 5)
    ref = om.stiffness(eta) @ x
    xd = torch.tensor(x, device=DEV)
    y_col = torch.empty_like(xd)
    column_env(lambda: gm.laplace_apply(xd, y_col))
    y_tile = torch.full_like(xd, float("nan"))
    gm.laplace_apply(xd, y_tile)
    assert rel(y_tile, ref) < 1e-12
    assert rel(y_tile, y_col.cpu().numpy()) < 1e-13
    y32 = torch.full((om.n,), float("nan"), dtype=torch.float32, device=DEV)
    gm.laplace_apply_f32(xd.float(), y32)
    assert rel(y32, ref) < 2e-6


def test_tiled_apply_is_deterministic_and_covers_every_node():
    wl, om, gm, eta = setup(P=6, Nx=70, Nz=4)
    x = torch.tensor(random_field(om.n, 8), device=DEV).float()
    a = torch.full((om.n,), float("nan"), dtype=torch.float32, device=DEV)
    b = torch.full((om.n,), float("nan"), dtype=torch.float32, device=DEV)
    gm.laplace_apply_f32(x, a)
    gm.laplace_apply_f32(x, b)
    assert bool(torch.isfinite(a).all()) and torch.equal(a, b)


def test_tiled_apply_rejects_bad_arguments():
    wl, om, gm, eta = setup(P=4, Nx=5, Nz=1)
    x = torch.zeros(om.n, dtype=torch.float32, device=DEV)
    with pytest.raises(sem.SemError):
        gm.laplace_apply_f32(x, x)
    with pytest.raises(ValueError):
        gm.laplace_apply_f32(x.double(), x)


def test_unaligned_input_takes_the_plain_staging_path():
    """Bulk copies need a 16-byte-aligned source; an input that starts 4 bytes into an allocation
    is staged with plain loads and gives the same result."""
    wl, om, gm, eta = setup(P=6, Nx=37, Nz=4)
    x = torch.tensor(random_field(om.n, 6), device=DEV).float()
    buf = torch.empty(om.n + 1, dtype=torch.float32, device=DEV)
    buf[1:] = x
    xu = buf[1:]
    assert xu.data_ptr() % 16 != 0
    a = torch.empty(om.n, dtype=torch.float32, device=DEV)
    b = torch.empty(om.n, dtype=torch.float32, device=DEV)
    gm.laplace_apply_f32(x, a)
    gm.laplace_apply_f32(xu, b)
    assert torch.equal(a, b)


TC_CASES = [
    dict(P=4, Nx=130, Nz=1),
    dict(P=5, Nx=70, Nz=2, periodic=False, bar=True),
    dict(P=6, Nx=47, Nz=4),
    dict(P=7, Nx=44, Nz=3, periodic=False),
    dict(P=6, Nx=16, Nz=4, periodic=False),
    dict(P=6, Nx=1, Nz=4, periodic=False),
    dict(P=5, Nx=25, Nz=5, bar=True),
    dict(P=7, Nx=9, Nz=1, periodic=False),
]


def tc_env(fn):
    old = os.environ.get("SEM_APPLY_F32")
    os.environ["SEM_APPLY_F32"] = "tc"
    try:
        return fn()
    finally:
        if old is None:
            del os.environ["SEM_APPLY_F32"]
        else:
            os.environ["SEM_APPLY_F32"] = old


@pytest.mark.parametrize("case", TC_CASES, ids=lambda c: "-".join(f"{k}{v}" for k, v in c.items()))
def test_tensor_core_fp32_apply_matches_the_oracle_and_the_scalar_kernel(case):
    """Orders 4..7 with SEM_APPLY_F32=tc take the tensor-core kernel (3×TF32 products, tiles of
    64/Nz − 1 elements): the cases cover one to several tiles with ragged last tiles, an odd block
    count (last block pair half empty), walls and periodic ends, a bar, and layer counts 1–5 (5:
    the run-time layer count).  Same tolerance as the CUDA-core FP32 kernel, 2e-6, against the
    oracle and against that kernel; the tensor-core result is bitwise reproducible."""
    wl, om, gm, eta = setup(**case)
    x = random_field(om.n, 9)
    ref = om.stiffness(eta) @ x
    xd = torch.tensor(x, device=DEV).float()
    y_sc = torch.full((om.n,), float("nan"), dtype=torch.float32, device=DEV)
    gm.laplace_apply_f32(xd, y_sc)
    y_tc = torch.full((om.n,), float("nan"), dtype=torch.float32, device=DEV)
    tc_env(lambda: gm.laplace_apply_f32(xd, y_tc))
    y_tc2 = torch.full((om.n,), float("nan"), dtype=torch.float32, device=DEV)
    tc_env(lambda: gm.laplace_apply_f32(xd, y_tc2))
    assert bool(torch.isfinite(y_tc).all()) and torch.equal(y_tc, y_tc2)
    assert rel(y_tc, ref) < 2e-6
    assert rel(y_sc, ref) < 2e-6
    assert rel(y_tc, y_sc.double().cpu().numpy()) < 2e-6
