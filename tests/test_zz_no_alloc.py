"""Allocation-free operator apply (sem_laplace_apply_noalloc) against the regular apply.

Some callers cannot allocate device memory when they call the library: a real-time loop
that forbids allocator calls (cudaMalloc and cudaFree can synchronise the device), or a
host whose own memory manager owns the GPU's memory and refuses raw cudaMalloc.  For
them the library offers an apply whose only temporary lives in a static device array.  This
test calls it through the C ABI twice in a row (the array keeps the first call's
contents) and checks each result against sem_laplace_apply at the tolerance of the
other operator tests; it also checks that a mesh too large for the array is refused.
The file is named so that pytest collects it last.
"""
import numpy as np
import pytest

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():
    pytest.skip("needs a CUDA GPU", allow_module_level=True)

import paper_1512_02548_gb300 as sem  # noqa: E402
from sem_workloads import small_case, random_field  # noqa: E402

pytestmark = pytest.mark.gpu
DEV = torch.device("cuda:0")
TOL_OP = 1e-12


def _tensor(x):
    return torch.tensor(np.ascontiguousarray(x), dtype=torch.float64, device=DEV)


def _rel(a, b):
    return float(torch.linalg.norm(a - b) / torch.linalg.norm(b))


@pytest.mark.parametrize("periodic", [True, False], ids=["periodic", "walls"])
def test_noalloc_apply_matches_regular_apply_on_two_calls(periodic):
    wl = small_case(P=5, Nx=9, Nz=2, periodic=periodic)
    h = np.full(wl.ncol, wl.depth)
    m = sem.Mesh.from_workload(wl, h=h)
    x_col = np.linspace(0.0, wl.length, wl.ncol, endpoint=periodic)
    eta = 0.06 * np.cos(2 * np.pi * x_col / wl.length) + 0.02
    m.update_geometry(_tensor(eta))
    for call, seed in enumerate((1, 2)):
        x = _tensor(random_field(m.n, seed))
        y_ref = torch.empty(m.n, dtype=torch.float64, device=DEV)
        m.laplace_apply(x, y_ref)
        y = torch.full((m.n,), float("nan"), dtype=torch.float64, device=DEV)
        m.laplace_apply_noalloc(x, y)
        torch.cuda.synchronize()
        assert torch.isfinite(y).all(), f"call {call}"
        assert _rel(y, y_ref) < TOL_OP, f"call {call}"


def test_noalloc_apply_rejects_meshes_beyond_its_scratch():
    wl = small_case(P=2, Nx=32000, Nz=16, periodic=True)     # Nx*Nrow = 32000*33 > 2^20
    m = sem.Mesh.from_workload(wl, h=np.full(wl.ncol, wl.depth))
    x = torch.zeros(m.n, dtype=torch.float64, device=DEV)
    y = torch.zeros_like(x)
    with pytest.raises(sem.SemError) as ei:
        m.laplace_apply_noalloc(x, y)
    assert ei.value.code == 1 and "exceeds the static scratch" in str(ei.value)
