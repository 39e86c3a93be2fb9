"""The C ABI library builds, loads without a GPU and exports every symbol include/sem.h declares."""
import ctypes
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
HEADER = os.path.join(ROOT, "include", "sem.h")


def declared_symbols():
    text = open(HEADER).read()
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    return sorted(set(re.findall(r"\b(sem_[a-z0-9_]+)\s*\(", text)))


@pytest.fixture(scope="module")
def lib():
    import paper_1512_02548_gb300 as sem
    if not os.path.exists(sem.LIB_PATH):
        from paper_1512_02548_gb300.build import build_library
        build_library()
    return ctypes.CDLL(sem.LIB_PATH)


def test_header_declares_the_boundary():
    syms = declared_symbols()
    for name in ("sem_mesh_create", "sem_update_geometry", "sem_laplace_solve",
                 "sem_recover_gradient", "sem_zakharov_rhs", "sem_rk4_step"):
        assert name in syms


def test_every_declared_symbol_is_exported(lib):
    missing = [s for s in declared_symbols() if not hasattr(lib, s)]
    assert not missing, missing


def test_binding_covers_every_symbol():
    import paper_1512_02548_gb300 as sem
    assert sorted(sem.EXPORTED) == declared_symbols()


def test_no_compute_without_gpu_is_an_error_not_a_fallback(lib):
    # host-only calls work; creating a mesh without a GPU must fail with an error code
    lib.sem_last_error.restype = ctypes.c_char_p
    lib.sem_launch_count.restype = ctypes.c_int64
    assert lib.sem_launch_count() >= 0
    import torch
    if torch.cuda.is_available():
        pytest.skip("GPU present")
    import paper_1512_02548_gb300 as sem
    import numpy as np
    with pytest.raises(sem.SemError):
        sem.Mesh(4, 4, 1, np.linspace(0, 1, 5), np.ones(16))
