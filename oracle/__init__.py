"""CPU FP64 oracle for the σ-transformed nodal SEM water-wave model (arXiv 1512.02548).

TEST INFRASTRUCTURE ONLY.  This is a plain, slow and obviously correct
restatement of the paper's method: global assembly of the SEM stiffness
matrix, a reverse Cuthill–McKee ordered banded direct solve, gradient
recovery by global L² projection, the over-integrated Zakharov right-hand
side, the per-element modal filter and classical RK4.  Only ``tests/``,
``__graft_entry__.smoke()`` and the CPU-baseline leg of ``bench.py`` may
import it.  It shares no code with the CUDA library and never calls it.

Parity status per function is recorded in each module's docstring; every
function here is pinned by a ``-m "not gpu"`` test against closed forms,
brute force or invariants, except where a docstring says "parity unpinned".
"""
from . import poly, banded, sem  # noqa: F401
