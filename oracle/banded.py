"""Oracle, layer 3: reverse Cuthill–McKee ordering and a banded direct solver.

TEST INFRASTRUCTURE ONLY (see ``oracle/__init__.py``).

§3.1.2 of the paper permutes the symmetric system with reverse
Cuthill–McKee to minimise its bandwidth and then solves it with banded
Gaussian elimination, O(n) work in 2D.  The SPD systems here (−L on the
interior nodes, the 2D mass) are factored by Cholesky in band form.  A
matrix whose half-bandwidth is b is block tridiagonal with blocks of size
b, so the factorisation is written as the block recurrence

    L_00 L_00ᵀ = A_00,
    C_i = A_{i,i−1} L_{i−1}^{−ᵀ},   L_ii L_iiᵀ = A_ii − C_i C_iᵀ,

with dense Cholesky and triangular solves of the b×b blocks as library
primitives.  Nothing is reordered beyond the RCM permutation.
"""
from __future__ import annotations

from collections import deque

import numpy as np
import scipy.linalg as sla
import scipy.sparse as sp


def rcm_order(A: sp.csr_matrix) -> np.ndarray:
    """Reverse Cuthill–McKee permutation of the graph of symmetric A.

    Breadth-first search from a minimum-degree node of each connected
    component, visiting the unvisited neighbours of every node in order of
    increasing degree; the final order is reversed.
    """
    A = sp.csr_matrix(A)
    n = A.shape[0]
    indptr, indices = A.indptr, A.indices
    degree = np.diff(indptr)
    visited = np.zeros(n, dtype=bool)
    order = []
    for start in np.argsort(degree, kind="stable"):
        if visited[start]:
            continue
        visited[start] = True
        queue = deque([start])
        while queue:
            v = queue.popleft()
            order.append(v)
            nb = indices[indptr[v]:indptr[v + 1]]
            nb = nb[~visited[nb]]
            if nb.size:
                nb = nb[np.argsort(degree[nb], kind="stable")]
                visited[nb] = True
                queue.extend(nb.tolist())
    return np.array(order[::-1], dtype=np.int64)


def bandwidth(A: sp.spmatrix) -> int:
    C = sp.coo_matrix(A)
    if C.nnz == 0:
        return 0
    return int(np.max(np.abs(C.row - C.col)))


class BandedCholesky:
    """Cholesky factor of a sparse SPD matrix after RCM, stored as block-tridiagonal blocks."""

    def __init__(self, A: sp.spmatrix, perm: np.ndarray | None = None):
        A = sp.csr_matrix(A)
        self.n = A.shape[0]
        self.perm = rcm_order(A) if perm is None else np.asarray(perm)
        Ap = A[self.perm][:, self.perm].tocsr()
        self.b = max(1, bandwidth(Ap))
        n, b = self.n, self.b
        self.starts = list(range(0, n, b))
        self.diag = []     # L_ii (lower triangular)
        self.sub = []      # C_i  (block below the diagonal, i >= 1)
        prev = None
        for i, s in enumerate(self.starts):
            e = min(s + b, n)
            Aii = Ap[s:e, s:e].toarray()
            if i > 0:
                ps = self.starts[i - 1]
                Ai_im1 = Ap[s:e, ps:s].toarray()
                # C_i = A_{i,i-1} L_{i-1}^{-T}  <=>  L_{i-1} C_iᵀ = A_{i,i-1}ᵀ
                Ci = sla.solve_triangular(prev, Ai_im1.T, lower=True).T
                Aii = Aii - Ci @ Ci.T
                self.sub.append(Ci)
            Lii = np.linalg.cholesky(Aii)
            self.diag.append(Lii)
            prev = Lii

    def solve(self, rhs: np.ndarray) -> np.ndarray:
        rhs = np.asarray(rhs, dtype=np.float64)
        squeeze = rhs.ndim == 1
        f = rhs.reshape(self.n, -1)[self.perm]
        nb = len(self.starts)
        y = [None] * nb
        for i, s in enumerate(self.starts):
            e = min(s + self.b, self.n)
            t = f[s:e]
            if i > 0:
                t = t - self.sub[i - 1] @ y[i - 1]
            y[i] = sla.solve_triangular(self.diag[i], t, lower=True)
        x = [None] * nb
        for i in range(nb - 1, -1, -1):
            t = y[i]
            if i < nb - 1:
                t = t - self.sub[i].T @ x[i + 1]
            x[i] = sla.solve_triangular(self.diag[i], t, lower=True, trans="T")
        xp = np.vstack(x)
        out = np.empty_like(xp)
        out[self.perm] = xp
        return out[:, 0] if squeeze else out
