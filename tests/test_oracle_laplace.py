"""Pins for the oracle's σ-geometry, stiffness and Laplace solve (§2, §3.1.2).

* The K formula is checked against the Dirichlet energy computed in the
  PHYSICAL domain by finite differences (no K involved), so a dropped ∂xh
  term or a sign slip in K12 fails.
* The assembled operator is symmetric, annihilates constants (Neumann
  everywhere before the Dirichlet lift) and is negative semidefinite.
* The banded RCM Cholesky equals a dense solve.
* A harmonic potential cosh(k(z+h))·sin(kx) under a curved free surface is
  reproduced with exponential convergence in P.
"""
import math

import numpy as np
import pytest

from oracle import sem, poly
from oracle.banded import BandedCholesky, rcm_order, bandwidth


def make_mesh(P, Nx, Nz, periodic=True, h=None, L=2 * math.pi):
    edges = np.linspace(0.0, L, Nx + 1)
    ncol = Nx * P if periodic else Nx * P + 1
    if h is None:
        h = np.ones(ncol)
    return sem.Mesh(P, Nx, Nz, edges, periodic, h)


# --- K: σ-transformed Dirichlet energy equals the physical one ------------------------------
def _bathy(x):
    return 1.0 - 0.3 * np.exp(-((x - 1.5) ** 2)), 0.3 * 2 * (x - 1.5) * np.exp(-((x - 1.5) ** 2))


def _surf(x):
    return 0.15 * np.sin(1.3 * x) + 0.05, 0.15 * 1.3 * np.cos(1.3 * x)


def _U(x, s):
    return np.sin(0.9 * x) * np.cosh(1.1 * s) + 0.3 * x * s ** 2


def test_sigma_K_matches_physical_dirichlet_energy():
    X0, X1 = 0.0, 3.0
    xg, wx = np.polynomial.legendre.leggauss(160)
    xg = X0 + 0.5 * (xg + 1) * (X1 - X0)
    wx = 0.5 * (X1 - X0) * wx
    sg, ws = np.polynomial.legendre.leggauss(40)
    eps = 1e-5
    # computational side: ∫∫ (K ∇U)·∇U dx dσ, ∇U by central differences in (x, σ)
    Xc, Sc = np.meshgrid(xg, 0.5 * (sg + 1), indexing="ij")
    Wc = np.outer(wx, 0.5 * ws)
    Ux = (_U(Xc + eps, Sc) - _U(Xc - eps, Sc)) / (2 * eps)
    Us = (_U(Xc, Sc + eps) - _U(Xc, Sc - eps)) / (2 * eps)
    h, hx = _bathy(Xc)
    eta, etax = _surf(Xc)
    K11, K12, K22 = sem.sigma_K(eta + h, hx, etax + hx, Sc)
    lhs = np.sum(Wc * (K11 * Ux * Ux + 2 * K12 * Ux * Us + K22 * Us * Us))
    # physical side: ∫∫ |∇u|² dx dz over -h(x) < z < η(x), u(x,z) = U(x, σ(x,z))
    def u(x, z):
        hh, _ = _bathy(x)
        ee, _ = _surf(x)
        return _U(x, (z + hh) / (ee + hh))
    hq, _ = _bathy(xg)
    eq, _ = _surf(xg)
    zq = -hq[:, None] + 0.5 * (sg[None, :] + 1) * (eq + hq)[:, None]
    Wp = wx[:, None] * 0.5 * ws[None, :] * (eq + hq)[:, None]
    Xp = np.broadcast_to(xg[:, None], zq.shape)
    ux = (u(Xp + eps, zq) - u(Xp - eps, zq)) / (2 * eps)
    uz = (u(Xp, zq + eps) - u(Xp, zq - eps)) / (2 * eps)
    rhs = np.sum(Wp * (ux * ux + uz * uz))
    assert abs(lhs - rhs) < 1e-7 * abs(rhs)
    # the flat-bottom K printed in §2 (K12 = -σ ∂xη) is NOT enough here
    K11f, K12f, K22f = sem.sigma_K(eta + h, 0 * hx, etax, Sc)
    wrong = np.sum(Wc * (K11f * Ux * Ux + 2 * K12f * Ux * Us + K22f * Us * Us))
    assert abs(wrong - rhs) > 1e-3 * abs(rhs)


def test_sigma_K_flat_bottom_reduces_to_printed_form():
    d, ex, s = 1.3, 0.2, 0.7
    K11, K12, K22 = sem.sigma_K(d, 0.0, ex, s)
    assert K11 == pytest.approx(d)
    assert K12 == pytest.approx(-s * ex)
    assert K22 == pytest.approx((1 + (s * ex) ** 2) / d)


def test_element_K_uses_exact_local_derivatives():
    # η and h quadratic in x on a walls mesh: element-local collocation derivatives are exact
    P, Nx, Nz = 3, 3, 2
    L = 2.0
    edges = np.linspace(0, L, Nx + 1)
    m0 = make_mesh(P, Nx, Nz, periodic=False, L=L)
    x = m0.xcol
    h = 1.0 + 0.1 * x - 0.05 * x ** 2
    eta = 0.02 + 0.03 * x ** 2
    m = sem.Mesh(P, Nx, Nz, edges, False, h)
    K11, K12, K22 = m.element_K(eta)
    xe = x[m.col]                                        # (Nx, P+1)
    hx = 0.1 - 0.1 * xe
    dx = 0.06 * xe + hx
    d = (eta + h)[m.col]
    sig = m.sigma_row[m.row]
    for ex_ in range(Nx):
        for l in range(Nz):
            e11, e12, e22 = sem.sigma_K(d[ex_][:, None], hx[ex_][:, None], dx[ex_][:, None], sig[l][None, :])
            np.testing.assert_allclose(K12[ex_, l], e12, atol=1e-13)
            np.testing.assert_allclose(K22[ex_, l], e22, atol=1e-13)
            np.testing.assert_allclose(K11[ex_, l], e11, atol=1e-13)


# --- assembled operator structure ---------------------------------------------------------------
@pytest.mark.parametrize("periodic", [True, False])
def test_stiffness_structure(periodic):
    m = make_mesh(4, 3, 2, periodic=periodic)
    x = m.xcol
    eta = 0.1 * np.cos(x) + 0.03 * np.sin(3 * x)
    L = m.stiffness(eta).toarray()
    np.testing.assert_allclose(L, L.T, atol=1e-12)
    np.testing.assert_allclose(L @ np.ones(m.n), 0.0, atol=1e-11)
    ev = np.linalg.eigvalsh(-L)
    assert ev.min() > -1e-10 and np.sum(ev < 1e-10) == 1      # one null vector: constants
    # Dirichlet-eliminated block is SPD
    A = -L[np.ix_(m.interior, m.interior)]
    assert np.linalg.eigvalsh(A).min() > 1e-8


def test_l2g_layout():
    m = make_mesh(3, 4, 2, periodic=True)
    # column-major canonical numbering and periodic wrap of the last element's right column
    assert m.l2g[0, 0, 0, 0] == 0
    assert m.l2g[0, 1, 0, 0] == 3                       # row l·P + b
    assert m.l2g[3, 0, 3, 0] == 0                       # col (3·3+3) mod 12 = 0
    counts = np.bincount(m.l2g.ravel(), minlength=m.n)
    assert counts.min() >= 1 and counts.max() == 4      # corner nodes are shared by 4 elements


# --- banded direct solver ----------------------------------------------------------------------
def test_banded_cholesky_equals_dense_solve():
    rng = np.random.default_rng(1)
    m = make_mesh(3, 2, 2, periodic=True)
    eta = 0.1 * np.cos(m.xcol)
    L = m.stiffness(eta)
    A = -L[m.interior][:, m.interior]
    b = rng.standard_normal((A.shape[0], 3))
    x = BandedCholesky(A).solve(b)
    np.testing.assert_allclose(x, np.linalg.solve(A.toarray(), b), rtol=1e-11, atol=1e-11)


def test_rcm_reduces_bandwidth_of_scrambled_matrix():
    import scipy.sparse as sp
    n = 400
    A = sp.kron(sp.eye(20), sp.diags([np.full(19, -1.0), np.full(20, 4.0), np.full(19, -1.0)], [-1, 0, 1])) \
        + sp.kron(sp.diags([np.full(19, -1.0), np.full(19, -1.0)], [-1, 1]), sp.eye(20))
    p = np.random.default_rng(0).permutation(n)
    As = A.tocsr()[p][:, p]
    q = rcm_order(As)
    assert bandwidth(As[q][:, q]) <= 25 < bandwidth(As)
    x = BandedCholesky(As).solve(np.ones(n))
    np.testing.assert_allclose(As @ x, np.ones(n), atol=1e-11)


# --- manufactured harmonic potential ---------------------------------------------------------
def _harmonic_errors(P, Nx=4, Nz=2, k=1.0):
    m = make_mesh(P, Nx, Nz)
    x = m.xcol
    eta = 0.1 * np.cos(x) + 0.05 * np.sin(2 * x)
    phis = np.cosh(k * (eta + 1.0)) * np.sin(k * x)
    Phi = m.laplace_solve(eta, phis)
    d = eta + m.h
    X = np.repeat(x, m.nrow)
    Z = np.tile(m.sigma_row, m.ncol) * np.repeat(d, m.nrow) - np.repeat(m.h, m.nrow)
    exact = np.cosh(k * (Z + 1.0)) * np.sin(k * X)
    wt = m.w_surface(eta, Phi)
    w_exact = k * np.sinh(k * (eta + 1.0)) * np.sin(k * x)
    return np.abs(Phi - exact).max(), np.abs(wt - w_exact).max()


def test_harmonic_potential_exponential_convergence():
    errs = [_harmonic_errors(P) for P in (4, 6, 8, 10)]
    e_phi = [e[0] for e in errs]
    e_w = [e[1] for e in errs]
    for a, b in zip(e_phi, e_phi[1:]):
        assert b < a / 20
    for a, b in zip(e_w, e_w[1:]):
        assert b < a / 15
    assert e_phi[-1] < 2e-8 and e_w[-1] < 5e-7


def test_variable_depth_p_self_convergence():
    # no closed form over a bar; successive p-refinements must contract geometrically
    vals = []
    for P in (4, 6, 8, 10):
        m = make_mesh(P, 6, 2)
        x = m.xcol
        h = 1.0 - 0.4 * np.exp(-((x - math.pi) ** 2))
        m = sem.Mesh(P, 6, 2, np.linspace(0, 2 * math.pi, 7), True, h)
        eta = 0.08 * np.cos(x)
        phis = 0.3 * np.sin(x)
        Phi = m.laplace_solve(eta, phis)
        wt = m.w_surface(eta, Phi)
        # sample w̃ at the element edges (nodes common to every P)
        vals.append(wt[m.col[:, 0]])
    diffs = [np.abs(vals[i + 1] - vals[i]).max() for i in range(3)]
    assert diffs[1] < diffs[0] / 5 and diffs[2] < diffs[1] / 5
