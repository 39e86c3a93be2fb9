"""Pins for the oracle's 1D tables (§3.1.4, §3.3, §3.4) against closed forms.

Each check fails on a plausible slip: a wrong recurrence coefficient breaks
the GLL closed forms, a transposed Vandermonde breaks D or M exactness, a
wrong bubble basis breaks the filter's interface/mean invariants.
"""
import json
import math
import os

import numpy as np
import pytest

from oracle import poly

GOLDEN = os.path.join(os.path.dirname(__file__), "golden", "gll_closed_forms.json")


def monomial_integral(m):
    return 0.0 if m % 2 else 2.0 / (m + 1)


def test_gll_closed_forms_from_golden():
    data = json.load(open(GOLDEN))
    for entry in data["cases"]:
        P = entry["P"]
        r, w = poly.gll_nodes_weights(P)
        np.testing.assert_allclose(r, [eval(v, {"sqrt": math.sqrt}) for v in entry["nodes"]], atol=1e-15)
        np.testing.assert_allclose(w, [eval(v, {"sqrt": math.sqrt}) for v in entry["weights"]], atol=1e-15)


@pytest.mark.parametrize("P", range(1, 13))
def test_gll_quadrature_degree(P):
    r, w = poly.gll_nodes_weights(P)
    assert np.all(np.diff(r) > 0)
    for m in range(2 * P):          # exact up to degree 2P-1
        assert abs(w @ r ** m - monomial_integral(m)) < 1e-13
    # degree 2P is NOT integrated exactly (Lobatto rule): guards against a Gauss rule by mistake
    assert abs(w @ r ** (2 * P) - monomial_integral(2 * P)) > 1e-9


@pytest.mark.parametrize("P", range(1, 13))
def test_derivative_exact_on_monomials(P):
    r, _ = poly.gll_nodes_weights(P)
    D = poly.derivative_matrix(P)
    for m in range(P + 1):
        exact = m * r ** (m - 1) if m > 0 else np.zeros_like(r)
        np.testing.assert_allclose(D @ r ** m, exact, atol=1e-11 * max(1, P * P))


@pytest.mark.parametrize("P", range(1, 13))
def test_mass_exact_integrals(P):
    r, _ = poly.gll_nodes_weights(P)
    M = poly.mass_matrix(P)
    assert abs(np.ones(P + 1) @ M @ np.ones(P + 1) - 2.0) < 1e-13
    np.testing.assert_allclose(M, M.T, atol=1e-14)
    for i in range(P + 1):
        for j in range(P + 1):
            assert abs(r ** i @ M @ r ** j - monomial_integral(i + j)) < 1e-12


def test_orthonormal_legendre():
    # ∫ P̃_i P̃_j = δ_ij checked with a 40-point Gauss-Legendre rule (independent of GLL)
    x, wq = np.polynomial.legendre.leggauss(40)
    p, _ = poly.orthonormal_legendre(12, x)
    np.testing.assert_allclose(p @ np.diag(wq) @ p.T, np.eye(13), atol=1e-13)


@pytest.mark.parametrize("P,Pf", [(4, 6), (6, 9), (6, 12), (8, 12), (3, 3)])
def test_interpolation_exact(P, Pf):
    r, _ = poly.gll_nodes_weights(P)
    rf, _ = poly.gll_nodes_weights(Pf)
    I = poly.interpolation_matrix(P, Pf)
    for m in range(P + 1):
        np.testing.assert_allclose(I @ r ** m, rf ** m, atol=1e-13)
    # Iᵀ M_f I = M  (the fine mass integrates the degree-2P product exactly)
    np.testing.assert_allclose(I.T @ poly.mass_matrix(Pf) @ I, poly.mass_matrix(P), atol=1e-13)


@pytest.mark.parametrize("P", [3, 4, 6, 8, 10])
def test_filter_top_mode(P):
    alpha, s = 36.0, 12.0
    F = poly.filter_matrix(P, alpha, s, P - 1)
    r, _ = poly.gll_nodes_weights(P)
    # polynomials of degree < P pass unchanged
    for m in range(P):
        np.testing.assert_allclose(F @ r ** m, r ** m, atol=1e-12)
    # endpoint values untouched (no interface jumps)
    np.testing.assert_allclose(F[0], np.eye(P + 1)[0], atol=1e-13)
    np.testing.assert_allclose(F[-1], np.eye(P + 1)[-1], atol=1e-13)
    # eigenvalues {1,…,1, exp(-α)}
    ev = np.sort(np.linalg.eigvals(F).real)
    np.testing.assert_allclose(ev, np.sort(np.r_[np.ones(P), math.exp(-alpha)]), atol=1e-10)
    # the element mean is preserved exactly for P ≥ 3: ∫(1-r²)P^(1,1)_m = 0 for m ≥ 1
    wint = poly.mass_matrix(P) @ np.ones(P + 1)
    q = np.random.default_rng(P).standard_normal(P + 1)
    assert abs(wint @ (F @ q) - wint @ q) < 1e-13


def test_filter_mild_removes_five_percent_of_top_mode():
    # (α,s) = (0.0513, 0): the top modal coefficient is multiplied by e^{-0.0513} ≈ 0.95 (§3.4)
    P = 6
    sig = poly.filter_response(P, 0.0513, 0.0, P - 1)
    assert abs(sig[-1] - 0.95) < 2e-4 and np.all(sig[:-1] == 1.0)
    r, _ = poly.gll_nodes_weights(P)
    Vh = poly.boundary_bubble_basis(P, r)
    top = Vh[:, -1]
    np.testing.assert_allclose(poly.filter_matrix(P, 0.0513, 0.0, P - 1) @ top, sig[-1] * top, atol=1e-13)


def test_filter_response_shape():
    sig = poly.filter_response(8, 36.0, 12.0, 4)
    assert np.all(sig[:5] == 1.0)
    assert sig[-1] == pytest.approx(math.exp(-36.0))
    assert np.all(np.diff(sig[4:]) < 0)
    assert np.all(poly.filter_response(8, 36.0, 12.0, -1) == 1.0)
