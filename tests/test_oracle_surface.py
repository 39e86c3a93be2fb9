"""Pins for gradient recovery (§3.1.3), the Zakharov right-hand side with
over-integration (§3.1.1, §3.3) and the filter's conservation (§3.4).

* Recovery is exact when the derivative lies in the discrete space.
* With P_f ≥ 3P the over-integrated right-hand side equals the exact
  integral of the interpolated integrands (computed with a 60-point
  Gauss–Legendre rule, no GLL tables involved); with P_f = P it does not.
* In the small-amplitude limit the right-hand side tends to (w̃, −gη).
"""
import math

import numpy as np
import pytest

from oracle import sem, poly


def make_mesh(P, Nx, Nz, periodic=True, h=None, L=2 * math.pi, **prm):
    edges = np.linspace(0.0, L, Nx + 1)
    ncol = Nx * P if periodic else Nx * P + 1
    if h is None:
        h = np.ones(ncol)
    return sem.Mesh(P, Nx, Nz, edges, periodic, h, sem.Params(**prm))


@pytest.mark.parametrize("P", [3, 5])
def test_surface_gradient_exact_for_polynomials(P):
    m = make_mesh(P, 4, 1, periodic=False, L=3.0)
    x = m.xcol
    f = 0.5 * x ** P - x ** 2 + 3.0
    np.testing.assert_allclose(m.surface_gradient(f), 0.5 * P * x ** (P - 1) - 2 * x, atol=1e-10)


def test_surface_gradient_periodic_converges():
    errs = []
    for P in (4, 6, 8):
        m = make_mesh(P, 5, 1)
        errs.append(np.abs(m.surface_gradient(np.sin(2 * m.xcol)) - 2 * np.cos(2 * m.xcol)).max())
    assert errs[1] < errs[0] / 20 and errs[2] < errs[1] / 20


@pytest.mark.parametrize("Nz,depth", [(1, 1.0), (2, 2.0), (3, 0.7)])
def test_w_recovery_exact_when_derivative_in_space(Nz, depth):
    # Φ(x,σ) = f(x)·g(σ) with g a global polynomial of degree ≤ P: w = f g'(σ)/d lies in V
    P = 4
    m = make_mesh(P, 3, Nz, h=np.full(3 * P, depth))
    x, s = m.xcol, m.sigma_row
    f = np.cos(x)
    g = s ** 4 - 2 * s ** 3 + 0.5 * s
    gp1 = 4 - 6 + 0.5
    Phi = np.outer(f, g).ravel()
    wt = m.w_surface(np.zeros(m.ncol), Phi)
    np.testing.assert_allclose(wt, f * gp1 / depth, atol=1e-12)


def _rhs_by_gauss(m, eta, etax, phisx, wt, g):
    """∫ F N_i dx per node with a 60-point Gauss rule on the degree-P interpolants."""
    P = m.P
    xq, wq = np.polynomial.legendre.leggauss(60)
    r, _ = poly.gll_nodes_weights(P)
    # Lagrange basis on the GLL nodes evaluated at xq (built from scratch, not from poly)
    Lq = np.ones((xq.size, P + 1))
    for j in range(P + 1):
        for k in range(P + 1):
            if k != j:
                Lq[:, j] *= (xq - r[k]) / (r[j] - r[k])
    re = np.zeros(m.ncol)
    rp = np.zeros(m.ncol)
    for ex in range(m.Nx):
        c = m.col[ex]
        e, ex_, px, w = (Lq @ v[c] for v in (eta, etax, phisx, wt))
        Fe = -ex_ * px + w * (1 + ex_ * ex_)
        Fp = -g * e - 0.5 * (px * px - w * w * (1 + ex_ * ex_))
        J = 0.5 * m.dx_e[ex]
        np.add.at(re, c, J * (Lq.T @ (wq * Fe)))
        np.add.at(rp, c, J * (Lq.T @ (wq * Fp)))
    return re, rp


@pytest.mark.parametrize("P", [3, 4])
def test_over_integration_exact_at_3P(P):
    for Pf, exact in ((3 * P, True), (P, False)):
        m = make_mesh(P, 4, 1, Pf=Pf)
        x = m.xcol
        eta = 0.2 * np.cos(x)
        phis = 0.5 * np.sin(x) + 0.1 * np.cos(2 * x)
        _, _, parts = m.zakharov_rhs(eta, phis, return_parts=True)
        re, rp = _rhs_by_gauss(m, eta, parts["etax"], parts["phisx"], parts["w"], m.params.g)
        err = max(np.abs(re - parts["rhs_eta"]).max(), np.abs(rp - parts["rhs_phi"]).max())
        if exact:
            assert err < 1e-12
        else:
            assert err > 1e-8          # standard Galerkin (no over-integration) aliases


def test_small_amplitude_limit_is_linear():
    m = make_mesh(5, 4, 2, Pf=8)
    x = m.xcol
    eps = 1e-6
    eta = eps * np.cos(x)
    phis = eps * 3.0 * np.sin(x)
    de, dp, parts = m.zakharov_rhs(eta, phis, return_parts=True)
    np.testing.assert_allclose(de / eps, parts["w"] / eps, atol=1e-5)
    np.testing.assert_allclose(dp / eps, -m.params.g * eta / eps, atol=1e-5)


def test_filter_preserves_mass_and_interfaces():
    m = make_mesh(6, 5, 1, filter_alpha=36.0, filter_s=12.0, filter_ic=5)
    q = np.random.default_rng(3).standard_normal(m.ncol)
    fq = m.apply_filter(q)
    assert abs(m.mass(fq) - m.mass(q)) < 1e-13
    np.testing.assert_allclose(fq[m.col[:, 0]], q[m.col[:, 0]], atol=1e-14)
    assert np.linalg.norm(fq - q) > 1e-3      # it does act on the top mode of random data


def _rates(P):
    from sem_workloads import small_case
    wl = small_case(P=P, Nx=6, Nz=2, filt=False)
    m = sem.mesh_for(wl)
    x = m.xcol
    eta = 0.12 * np.cos(x + 0.3) + 0.05 * np.sin(2 * x)
    phis = 0.5 * np.sin(x) + 0.15 * np.cos(2 * x + 1)
    de, dp, parts = m.zakharov_rhs(eta, phis, return_parts=True)
    h = 1e-5
    dE = (m.energy(eta + h * de, phis + h * dp) - m.energy(eta - h * de, phis - h * dp)) / (2 * h)
    return parts["rhs_eta"].sum(), dE


def test_nonlinear_terms_conserve_mass_and_energy():
    """The Zakharov system conserves volume and energy; the Galerkin form does so
    up to truncation error, which must shrink exponentially in P.  A wrong sign in
    any nonlinear term of eq. (FSeqs) gives O(0.1) rates on this steep asymmetric
    state (checked by planting such mistakes by hand)."""
    m4, e4 = _rates(4)
    m8, e8 = _rates(8)
    assert abs(m4) < 1e-3 and abs(e4) < 1e-3
    assert abs(m8) < 1e-9 and abs(e8) < 1e-7
    assert abs(m8) < abs(m4) / 1e4
