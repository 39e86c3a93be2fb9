"""Pins for the oracle's time stepping (§3.1.1, §4.2).

* RK4 stage coefficients: on a linear right-hand side q' = Aq, one step
  must equal R(ΔtA) q with R(z) = 1 + z + z²/2 + z³/6 + z⁴/24 exactly.
* Linear dispersion: the discrete frequency ω_h² = g⟨c, M'w̃(c)⟩/⟨c, M'c⟩
  of a standing cos(kx) mode converges to ω² = g k tanh(kh) exponentially in P.
* C1 (one period of a small standing wave): the elevation returns after
  T = 2π/ω within the small-amplitude nonlinear deviation; the returned
  period from a parabolic fit is within 1e-3 of T.
"""
import math

import numpy as np
import pytest

from oracle import sem
from sem_workloads import c1_linear_standing, initial_state, linear_omega


def test_rk4_equals_taylor_polynomial_on_linear_rhs():
    wl = c1_linear_standing()
    m = sem.mesh_for(wl)
    n = m.ncol
    rng = np.random.default_rng(7)
    A = rng.standard_normal((2 * n, 2 * n)) * 0.3
    m.zakharov_rhs = lambda e, p, **kw: tuple(np.split(A @ np.r_[e, p], 2))
    q = rng.standard_normal(2 * n)
    dt = 0.11
    e1, p1 = m.rk4_step(q[:n], q[n:], dt)
    Z = dt * A
    R = np.eye(2 * n) + Z + Z @ Z / 2 + Z @ Z @ Z / 6 + Z @ Z @ Z @ Z / 24
    np.testing.assert_allclose(np.r_[e1, p1], R @ q, rtol=1e-13, atol=1e-13)


def test_discrete_dispersion_converges_to_linear_theory():
    om = linear_omega(1.0, 1.0)
    assert om == pytest.approx(2.733357, abs=1e-6)
    errs = []
    for P in (4, 6, 8):
        wl = c1_linear_standing()
        wl.P = P
        m = sem.mesh_for(wl)
        c = np.cos(m.xcol)
        z = np.zeros(m.ncol)
        wt = m.w_surface(z, m.laplace_solve(z, c))
        Mp = m.surface_mass()
        errs.append(abs(math.sqrt(9.81 * (c @ (Mp @ wt)) / (c @ (Mp @ c))) - om))
    assert errs[0] < 1e-3 and errs[1] < errs[0] / 100 and errs[2] < errs[1] / 100
    assert errs[2] < 1e-8


def test_c1_linear_standing_wave_period():
    wl = c1_linear_standing()
    m = sem.mesh_for(wl)
    eta, phis = initial_state(wl, m.xcol, m.h)
    e0 = eta.copy()
    T = 2 * math.pi / linear_omega(1.0, 1.0)
    samples = []
    for s in range(wl.nsteps + 2):
        eta, phis = m.rk4_step(eta, phis, wl.dt)
        samples.append(eta[0])
        if s == wl.nsteps - 1:
            eta_T = eta.copy()
    assert np.linalg.norm(eta_T - e0) / np.linalg.norm(e0) < 1e-2
    # parabolic fit through the three samples around the maximum near t = T
    y = np.array(samples)
    i = int(np.argmax(y[40:])) + 40
    y0, y1, y2 = y[i - 1], y[i], y[i + 1]
    shift = 0.5 * (y0 - y2) / (y0 - 2 * y1 + y2)
    t_max = (i + 1 + shift) * wl.dt
    assert abs(t_max - T) / T < 1e-3


@pytest.mark.slow
def test_c1_energy_and_mass_drift_small():
    wl = c1_linear_standing()
    m = sem.mesh_for(wl)
    eta, phis = initial_state(wl, m.xcol, m.h)
    E0, M0 = m.energy(eta, phis), m.mass(eta)
    for _ in range(wl.nsteps):
        eta, phis = m.rk4_step(eta, phis, wl.dt)
    assert abs(m.energy(eta, phis) / E0 - 1) < 1e-5
    assert abs(m.mass(eta) - M0) < 1e-10
