"""Pins for the relaxation zones of §2.2 and the generated wave signal.

* γ(x) is 1 outside the zones and rises smoothly (C¹) from 0 at a zone's outer end to 1 at
  its inner end.
* The generated signal η_a, φ̃_a satisfies the linearised free-surface equations: with the
  oracle's own Laplace solve, ∂tη_a equals w̃(φ̃_a) and ∂tφ̃_a equals −gη_a (a sign slip in
  φ̃_a fails the first).
* The zones change the right-hand side only at nodes inside them.
* An absorbing zone drains the energy of waves that run into it; without zones the energy
  is conserved.
"""
import math

import numpy as np
import pytest

from oracle import sem
from sem_workloads import (Workload, linear_omega, wavenumber, jonswap_components, c4_shoal,
                           shoal_depth)


def test_gamma_profile():
    x = np.linspace(0, 10, 10001)
    g = sem.relaxation_gamma(x, 0.0, 10.0, 2.0, 3.0)
    assert np.all(g[(x >= 2.0) & (x <= 7.0)] == 1.0)
    assert g[0] == 0.0 and g[-1] == 0.0
    assert np.all(np.diff(g[x <= 2.0]) >= 0) and np.all(np.diff(g[x >= 7.0]) <= 0)
    d = np.gradient(g, x)
    assert abs(d[0]) < 1e-2 and abs(d[np.searchsorted(x, 2.0)]) < 1e-2     # C¹ at both ends of a ramp


def test_generated_signal_solves_linear_equations():
    P, Nx, Nz, h = 8, 4, 2, 1.0
    k = 1.0
    om = linear_omega(k, h)
    edges = np.linspace(0, 2 * math.pi / k, Nx + 1)
    m = sem.Mesh(P, Nx, Nz, edges, True, np.full(Nx * P, h))
    wave = (np.array([0.01]), np.array([om]), np.array([k]), np.array([0.3]))
    t, dt = 0.37, 1e-6
    ea, pa = sem.linear_wave_signal(m.xcol, t, wave, 9.81)
    ea2, pa2 = sem.linear_wave_signal(m.xcol, t + dt, wave, 9.81)
    ea0, pa0 = sem.linear_wave_signal(m.xcol, t - dt, wave, 9.81)
    dedt = (ea2 - ea0) / (2 * dt)
    dpdt = (pa2 - pa0) / (2 * dt)
    z = np.zeros(m.ncol)
    w = m.w_surface(z, m.laplace_solve(z, pa))
    assert np.abs(dedt - w).max() < 1e-6 * np.abs(dedt).max() + 1e-9
    np.testing.assert_allclose(dpdt, -9.81 * ea, atol=1e-8)


def _zone_workload(left, right, wave=None, tau=0.05):
    return Workload(name="zone test", P=4, Nx=12, Nz=1, length=4 * math.pi, periodic=False, depth=1.0,
                    Pf=6, filter_alpha=36.0, filter_s=12.0, filter_ic=3, dt=0.05, init="rest",
                    relax_left=left, relax_right=right, relax_tau=tau, wave=wave)


def test_zones_act_only_inside():
    wl = _zone_workload(2.0, 3.0, wave=(np.array([0.02]), np.array([2.7]), np.array([0.8]), np.array([0.1])))
    m = sem.mesh_for(wl)
    x = m.xcol
    eta = 0.03 * np.cos(x)
    phis = 0.1 * np.sin(x)
    de1, dp1 = m.zakharov_rhs(eta, phis, t=0.4, tau=0.05)
    m0 = sem.mesh_for(_zone_workload(0.0, 0.0))
    de0, dp0 = m0.zakharov_rhs(eta, phis, t=0.4)
    inside = (x < 2.0) | (x > 4 * math.pi - 3.0)
    np.testing.assert_allclose(de1[~inside], de0[~inside], atol=1e-14)
    np.testing.assert_allclose(dp1[~inside], dp0[~inside], atol=1e-14)
    assert np.abs(de1[inside] - de0[inside]).max() > 1e-3


@pytest.mark.slow
def test_absorbing_zones_drain_energy():
    def run(zones):
        wl = _zone_workload(2.5 if zones else 0.0, 2.5 if zones else 0.0, tau=0.0)
        m = sem.mesh_for(wl)
        x = m.xcol
        L = x[-1]
        eta = 0.01 * np.exp(-((x - L / 2) ** 2))          # a hump that splits and runs to both ends
        phis = np.zeros_like(x)
        E0 = m.energy(eta, phis)
        for _ in range(200):
            eta, phis = m.rk4_step(eta, phis, 0.05)
        return m.energy(eta, phis) / E0
    # dispersive short waves reach the zones late, so absorption is partial after 10 s
    assert run(True) < 0.45
    assert abs(run(False) - 1.0) < 0.02


def test_jonswap_and_shoal_inputs():
    wl = c4_shoal()
    a, om, k, th = wl.wave
    assert 4 * math.sqrt(0.5 * np.sum(a * a)) == pytest.approx(2 * 0.05 / 1.5)
    np.testing.assert_allclose(om ** 2, 9.81 * k * np.tanh(k), rtol=1e-12)
    x = np.linspace(0, wl.length, 4001)
    h = shoal_depth(x, wl.length)
    assert h.min() == pytest.approx(0.25) and h.max() == pytest.approx(1.0)
    assert np.abs(np.diff(h) / np.diff(x)).max() <= 0.1 + 1e-9
    assert wavenumber(linear_omega(1.5, 1.0), 1.0) == pytest.approx(1.5)
