"""Seeded synthetic workloads for the σ-transformed SEM wave model.

This module only builds inputs: mesh parameters, still-water depth h(x) at
the mesh columns, and initial free-surface states (η, φ̃).  It holds none of
the method's arithmetic (no basis, no operator, no solver), so both the CPU
oracle and the CUDA library can be fed from it without sharing code.

Node layout used by every array here: the mesh has ``Ncol`` columns
(``Nx*P`` when periodic, ``Nx*P+1`` between walls); column ``ix`` sits at
the GLL node ``a = ix - P*ex`` of x-element ``ex``.  Column positions are
returned by :func:`column_x`, which needs the GLL nodes and therefore takes
them as an argument (callers pass their own).

Workloads (paper §4.2 linear theory, §4.3 steep waves, §5.3 bar):

* ``c1_linear_standing`` – L=2π, h=1, 4×1 elements, P=4, H/L=0.001,
  η=(H/2)cos x, φ̃=0, dt=T/64, one period.
* ``c2_steep_periodic`` – L=2π, h=1, 64×4 elements, P=6, H/L=0.08,
  η=(H/2)cos x+(kH²/8)cos 2x, φ̃ from linear theory at z=η, dt=T/200,
  over-integration P_f=⌈3P/2⌉, filter (α,s,i_c)=(36,12,P-1).
* ``c3_instances`` – 512 periodic tanks from splitmix64(seed 0).
* ``c5_requests`` – Poisson request stream (Laplace solves and short RK4 runs) for the
  serving loop.
* ``roofline_tank`` – one long periodic tank (Nx=65536, Nz=4, P=6) for
  HBM-bound operator measurements.
"""
from __future__ import annotations

import math
from dataclasses import dataclass, field, asdict

import numpy as np

G_EARTH = 9.81


def linear_omega(k: float, h: float, g: float = G_EARTH) -> float:
    """Angular frequency from the linear dispersion relation ω² = g k tanh(kh) (§4.2)."""
    return math.sqrt(g * k * math.tanh(k * h))


@dataclass
class Workload:
    name: str
    P: int
    Nx: int
    Nz: int
    length: float
    periodic: bool
    depth: float
    g: float = G_EARTH
    Pf: int = 0                 # over-integration order; 0 means P (none)
    filter_alpha: float = 0.0
    filter_s: float = 0.0
    filter_ic: int = -1         # -1: no filter
    dt: float = 0.0
    nsteps: int = 0
    wave_height: float = 0.0
    wavenumber: float = 1.0
    init: str = "progressive"   # "standing": η=(H/2)cos kx, φ̃=0; "rest": η=φ̃=0
    bathymetry: str = "flat"    # "flat", "bar" (raised cosine) or "shoal" (trapezoidal bar)
    relax_left: float = 0.0     # generation zone length at the left end
    relax_right: float = 0.0    # absorption zone length at the right end
    relax_tau: float = 0.0      # 0: τ = dt
    wave: tuple | None = None   # generated signal components (a, ω, k, θ)
    extra: dict = field(default_factory=dict)

    @property
    def ncol(self) -> int:
        return self.Nx * self.P if self.periodic else self.Nx * self.P + 1

    @property
    def nrow(self) -> int:
        return self.Nz * self.P + 1

    @property
    def n_nodes(self) -> int:
        return self.ncol * self.nrow

    @property
    def n_unknowns(self) -> int:
        return self.ncol * (self.nrow - 1)

    def element_edges(self) -> np.ndarray:
        return np.linspace(0.0, self.length, self.Nx + 1)

    def as_dict(self) -> dict:
        d = asdict(self)
        d["ncol"], d["nrow"] = self.ncol, self.nrow
        return d


def column_x(wl: Workload, gll_nodes: np.ndarray, edges: np.ndarray | None = None) -> np.ndarray:
    """x-coordinate of each mesh column, given the caller's GLL nodes on [-1, 1]."""
    if edges is None:
        edges = wl.element_edges()
    P = wl.P
    ix = np.arange(wl.ncol)
    ex = np.minimum(ix // P, wl.Nx - 1)
    a = ix - ex * P
    x0, x1 = edges[ex], edges[ex + 1]
    return x0 + 0.5 * (np.asarray(gll_nodes)[a] + 1.0) * (x1 - x0)


def c1_linear_standing() -> Workload:
    k, h = 1.0, 1.0
    T = 2 * math.pi / linear_omega(k, h)
    return Workload(name="C1 linear standing wave 4x1 P=4", P=4, Nx=4, Nz=1,
                    length=2 * math.pi, periodic=True, depth=h, dt=T / 64, nsteps=64,
                    wave_height=0.001 * 2 * math.pi, wavenumber=k, init="standing")


def c2_steep_periodic() -> Workload:
    k, h, P = 1.0, 1.0, 6
    T = 2 * math.pi / linear_omega(k, h)
    return Workload(name="C2 steep periodic wave 64x4 P=6", P=P, Nx=64, Nz=4,
                    length=2 * math.pi, periodic=True, depth=h,
                    Pf=(3 * P + 1) // 2, filter_alpha=36.0, filter_s=12.0, filter_ic=P - 1,
                    dt=T / 200, nsteps=20000, wave_height=0.08 * 2 * math.pi, wavenumber=k)


def roofline_tank(Nx: int = 65536, Nz: int = 4, P: int = 6) -> Workload:
    k, h = 1.0, 1.0
    T = 2 * math.pi / linear_omega(k, h)
    return Workload(name=f"long periodic tank {Nx}x{Nz} P={P}", P=P, Nx=Nx, Nz=Nz,
                    length=2 * math.pi * Nx / 64, periodic=True, depth=h,
                    Pf=(3 * P + 1) // 2, filter_alpha=36.0, filter_s=12.0, filter_ic=P - 1,
                    dt=T / 200, nsteps=1, wave_height=0.04 * 2 * math.pi, wavenumber=k)


def small_case(P: int = 5, Nx: int = 6, Nz: int = 2, periodic: bool = True,
               H_over_L: float = 0.05, Pf: int | None = None, filt: bool = True) -> Workload:
    """A small steep-wave tank that spans several elements and layers (parity cases)."""
    k, h = 1.0, 1.0
    T = 2 * math.pi / linear_omega(k, h)
    return Workload(name=f"small {Nx}x{Nz} P={P} {'periodic' if periodic else 'walls'}",
                    P=P, Nx=Nx, Nz=Nz, length=2 * math.pi, periodic=periodic, depth=h,
                    Pf=(3 * P + 1) // 2 if Pf is None else Pf,
                    filter_alpha=36.0 if filt else 0.0, filter_s=12.0 if filt else 0.0,
                    filter_ic=(P - 1) if filt else -1,
                    dt=T / 100, nsteps=2, wave_height=H_over_L * 2 * math.pi, wavenumber=k)


def _smooth_ramp(s: np.ndarray, delta: float) -> np.ndarray:
    """clamp(s, 0, 1) with C¹ quadratic blends of half-width delta at both corners."""
    out = np.clip(s, 0.0, 1.0)
    lo = np.abs(s) < delta
    out = np.where(lo, (s + delta) ** 2 / (4 * delta), out)
    hi = np.abs(s - 1.0) < delta
    out = np.where(hi, 1.0 - (1.0 + delta - s) ** 2 / (4 * delta), out)
    return out


def shoal_depth(x: np.ndarray, length: float, depth: float = 1.0, crest: float = 0.25,
                up_slope: float = 1 / 20, down_slope: float = 1 / 10, blend: float = 0.5) -> np.ndarray:
    """Trapezoidal bar in the middle third: rises from `depth` to `crest` at `up_slope`, stays
    at the crest, falls back at `down_slope`; corners smoothed over `blend` metres (C¹)."""
    x = np.asarray(x, dtype=np.float64)
    rise = depth - crest
    xa = length / 3.0
    run_up, run_dn = rise / up_slope, rise / down_slope
    xb = 2.0 * length / 3.0 - run_dn
    up = _smooth_ramp((x - xa) / run_up, 0.5 * blend / run_up)
    dn = _smooth_ramp((x - xb) / run_dn, 0.5 * blend / run_dn)
    return depth - rise * (up - dn)


def depth_columns(wl: Workload, xcol: np.ndarray, bar: bool = False) -> np.ndarray:
    """Still-water depth at each column: constant, or a smooth submerged bar.

    The bar (used for variable-bathymetry cases) rises from ``depth`` to
    ``depth/4`` over the middle third of the tank with a raised-cosine
    profile, so h and h_x are smooth.
    """
    h = np.full_like(xcol, wl.depth, dtype=np.float64)
    if wl.bathymetry == "shoal":
        return shoal_depth(xcol, wl.length, wl.depth)
    if bar:
        L = wl.length
        x0, x1 = L / 3, 2 * L / 3
        s = np.clip((xcol - x0) / (x1 - x0), 0.0, 1.0)
        h = wl.depth - 0.75 * wl.depth * 0.5 * (1 - np.cos(2 * math.pi * s)) * (s > 0) * (s < 1)
    return h


def initial_state(wl: Workload, xcol: np.ndarray, h: np.ndarray | None = None):
    """Initial (η, φ̃) at the columns.

    ``init == "standing"``: η=(H/2)cos kx, φ̃=0.
    Otherwise: η=(H/2)cos kx + (kH²/8)cos 2kx and φ̃ from linear theory of a
    progressive wave evaluated at z=η:
    φ̃ = (gH/2ω)·cosh(k(η+h))/cosh(kh)·sin kx.
    """
    k, H = wl.wavenumber, wl.wave_height
    if h is None:
        h = np.full_like(xcol, wl.depth, dtype=np.float64)
    if wl.init == "standing":
        eta = 0.5 * H * np.cos(k * xcol)
        return eta, np.zeros_like(eta)
    if wl.init == "rest":
        return np.zeros_like(xcol, dtype=np.float64), np.zeros_like(xcol, dtype=np.float64)
    eta = 0.5 * H * np.cos(k * xcol) + (k * H * H / 8.0) * np.cos(2 * k * xcol)
    om = linear_omega(k, wl.depth, wl.g)
    phis = (wl.g * H / (2 * om)) * np.cosh(k * (eta + h)) / np.cosh(k * wl.depth) * np.sin(k * xcol)
    return eta, phis


# --- splitmix64: counter-based generator for instance lists (Steele, Lea & Flood 2014) ---
_MASK = (1 << 64) - 1


def splitmix64(seed: int):
    state = seed & _MASK
    while True:
        state = (state + 0x9E3779B97F4A7C15) & _MASK
        z = state
        z = ((z ^ (z >> 30)) * 0xBF58476D1CE4E5B9) & _MASK
        z = ((z ^ (z >> 27)) * 0x94D049BB133111EB) & _MASK
        yield z ^ (z >> 31)


def _uniform(gen) -> float:
    return (next(gen) >> 11) * (1.0 / (1 << 53))


def stable_dt(T: float, P: int, Nx: int, length: float, depth: float, H: float, k: float) -> float:
    """Explicit RK4 step for a periodic tank: min(T/200, dt_grav, dt_adv).

    Short gravity waves on the smallest GLL spacing Δx_min ≈ (Δx_e/2)(1 − cos π/P) have
    ω_max = (g π/Δx_min)^½, and RK4 needs ω_max dt ≤ 2.8 on the imaginary axis: dt_grav takes
    half of that.  The nonlinear terms advect with the surface velocity
    u_max = (g H k/2ω) cosh(k(h + η_max))/cosh(kh) (linear theory at the crest, 20% margin):
    dt_adv = Δx_min/(2 u_max), a Courant number of ½ on the finest spacing."""
    dx_min = 0.5 * (length / Nx) * (1 - math.cos(math.pi / P))
    om = linear_omega(k, depth)
    u_max = 1.2 * (G_EARTH * H * k / (2 * om)) * math.cosh(k * (depth + H / 2 + k * H * H / 8)) / math.cosh(k * depth)
    return min(T / 200, 0.5 * 2.8 / math.sqrt(G_EARTH * math.pi / dx_min), 0.5 * dx_min / u_max)


def c3_instances(count: int = 512, seed: int = 0) -> list[Workload]:
    """Uneven periodic tanks: Nx∈[16,128], Nz∈{1,2,4}, P∈{4..8}, kh∈[0.5,3], H/L∈[0.01,0.09];
    step stable_dt."""
    gen = splitmix64(seed)
    out = []
    for i in range(count):
        Nx = 16 + int(_uniform(gen) * 113)
        Nz = (1, 2, 4)[int(_uniform(gen) * 3)]
        P = 4 + int(_uniform(gen) * 5)
        kh = 0.5 + 2.5 * _uniform(gen)
        HL = 0.01 + 0.08 * _uniform(gen)
        k = 1.0
        h = kh / k
        T = 2 * math.pi / linear_omega(k, h)
        H = HL * 2 * math.pi / k
        out.append(Workload(name=f"C3 tank {i}", P=P, Nx=Nx, Nz=Nz, length=2 * math.pi / k,
                            periodic=True, depth=h, Pf=(3 * P + 1) // 2,
                            filter_alpha=36.0, filter_s=12.0, filter_ic=P - 1,
                            dt=stable_dt(T, P, Nx, 2 * math.pi / k, h, H, k), nsteps=1, wave_height=H,
                            wavenumber=k))
    return out


def wavenumber(omega: float, h: float, g: float = G_EARTH) -> float:
    """k with ω² = g k tanh(kh), by Newton's method."""
    k = omega * omega / g / math.sqrt(math.tanh(omega * omega * h / g))
    for _ in range(60):
        th = math.tanh(k * h)
        f = g * k * th - omega * omega
        df = g * th + g * k * h * (1 - th * th)
        dk = f / df
        k -= dk
        if abs(dk) < 1e-15 * k:
            break
    return k


def jonswap_components(omega_p: float, Hs: float, n: int = 256, lo: float = 0.6, hi: float = 3.0,
                       gamma: float = 3.3, sigma_a: float = 0.07, sigma_b: float = 0.09,
                       depth: float = 1.0, seed: int = 0, g: float = G_EARTH):
    """Components (a_i, ω_i, k_i, θ_i) of a JONSWAP sea (Hasselmann et al. 1973 shape) on a
    uniform ω grid in [lo·ω_p, hi·ω_p]; amplitudes √(2SΔω) rescaled so that 4√m0 = Hs, phases
    uniform in [0, 2π) from splitmix64(seed), wavenumbers from the linear dispersion relation."""
    dw = (hi - lo) * omega_p / n
    om = lo * omega_p + (np.arange(n) + 0.5) * dw
    sig = np.where(om <= omega_p, sigma_a, sigma_b)
    S = om ** -5 * np.exp(-1.25 * (omega_p / om) ** 4) * gamma ** np.exp(-((om - omega_p) ** 2) / (2 * sig ** 2 * omega_p ** 2))
    a = np.sqrt(2 * S * dw)
    m0 = 0.5 * np.sum(a * a)
    a *= Hs / (4 * math.sqrt(m0))
    gen = splitmix64(seed)
    th = np.array([2 * math.pi * _uniform(gen) for _ in range(n)])
    k = np.array([wavenumber(w, depth, g) for w in om])
    return a, om, k, th


def c4_shoal(Nx: int = 2048, Nz: int = 2, P: int = 6, n_comp: int = 256, nsteps: int = 5000) -> Workload:
    """Irregular waves over a synthetic shoal: tank of 50 peak wavelengths (k_p h = 1.5),
    walls, trapezoidal bar to h = 0.25 in the middle third, JONSWAP (γ = 3.3, Hs k_p/2 = 0.05)
    generated in a 2L_p zone on the left and absorbed in a 2L_p zone on the right; dt from a
    Courant number 0.5 on the element length."""
    h, kp = 1.0, 1.5
    om_p = linear_omega(kp, h)
    Lp = 2 * math.pi / kp
    L = 50 * Lp
    Hs = 2 * 0.05 / kp
    cp = om_p / kp
    dx_e = L / Nx
    wave = jonswap_components(om_p, Hs, n=n_comp, depth=h)
    return Workload(name=f"C4 JONSWAP over shoal {Nx}x{Nz} P={P}", P=P, Nx=Nx, Nz=Nz, length=L,
                    periodic=False, depth=h, Pf=(3 * P + 1) // 2, filter_alpha=36.0, filter_s=12.0,
                    filter_ic=P - 1, dt=0.5 * dx_e / cp, nsteps=nsteps, wave_height=Hs, wavenumber=kp,
                    init="rest", bathymetry="shoal", relax_left=2 * Lp, relax_right=2 * Lp, wave=wave)


def c5_requests(rate: float, count: int = 2000, seed: int = 0, nmin: float = 1e3, nmax: float = 2e5,
                nsteps: int = 10) -> list[tuple[str, float, Workload, int]]:
    """Request stream for the serving loop: Poisson arrivals at ``rate`` per second, half
    Laplace solves and half ``nsteps``-step RK4 runs, on periodic tanks whose node count is
    log-uniform in [nmin, nmax]: P∈{4..10}, Nz∈{1,2,4}, Nx = max(2, round(n/(P(Nz·P+1)))),
    kh∈[0.5,3] and H/L∈[0.01,0.09] as for the uneven batch.  Returns (kind, arrival s,
    workload, steps) sorted by arrival.

    The step is stable_dt (T/200, bounded by RK4 stability on the finest GLL spacing)."""
    gen = splitmix64(seed)
    t = 0.0
    out = []
    for i in range(count):
        t += -math.log(1.0 - _uniform(gen)) / rate
        kind = "laplace" if _uniform(gen) < 0.5 else "rk4"
        n = math.exp(math.log(nmin) + _uniform(gen) * (math.log(nmax) - math.log(nmin)))
        P = 4 + int(_uniform(gen) * 7)
        Nz = (1, 2, 4)[int(_uniform(gen) * 3)]
        Nx = max(2, int(round(n / (P * (Nz * P + 1)))))
        kh = 0.5 + 2.5 * _uniform(gen)
        HL = 0.01 + 0.08 * _uniform(gen)
        k = 1.0
        T = 2 * math.pi / linear_omega(k, kh / k)
        H = HL * 2 * math.pi / k
        wl = Workload(name=f"C5 request {i}", P=P, Nx=Nx, Nz=Nz, length=2 * math.pi / k, periodic=True,
                      depth=kh / k, Pf=(3 * P + 1) // 2, filter_alpha=36.0, filter_s=12.0, filter_ic=P - 1,
                      dt=stable_dt(T, P, Nx, 2 * math.pi / k, kh / k, H, k), nsteps=nsteps if kind == "rk4" else 0,
                      wave_height=H, wavenumber=k)
        out.append((kind, t, wl, nsteps if kind == "rk4" else 0))
    return out


def random_field(n: int, seed: int) -> np.ndarray:
    """Seeded standard-normal vector (parity inputs for operator applies)."""
    return np.random.default_rng(seed).standard_normal(n)
