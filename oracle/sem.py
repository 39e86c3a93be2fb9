"""Oracle, layers 1–5: mesh, σ-geometry, Laplace solve, recovery, Zakharov RHS, filter, RK4.

TEST INFRASTRUCTURE ONLY (see ``oracle/__init__.py``).  Plain FP64 numpy,
written in the paper's order and notation; nothing is fused or reordered.

Mesh and numbering.  The x-interval is split into Nx elements (edges
``x_edges``), the σ-interval [0,1] into Nz layers; each element carries the
(P+1)² tensor GLL nodes (§3.1.4).  Global node (ix, iz) — column ix of
Ncol = Nx·P (periodic) or Nx·P+1 (walls), row iz of Nrow = Nz·P+1 counted
from the bottom (iz = Nrow−1 is the free surface) — has id ix·Nrow + iz.
Element (ex, l) maps its local node (a, b) to column (ex·P+a) mod Ncol and
row l·P+b: ``l2g[ex, l, a, b]``.

Readings of the paper taken here (each also listed in the design notes):

1. K is derived from the printed Jacobian (§2, eq. jacobian) as
   K = J Jᵀ / det J, which keeps the ∂x h terms the printed K (flat bottom)
   omits.
2. The stiffness integral of §3.1.2 is evaluated with GLL quadrature at
   the element nodes (symmetric, as the paper states); the mass matrices are
   the exact (V Vᵀ)⁻¹ of eq. (massmatrix).
3. The geometry uses the element-local collocation derivative of d = η + h
   (exact Jacobian of the σ-map interpolated per element); the Zakharov
   right-hand side uses the C⁰ recovered ∂xη, ∂xφ̃ (§3.1.3).
4. The projection for w (eq. velocpot) uses the computational measure
   dx dσ: M is the constant 2D mass and S_z carries ∂zσ = 1/d as a nodal
   factor.
5. Dirichlet data Φ = φ̃ at σ = 1 are imposed by eliminating the surface
   unknowns (lifting), which keeps the system SPD.
6. The semi-discrete free-surface system (eq. semidiscrete) is taken from
   the PDE (eq. FSeqs): ∂tφ̃ = −gη − ½(φ̃x² − w̃²(1+ηx²)); the printed
   matrix form misplaces a sign.
7. Over-integration: the integrands are evaluated at the GLL nodes of
   order P_f from interpolated fields and integrated with the exact order-P_f
   mass (§3.3).
8. Filter: σ(i)=1 for i ≤ i_c, exp(−α((i−i_c)/(P−i_c))^s) above (§3.4);
   applied once after each full RK4 step to η and φ̃.
"""
from __future__ import annotations

from dataclasses import dataclass

import numpy as np
import scipy.sparse as sp

from . import poly
from .banded import BandedCholesky, rcm_order


@dataclass
class Params:
    g: float = 9.81
    Pf: int = 0             # 0: P (no over-integration)
    filter_alpha: float = 0.0
    filter_s: float = 0.0
    filter_ic: int = -1     # -1: no filter
    relax_left: float = 0.0     # length of the generation zone at the left end (0: none)
    relax_right: float = 0.0    # length of the absorption zone at the right end (0: none)
    relax_tau: float = 0.0      # relaxation time τ; 0: the RK4 step size (§2.2 takes τ = Δt)
    wave: tuple | None = None   # (a_i, ω_i, k_i, θ_i) arrays of the generated signal


def relaxation_gamma(x, x0: float, x1: float, left: float, right: float):
    """γ(x) of §2.2: 1 outside the zones, a smooth step ξ²(3−2ξ) from 0 at the outer end of a
    zone to 1 at its inner end (reading: the paper leaves the shape open)."""
    x = np.asarray(x, dtype=np.float64)
    g = np.ones_like(x)
    if left > 0:
        xi = np.clip((x - x0) / left, 0.0, 1.0)
        g = np.where(x < x0 + left, xi * xi * (3 - 2 * xi), g)
    if right > 0:
        xi = np.clip((x1 - x) / right, 0.0, 1.0)
        g = np.where(x > x1 - right, np.minimum(g, xi * xi * (3 - 2 * xi)), g)
    return g


def linear_wave_signal(x, t: float, wave, g: float):
    """Linear superposition at the free surface (§4.2 linear theory per component):
    η_a = Σ a cos(ωt − kx + θ),  φ̃_a = −Σ (g a/ω) sin(ωt − kx + θ)."""
    a, om, k, th = (np.asarray(v, dtype=np.float64) for v in wave)
    ph = np.outer(np.asarray(x, dtype=np.float64), -k) + (om * t + th)[None, :]
    return np.cos(ph) @ a, -(np.sin(ph) @ (g * a / om))


def sigma_K(d, hx, dxd, sig):
    """Coefficient matrix of the σ-transformed Laplacian, K = J Jᵀ / det J.

    J is the Jacobian of (x, z) ↦ (x, σ) from eq. (jacobian):
    J = [[1, 0], [∂xh/d − σ ∂xd/d, 1/d]], with d = η + h.  Returns
    (K11, K12, K22) with the shape of the broadcast inputs.
    """
    d, hx, dxd, sig = np.broadcast_arrays(*(np.asarray(v, dtype=np.float64) for v in (d, hx, dxd, sig)))
    J = np.zeros(d.shape + (2, 2))
    J[..., 0, 0] = 1.0
    J[..., 0, 1] = 0.0
    J[..., 1, 0] = hx / d - sig * dxd / d
    J[..., 1, 1] = 1.0 / d
    detJ = J[..., 0, 0] * J[..., 1, 1] - J[..., 0, 1] * J[..., 1, 0]
    K = np.einsum("...ik,...jk->...ij", J, J) / detJ[..., None, None]
    return K[..., 0, 0], K[..., 0, 1], K[..., 1, 1]


class Mesh:
    """Tensor-product GLL mesh on the σ-domain [x0,x1]×[0,1] (§3.1, §3.1.4)."""

    def __init__(self, P: int, Nx: int, Nz: int, x_edges, periodic: bool, h_col,
                 params: Params | None = None, sigma_edges=None):
        self.P, self.Nx, self.Nz, self.periodic = P, Nx, Nz, bool(periodic)
        self.params = params or Params()
        self.x_edges = np.asarray(x_edges, dtype=np.float64)
        self.sigma_edges = (np.linspace(0.0, 1.0, Nz + 1) if sigma_edges is None
                            else np.asarray(sigma_edges, dtype=np.float64))
        self.ncol = Nx * P if periodic else Nx * P + 1
        self.nrow = Nz * P + 1
        self.n = self.ncol * self.nrow
        self.r, self.w = poly.gll_nodes_weights(P)
        self.D = poly.derivative_matrix(P)
        self.M1 = poly.mass_matrix(P)
        self.dx_e = np.diff(self.x_edges)            # element widths Δx
        self.ds_l = np.diff(self.sigma_edges)        # layer heights Δσ
        a = np.arange(P + 1)
        self.col = (np.arange(Nx)[:, None] * P + a[None, :]) % self.ncol     # (Nx, P+1)
        self.row = np.arange(Nz)[:, None] * P + a[None, :]                    # (Nz, P+1)
        self.l2g = (self.col[:, None, :, None] * self.nrow
                    + self.row[None, :, None, :]).astype(np.int64)           # (Nx,Nz,P+1,P+1)
        ex = np.minimum(np.arange(self.ncol) // P, Nx - 1)
        ax = np.arange(self.ncol) - ex * P
        self.xcol = self.x_edges[ex] + 0.5 * (self.r[ax] + 1) * self.dx_e[ex]
        lz = np.minimum(np.arange(self.nrow) // P, Nz - 1)
        bz = np.arange(self.nrow) - lz * P
        self.sigma_row = self.sigma_edges[lz] + 0.5 * (self.r[bz] + 1) * self.ds_l[lz]
        self.h = np.asarray(h_col, dtype=np.float64)
        if self.h.shape != (self.ncol,):
            raise ValueError("h must have one value per column")
        self.surface = np.arange(self.ncol) * self.nrow + (self.nrow - 1)
        mask = np.ones(self.n, dtype=bool)
        mask[self.surface] = False
        self.interior = np.nonzero(mask)[0]
        self._cache = {}

    # ---- one-dimensional surface operators (§3.1.1, §3.1.3) --------------------------
    def surface_mass(self) -> sp.csr_matrix:
        """M'_ij = ∫ N_i N_j dx, assembled from (Δx/2)·M (eq. massmatrix)."""
        if "Mp" not in self._cache:
            rows, cols, vals = [], [], []
            for ex in range(self.Nx):
                c = self.col[ex]
                rows.append(np.repeat(c, self.P + 1))
                cols.append(np.tile(c, self.P + 1))
                vals.append((0.5 * self.dx_e[ex] * self.M1).ravel())
            Mp = sp.coo_matrix((np.concatenate(vals), (np.concatenate(rows), np.concatenate(cols))),
                               shape=(self.ncol, self.ncol)).tocsr()
            self._cache["Mp"] = Mp
            self._cache["Mp_chol"] = BandedCholesky(Mp)
        return self._cache["Mp"]

    def surface_mass_solve(self, rhs: np.ndarray) -> np.ndarray:
        self.surface_mass()
        return self._cache["Mp_chol"].solve(rhs)

    def surface_gradient(self, f: np.ndarray) -> np.ndarray:
        """C⁰ recovery of ∂x f by M' u = S_x f, S_x,ij = ∫ N_i ∂x N_j dx (§3.1.3).

        Per element S_x = (Δx/2)·M·(2/Δx)·D = M·D.
        """
        rhs = np.zeros(self.ncol)
        for ex in range(self.Nx):
            c = self.col[ex]
            np.add.at(rhs, c, self.M1 @ (self.D @ f[c]))
        return self.surface_mass_solve(rhs)

    # ---- σ-geometry (§2, eqs. sigtrans, jacobian, symTransformedLaplace2) --------------
    def element_K(self, eta: np.ndarray):
        """K = J Jᵀ / det J at every element-local node, arrays (Nx, Nz, P+1, P+1)."""
        P = self.P
        rx = 2.0 / self.dx_e
        d_col = eta + self.h
        eta_e, h_e = eta[self.col], self.h[self.col]                  # (Nx, P+1)
        hx = rx[:, None] * (h_e @ self.D.T)                            # element-local ∂x h
        dxd = rx[:, None] * ((eta_e + h_e) @ self.D.T)                 # element-local ∂x d
        d = d_col[self.col]
        sig = self.sigma_row[self.row]                                 # (Nz, P+1)
        shape = (self.Nx, self.Nz, P + 1, P + 1)
        return sigma_K(np.broadcast_to(d[:, None, :, None], shape),
                       np.broadcast_to(hx[:, None, :, None], shape),
                       np.broadcast_to(dxd[:, None, :, None], shape),
                       np.broadcast_to(sig[None, :, None, :], shape))

    # ---- Laplace operator (§3.1.2) ---------------------------------------------------
    def element_stiffness(self, eta: np.ndarray) -> np.ndarray:
        """Element matrices L^k_ij = −∫ |J^k| (K ∇N_j)·∇N_i dr by GLL quadrature.

        Local index q = a·(P+1) + b; returns (Nx, Nz, Q, Q) with Q = (P+1)².
        """
        P = self.P
        K11, K12, K22 = self.element_K(eta)
        I = np.eye(P + 1)
        Dr = np.kron(self.D, I)            # ∂r acting on the x-index a
        Dt = np.kron(I, self.D)            # ∂t acting on the σ-index b
        wq = np.outer(self.w, self.w).ravel()
        Q = (P + 1) ** 2
        out = np.zeros((self.Nx, self.Nz, Q, Q))
        for ex in range(self.Nx):
            rx = 2.0 / self.dx_e[ex]
            for l in range(self.Nz):
                ts = 2.0 / self.ds_l[l]
                jac = 0.5 * self.dx_e[ex] * 0.5 * self.ds_l[l]
                Gx, Gs = rx * Dr, ts * Dt
                W = wq * jac
                k11, k12, k22 = (K[ex, l].ravel() * W for K in (K11, K12, K22))
                out[ex, l] = -(Gx.T @ (k11[:, None] * Gx) + Gx.T @ (k12[:, None] * Gs)
                               + Gs.T @ (k12[:, None] * Gx) + Gs.T @ (k22[:, None] * Gs))
        return out

    def stiffness(self, eta: np.ndarray) -> sp.csr_matrix:
        """Assembled 𝓛 (n×n, negative semidefinite, no Dirichlet modification)."""
        Le = self.element_stiffness(eta)
        Q = (self.P + 1) ** 2
        g = self.l2g.reshape(self.Nx * self.Nz, Q)
        rows = np.repeat(g, Q, axis=1).ravel()
        cols = np.tile(g, (1, Q)).ravel()
        return sp.coo_matrix((Le.reshape(-1), (rows, cols)), shape=(self.n, self.n)).tocsr()

    def laplace_solve(self, eta: np.ndarray, phis: np.ndarray, return_matrix: bool = False):
        """Φ with 𝓛Φ = 0 at interior nodes and Φ = φ̃ at the surface (eq. laplaceproblemdiscrete).

        Eliminating the surface unknowns gives (−𝓛_II) Φ_I = 𝓛_IB φ̃, solved by
        RCM + banded Cholesky (§3.1.2).
        """
        L = self.stiffness(eta)
        I, B = self.interior, self.surface
        A = -L[I][:, I]
        rhs = L[I][:, B] @ phis
        if "perm_I" not in self._cache:
            self._cache["perm_I"] = rcm_order(A)
        chol = BandedCholesky(A, perm=self._cache["perm_I"])
        Phi = np.empty(self.n)
        Phi[B] = phis
        Phi[I] = chol.solve(rhs)
        return (Phi, L) if return_matrix else Phi

    # ---- vertical velocity at the surface (§3.1.3, eqs. velocpot, velocpot2) ----------
    def mass2d(self) -> sp.csr_matrix:
        """𝓜_ij = ∫ N_i N_j dx dσ, assembled from |J^k| (M ⊗ M)."""
        if "M2" not in self._cache:
            Q = (self.P + 1) ** 2
            M2 = np.kron(self.M1, self.M1)
            g = self.l2g.reshape(self.Nx * self.Nz, Q)
            jac = (0.5 * self.dx_e[:, None] * 0.5 * self.ds_l[None, :]).ravel()
            vals = (jac[:, None, None] * M2[None]).ravel()
            rows = np.repeat(g, Q, axis=1).ravel()
            cols = np.tile(g, (1, Q)).ravel()
            M = sp.coo_matrix((vals, (rows, cols)), shape=(self.n, self.n)).tocsr()
            self._cache["M2"] = M
            self._cache["M2_chol"] = BandedCholesky(M)
        return self._cache["M2"]

    def w_surface(self, eta: np.ndarray, Phi: np.ndarray) -> np.ndarray:
        """w̃ = w at S^FS where 𝓜 w = 𝓢_z Φ, 𝓢_z,ij = ∫ ∂zσ ∂σN_j N_i dx dσ, ∂zσ = 1/d."""
        self.mass2d()
        P = self.P
        I = np.eye(P + 1)
        Dt = np.kron(I, self.D)
        M2 = np.kron(self.M1, self.M1)
        d_col = eta + self.h
        rhs = np.zeros(self.n)
        for ex in range(self.Nx):
            inv_d = np.repeat(1.0 / d_col[self.col[ex]], P + 1)      # nodal 1/d, index a·(P+1)+b
            for l in range(self.Nz):
                g = self.l2g[ex, l].ravel()
                ts = 2.0 / self.ds_l[l]
                jac = 0.5 * self.dx_e[ex] * 0.5 * self.ds_l[l]
                f = inv_d * (ts * (Dt @ Phi[g]))
                np.add.at(rhs, g, jac * (M2 @ f))
        w = self._cache["M2_chol"].solve(rhs)
        return w[self.surface]

    # ---- free-surface right-hand side (§3.1.1, §3.3) ----------------------------------
    def relaxation(self, eta: np.ndarray, phis: np.ndarray, t: float, tau: float):
        """Embedded penalty source of §2.2 at the nodes: (1 − γ)(q_a − q)/τ for q = η, φ̃.
        The left zone relaxes towards the generated signal, the right zone towards rest."""
        prm = self.params
        x0, x1 = self.x_edges[0], self.x_edges[-1]
        gam = relaxation_gamma(self.xcol, x0, x1, prm.relax_left, prm.relax_right)
        ea = np.zeros(self.ncol)
        pa = np.zeros(self.ncol)
        if prm.wave is not None and prm.relax_left > 0:
            left = self.xcol < x0 + prm.relax_left
            ea[left], pa[left] = linear_wave_signal(self.xcol[left], t, prm.wave, prm.g)
        return (1 - gam) * (ea - eta) / tau, (1 - gam) * (pa - phis) / tau

    def zakharov_rhs(self, eta: np.ndarray, phis: np.ndarray, return_parts: bool = False,
                     t: float = 0.0, tau: float | None = None):
        """(∂tη, ∂tφ̃) from the Galerkin form of eq. (FSproblem) with over-integration, plus
        the relaxation source of §2.2 when zones are configured (τ = tau or Params.relax_tau)."""
        prm = self.params
        P = self.P
        Pf = prm.Pf if prm.Pf > 0 else P
        Phi = self.laplace_solve(eta, phis)
        wt = self.w_surface(eta, Phi)
        etax = self.surface_gradient(eta)
        phisx = self.surface_gradient(phis)
        Ip = poly.interpolation_matrix(P, Pf)
        Mf = poly.mass_matrix(Pf)
        rhs_e = np.zeros(self.ncol)
        rhs_p = np.zeros(self.ncol)
        for ex in range(self.Nx):
            c = self.col[ex]
            ef, exf, pxf, wf = (Ip @ v[c] for v in (eta, etax, phisx, wt))
            Fe = -exf * pxf + wf * (1.0 + exf * exf)
            Fp = -prm.g * ef - 0.5 * (pxf * pxf - wf * wf * (1.0 + exf * exf))
            scale = 0.5 * self.dx_e[ex]
            np.add.at(rhs_e, c, scale * (Ip.T @ (Mf @ Fe)))
            np.add.at(rhs_p, c, scale * (Ip.T @ (Mf @ Fp)))
        sol = self.surface_mass_solve(np.stack([rhs_e, rhs_p], axis=1))
        if prm.relax_left > 0 or prm.relax_right > 0:
            tau_ = prm.relax_tau if tau is None else tau
            if not tau_ > 0:
                raise ValueError("relaxation zones need τ > 0")
            se, sp_ = self.relaxation(eta, phis, t, tau_)
            sol = sol + np.stack([se, sp_], axis=1)
        if return_parts:
            return sol[:, 0], sol[:, 1], dict(Phi=Phi, w=wt, etax=etax, phisx=phisx,
                                              rhs_eta=rhs_e, rhs_phi=rhs_p)
        return sol[:, 0], sol[:, 1]

    # ---- modal filter (§3.4) and RK4 (§3.1.1) -------------------------------------
    def apply_filter(self, q: np.ndarray) -> np.ndarray:
        prm = self.params
        if prm.filter_ic < 0:
            return q.copy()
        F = poly.filter_matrix(self.P, prm.filter_alpha, prm.filter_s, prm.filter_ic)
        acc = np.zeros(self.ncol)
        cnt = np.zeros(self.ncol)
        for ex in range(self.Nx):
            c = self.col[ex]
            np.add.at(acc, c, F @ q[c])
            np.add.at(cnt, c, 1.0)
        return acc / cnt

    def rk4_step(self, eta: np.ndarray, phis: np.ndarray, dt: float, t: float = 0.0):
        """Classical four-stage RK4 on (η, φ̃) from time t, then the filter.  The relaxation
        time is Params.relax_tau, or dt when that is 0 (§2.2)."""
        tau = self.params.relax_tau if self.params.relax_tau > 0 else dt
        k1e, k1p = self.zakharov_rhs(eta, phis, t=t, tau=tau)
        k2e, k2p = self.zakharov_rhs(eta + 0.5 * dt * k1e, phis + 0.5 * dt * k1p, t=t + 0.5 * dt, tau=tau)
        k3e, k3p = self.zakharov_rhs(eta + 0.5 * dt * k2e, phis + 0.5 * dt * k2p, t=t + 0.5 * dt, tau=tau)
        k4e, k4p = self.zakharov_rhs(eta + dt * k3e, phis + dt * k3p, t=t + dt, tau=tau)
        eta_n = eta + dt / 6.0 * (k1e + 2 * k2e + 2 * k3e + k4e)
        phis_n = phis + dt / 6.0 * (k1p + 2 * k2p + 2 * k3p + k4p)
        return self.apply_filter(eta_n), self.apply_filter(phis_n)

    # ---- diagnostics -------------------------------------------------------------------
    def mass(self, eta: np.ndarray) -> float:
        """Displaced volume 1ᵀ M' η."""
        return float(np.ones(self.ncol) @ (self.surface_mass() @ eta))

    def energy(self, eta: np.ndarray, phis: np.ndarray) -> float:
        """E = ½ Φᵀ(−𝓛)Φ + ½ g ηᵀ M' η."""
        Phi, L = self.laplace_solve(eta, phis, return_matrix=True)
        return float(0.5 * Phi @ (-(L @ Phi)) + 0.5 * self.params.g * eta @ (self.surface_mass() @ eta))


def mesh_for(wl, h_col=None, bar: bool = False) -> Mesh:
    """Oracle mesh for a workload; bathymetry from ``wl.bathymetry`` unless given."""
    """Build an oracle mesh for a ``sem_workloads.Workload`` (inputs only; no arithmetic shared)."""
    P = wl.P
    r, _ = poly.gll_nodes_weights(P)
    edges = wl.element_edges()
    Ncol = wl.ncol
    ex = np.minimum(np.arange(Ncol) // P, wl.Nx - 1)
    a = np.arange(Ncol) - ex * P
    xcol = edges[ex] + 0.5 * (r[a] + 1) * (edges[ex + 1] - edges[ex])
    if h_col is None:
        from sem_workloads import depth_columns
        h_col = depth_columns(wl, xcol, bar=bar or wl.bathymetry == "bar")
    prm = Params(g=wl.g, Pf=wl.Pf, filter_alpha=wl.filter_alpha, filter_s=wl.filter_s,
                 filter_ic=wl.filter_ic, relax_left=wl.relax_left, relax_right=wl.relax_right,
                 relax_tau=wl.relax_tau, wave=wl.wave)
    return Mesh(P, wl.Nx, wl.Nz, edges, wl.periodic, h_col, prm)
