"""Oracle, layer 0: one-dimensional polynomial tables in FP64.

TEST INFRASTRUCTURE ONLY.  This package is the plain, slow CPU reference
that the CUDA library is checked against; only the tests, the smoke check
and the benchmark's CPU-baseline leg may import it.  It shares no code,
tables or constants with the CUDA library.

Everything follows the nodal/modal duality of the paper, §3.1.4:

* orthonormal Legendre polynomials P̃_n (the (0,0) Jacobi family of
  eq. (eq_basis)), built from Bonnet's recurrence
  (n+1) P_{n+1} = (2n+1) x P_n − n P_{n−1} and scaled by sqrt((2n+1)/2);
* Gauss–Lobatto–Legendre (GLL) nodes, the roots of (1−r²) P'_P(r);
* the generalised Vandermonde V_ij = P̃_j(r_i) and V_r,ij = P̃'_j(r_i);
* D_r = V_r V⁻¹ (eq. derivative) and the exact mass M = (V Vᵀ)⁻¹
  (eq. massmatrix);
* interpolation to a finer GLL set, I = V_coarse(r_fine) V⁻¹ (§3.3);
* the modal filter F = V̂ S V̂⁻¹ in the boundary/bubble basis of §3.4.
"""
from __future__ import annotations

import math

import numpy as np


def legendre(n_max: int, x) -> tuple[np.ndarray, np.ndarray]:
    """Values and first derivatives of the (unnormalised) Legendre P_0..P_n_max at x.

    Returns arrays of shape (n_max+1, len(x)).  Derivatives use
    P'_{n+1} = P'_{n-1} + (2n+1) P_n.
    """
    x = np.atleast_1d(np.asarray(x, dtype=np.float64))
    p = np.zeros((n_max + 1, x.size))
    dp = np.zeros((n_max + 1, x.size))
    p[0] = 1.0
    if n_max >= 1:
        p[1] = x
        dp[1] = 1.0
    for n in range(1, n_max):
        p[n + 1] = ((2 * n + 1) * x * p[n] - n * p[n - 1]) / (n + 1)
        dp[n + 1] = dp[n - 1] + (2 * n + 1) * p[n]
    return p, dp


def orthonormal_legendre(n_max: int, x) -> tuple[np.ndarray, np.ndarray]:
    """P̃_n = sqrt((2n+1)/2) P_n and its derivative, shape (n_max+1, len(x))."""
    p, dp = legendre(n_max, x)
    s = np.sqrt((2 * np.arange(n_max + 1) + 1) / 2.0)[:, None]
    return p * s, dp * s


def gll_nodes_weights(P: int) -> tuple[np.ndarray, np.ndarray]:
    """GLL nodes (ascending, with ±1) and weights for order P ≥ 1.

    Interior nodes solve P'_P(r)=0 by Newton's method started from the
    Chebyshev–Gauss–Lobatto points; P''_P comes from Legendre's equation
    (1−r²)P'' = 2rP' − P(P+1)P.  Weights are w_j = 2 / (P(P+1) P_P(r_j)²).
    """
    if P < 1:
        raise ValueError("P must be >= 1")
    r = -np.cos(np.pi * np.arange(P + 1) / P)
    inner = r[1:-1].copy()
    for _ in range(100):
        p, dp = legendre(P, inner)
        d2 = (2 * inner * dp[P] - P * (P + 1) * p[P]) / (1 - inner ** 2)
        step = dp[P] / d2
        inner -= step
        if np.max(np.abs(step), initial=0.0) < 1e-16:
            break
    r[1:-1] = inner
    r[0], r[-1] = -1.0, 1.0
    p, _ = legendre(P, r)
    w = 2.0 / (P * (P + 1) * p[P] ** 2)
    return r, w


def vandermonde(P: int, r) -> tuple[np.ndarray, np.ndarray]:
    """V_ij = P̃_j(r_i), V_r,ij = P̃'_j(r_i) for j = 0..P (§3.1.4)."""
    p, dp = orthonormal_legendre(P, r)
    return p.T.copy(), dp.T.copy()


def derivative_matrix(P: int) -> np.ndarray:
    """Nodal differentiation on the GLL nodes, D_r = V_r V⁻¹ (eq. derivative)."""
    r, _ = gll_nodes_weights(P)
    V, Vr = vandermonde(P, r)
    return Vr @ np.linalg.inv(V)


def mass_matrix(P: int) -> np.ndarray:
    """Exact nodal mass on [-1,1]: M = (V Vᵀ)⁻¹ (eq. massmatrix)."""
    r, _ = gll_nodes_weights(P)
    V, _ = vandermonde(P, r)
    return np.linalg.inv(V @ V.T)


def interpolation_matrix(P: int, Pf: int) -> np.ndarray:
    """Interpolation from the order-P GLL nodes to the order-Pf GLL nodes (§3.3)."""
    r, _ = gll_nodes_weights(P)
    rf, _ = gll_nodes_weights(Pf)
    V, _ = vandermonde(P, r)
    Vf, _ = vandermonde(P, rf)          # coarse modes at the fine nodes
    return Vf @ np.linalg.inv(V)


def boundary_bubble_basis(P: int, r) -> np.ndarray:
    """Modal basis of §3.4 at points r, columns j = 0..P.

    φ̂_0 = (1−r)/2, φ̂_1 = (1+r)/2,
    φ̂_{n+1} = ¼ (1−r)(1+r) P^{(1,1)}_{n−1}(r), n = 1..P−1,
    with P^{(1,1)}_{m} = 2/(m+2) · P'_{m+1} (derivative of Legendre).
    """
    r = np.atleast_1d(np.asarray(r, dtype=np.float64))
    out = np.zeros((r.size, P + 1))
    out[:, 0] = 0.5 * (1 - r)
    out[:, 1] = 0.5 * (1 + r)
    if P >= 2:
        _, dp = legendre(P, r)
        for n in range(1, P):
            m = n - 1
            jac11 = 2.0 / (m + 2) * dp[m + 1]
            out[:, n + 1] = 0.25 * (1 - r) * (1 + r) * jac11
    return out


def filter_response(P: int, alpha: float, s: float, ic: int) -> np.ndarray:
    """Modal attenuation σ(i), i = 0..P, for the exponential filter of §3.4.

    Reading of the printed formula: σ(i) = 1 for i ≤ i_c and
    σ(i) = exp(−α ((i − i_c)/(P − i_c))^s) for i_c < i ≤ P; with s = 0 the
    factor is exp(−α) on every mode above i_c.  Mode index = position in the
    boundary/bubble basis (the bubble φ̂_i has degree i).  ic < 0 disables it.
    """
    sig = np.ones(P + 1)
    if ic < 0 or ic >= P:
        return sig
    for i in range(ic + 1, P + 1):
        frac = (i - ic) / (P - ic)
        sig[i] = math.exp(-alpha * (frac ** s if s != 0 else 1.0))
    return sig


def filter_matrix(P: int, alpha: float, s: float, ic: int) -> np.ndarray:
    """F = V̂ S V̂⁻¹ with V̂_ij = φ̂_j(r_i) on the GLL nodes (§3.4)."""
    r, _ = gll_nodes_weights(P)
    Vh = boundary_bubble_basis(P, r)
    S = np.diag(filter_response(P, alpha, s, ic))
    return Vh @ S @ np.linalg.inv(Vh)
