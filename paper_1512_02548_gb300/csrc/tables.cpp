// One-dimensional GLL tables (§3.1.4, §3.3, §3.4), computed on the host.
//
// Formulation (chosen for accuracy in long double):
//  * GLL nodes: Newton iteration on q(x) = P_{P+1}(x) − P_{P−1}(x), whose zeros are
//    ±1 and the zeros of P'_P, from Chebyshev–Gauss–Lobatto starts;
//    weights w_j = 2 / (P(P+1) P_P(x_j)²).
//  * Differentiation: the closed form of the Lagrange-derivative matrix on GLL
//    nodes, D_ij = P_P(x_i)/(P_P(x_j)(x_i − x_j)) (i ≠ j), D_00 = −P(P+1)/4,
//    D_PP = P(P+1)/4, other diagonal entries 0 — the nodal form of D_r = V_r V⁻¹.
//  * Exact mass M_ij = ∫ l_i l_j, evaluated with a (P+2)-point Gauss–Legendre rule
//    (exact for degree 2P) — the same matrix as (V Vᵀ)⁻¹ of eq. (massmatrix).
//  * Filter: V̂ S V̂⁻¹ with the boundary/bubble modes of §3.4.
#include "tables.h"

#include <cmath>
#include <stdexcept>

namespace semgb {

namespace {

using ld = long double;

// Legendre P_0..P_n at x; returns P_n and fills pm1 = P_{n-1}.
ld legendre(int n, ld x, ld* pm1) {
  ld p0 = 1.0L, p1 = x;
  if (n == 0) { if (pm1) *pm1 = 0.0L; return p0; }
  for (int k = 1; k < n; ++k) {
    ld p2 = ((2 * k + 1) * x * p1 - k * p0) / (k + 1);
    p0 = p1;
    p1 = p2;
  }
  if (pm1) *pm1 = p0;
  return p1;
}

ld legendre_deriv(int n, ld x) {
  // P'_n = n (x P_n − P_{n−1}) / (x² − 1) away from ±1
  ld pm1;
  ld p = legendre(n, x, &pm1);
  return n * (x * p - pm1) / (x * x - 1.0L);
}

void gauss_legendre(int N, std::vector<ld>& x, std::vector<ld>& w) {
  x.assign(N, 0.0L);
  w.assign(N, 0.0L);
  const ld pi = 3.141592653589793238462643383279502884L;
  for (int i = 0; i < N; ++i) {
    ld xi = -std::cos(pi * (i + 0.75L) / (N + 0.5L));
    for (int it = 0; it < 100; ++it) {
      ld d = legendre_deriv(N, xi);
      ld dx = legendre(N, xi, nullptr) / d;
      xi -= dx;
      if (std::fabs(dx) < 1e-19L) break;
    }
    ld d = legendre_deriv(N, xi);
    x[i] = xi;
    w[i] = 2.0L / ((1.0L - xi * xi) * d * d);
  }
}

std::vector<ld> gll_nodes(int P) {
  std::vector<ld> x(P + 1);
  const ld pi = 3.141592653589793238462643383279502884L;
  for (int j = 0; j <= P; ++j) x[j] = -std::cos(pi * j / P);
  for (int j = 1; j < P; ++j) {
    ld xi = x[j];
    for (int it = 0; it < 100; ++it) {
      // q = P_{P+1} − P_{P−1};  q' = (2P+1) P_P
      ld pPm1;
      ld pP = legendre(P, xi, &pPm1);
      ld pP1 = ((2 * P + 1) * xi * pP - P * pPm1) / (P + 1);
      ld q = pP1 - pPm1;
      ld dq = (2 * P + 1) * pP;
      ld dx = q / dq;
      xi -= dx;
      if (std::fabs(dx) < 1e-19L) break;
    }
    x[j] = xi;
  }
  x[0] = -1.0L;
  x[P] = 1.0L;
  return x;
}

// Lagrange basis l_j of `nodes` at point t.
void lagrange(const std::vector<ld>& nodes, ld t, std::vector<ld>& out) {
  int n = static_cast<int>(nodes.size());
  out.assign(n, 1.0L);
  for (int j = 0; j < n; ++j)
    for (int k = 0; k < n; ++k)
      if (k != j) out[j] *= (t - nodes[k]) / (nodes[j] - nodes[k]);
}

std::vector<ld> to_ld(const std::vector<double>& v) { return std::vector<ld>(v.begin(), v.end()); }

}  // namespace

bool invert(std::vector<ld>& a, int n) {
  std::vector<ld> inv(n * n, 0.0L);
  for (int i = 0; i < n; ++i) inv[i * n + i] = 1.0L;
  for (int c = 0; c < n; ++c) {
    int piv = c;
    for (int r = c + 1; r < n; ++r)
      if (std::fabs(a[r * n + c]) > std::fabs(a[piv * n + c])) piv = r;
    if (std::fabs(a[piv * n + c]) < 1e-300L) return false;
    if (piv != c)
      for (int k = 0; k < n; ++k) {
        std::swap(a[c * n + k], a[piv * n + k]);
        std::swap(inv[c * n + k], inv[piv * n + k]);
      }
    ld s = 1.0L / a[c * n + c];
    for (int k = 0; k < n; ++k) { a[c * n + k] *= s; inv[c * n + k] *= s; }
    for (int r = 0; r < n; ++r) {
      if (r == c) continue;
      ld f = a[r * n + c];
      if (f == 0.0L) continue;
      for (int k = 0; k < n; ++k) {
        a[r * n + k] -= f * a[c * n + k];
        inv[r * n + k] -= f * inv[c * n + k];
      }
    }
  }
  a.swap(inv);
  return true;
}

void sym_eig(std::vector<ld> a, int n, std::vector<ld>& evals, std::vector<ld>& evecs) {
  std::vector<ld> v((size_t)n * n, 0.0L);
  for (int i = 0; i < n; ++i) v[(size_t)i * n + i] = 1.0L;
  for (int sweep = 0; sweep < 100; ++sweep) {
    ld off = 0.0L, diag = 0.0L;
    for (int i = 0; i < n; ++i)
      for (int j = 0; j < n; ++j)
        (i == j ? diag : off) += a[(size_t)i * n + j] * a[(size_t)i * n + j];
    if (off <= 1e-36L * diag) break;
    for (int p = 0; p < n - 1; ++p)
      for (int q = p + 1; q < n; ++q) {
        const ld apq = a[(size_t)p * n + q];
        if (std::fabs(apq) < 1e-300L) continue;
        const ld app = a[(size_t)p * n + p], aqq = a[(size_t)q * n + q];
        const ld theta = (aqq - app) / (2.0L * apq);
        const ld t = (theta >= 0 ? 1.0L : -1.0L) / (std::fabs(theta) + std::sqrt(theta * theta + 1.0L));
        const ld c = 1.0L / std::sqrt(t * t + 1.0L), sn = t * c;
        for (int k = 0; k < n; ++k) {   // A ← A J (columns p, q)
          const ld akp = a[(size_t)k * n + p], akq = a[(size_t)k * n + q];
          a[(size_t)k * n + p] = c * akp - sn * akq;
          a[(size_t)k * n + q] = sn * akp + c * akq;
        }
        for (int k = 0; k < n; ++k) {   // A ← Jᵀ A (rows p, q)
          const ld apk = a[(size_t)p * n + k], aqk = a[(size_t)q * n + k];
          a[(size_t)p * n + k] = c * apk - sn * aqk;
          a[(size_t)q * n + k] = sn * apk + c * aqk;
        }
        for (int k = 0; k < n; ++k) {   // V ← V J
          const ld vkp = v[(size_t)k * n + p], vkq = v[(size_t)k * n + q];
          v[(size_t)k * n + p] = c * vkp - sn * vkq;
          v[(size_t)k * n + q] = sn * vkp + c * vkq;
        }
      }
  }
  std::vector<int> order(n);
  for (int i = 0; i < n; ++i) order[i] = i;
  for (int i = 0; i < n; ++i)
    for (int j = i + 1; j < n; ++j)
      if (a[(size_t)order[j] * n + order[j]] < a[(size_t)order[i] * n + order[i]]) std::swap(order[i], order[j]);
  evals.resize(n);
  evecs.assign((size_t)n * n, 0.0L);
  for (int k = 0; k < n; ++k) {
    evals[k] = a[(size_t)order[k] * n + order[k]];
    for (int i = 0; i < n; ++i) evecs[(size_t)i * n + k] = v[(size_t)i * n + order[k]];
  }
}

Line make_line(int P) {
  if (P < 1 || P > 24) throw std::invalid_argument("GLL order out of range");
  Line L;
  L.P = P;
  const int n = P + 1;
  std::vector<ld> x = gll_nodes(P);
  std::vector<ld> pP(n);
  for (int j = 0; j < n; ++j) pP[j] = legendre(P, x[j], nullptr);
  L.r.resize(n);
  L.w.resize(n);
  for (int j = 0; j < n; ++j) {
    L.r[j] = static_cast<double>(x[j]);
    L.w[j] = static_cast<double>(2.0L / (P * (P + 1) * pP[j] * pP[j]));
  }
  L.D.assign(n * n, 0.0);
  for (int i = 0; i < n; ++i)
    for (int j = 0; j < n; ++j) {
      ld v;
      if (i != j) v = pP[i] / (pP[j] * (x[i] - x[j]));
      else if (i == 0) v = -(ld)P * (P + 1) / 4.0L;
      else if (i == P) v = (ld)P * (P + 1) / 4.0L;
      else v = 0.0L;
      L.D[i * n + j] = static_cast<double>(v);
    }
  std::vector<ld> gx, gw;
  gauss_legendre(P + 2, gx, gw);
  std::vector<ld> Mm(n * n, 0.0L), lv;
  for (size_t q = 0; q < gx.size(); ++q) {
    lagrange(x, gx[q], lv);
    for (int i = 0; i < n; ++i)
      for (int j = 0; j < n; ++j) Mm[i * n + j] += gw[q] * lv[i] * lv[j];
  }
  L.M.resize(n * n);
  for (int k = 0; k < n * n; ++k) L.M[k] = static_cast<double>(Mm[k]);
  return L;
}

std::vector<double> lagrange_at(const Line& L, const std::vector<double>& xq) {
  std::vector<ld> nodes = to_ld(L.r), lv;
  const int n = L.P + 1;
  std::vector<double> out(xq.size() * n);
  for (size_t q = 0; q < xq.size(); ++q) {
    lagrange(nodes, xq[q], lv);
    for (int j = 0; j < n; ++j) out[q * n + j] = static_cast<double>(lv[j]);
  }
  return out;
}

std::vector<double> interpolation(const Line& coarse, const Line& fine) {
  return lagrange_at(coarse, fine.r);
}

std::vector<double> filter_matrix(const Line& L, double alpha, double s, int ic) {
  const int P = L.P, n = P + 1;
  std::vector<double> F(n * n, 0.0);
  if (ic < 0 || ic >= P) {
    for (int i = 0; i < n; ++i) F[i * n + i] = 1.0;
    return F;
  }
  // V̂_ij = φ̂_j(r_i): hats (1∓r)/2 and bubbles ¼(1−r)(1+r)P^{(1,1)}_{j−2}(r); the bubble
  // scale does not affect F, so P^{(1,1)}_{m} is taken as P'_{m+1} (a multiple of it).
  std::vector<ld> V(n * n), Vi;
  for (int i = 0; i < n; ++i) {
    ld r = L.r[i];
    V[i * n + 0] = 0.5L * (1 - r);
    V[i * n + 1] = 0.5L * (1 + r);
    for (int j = 2; j <= P; ++j) {
      ld dP;
      if (i == 0 || i == P) dP = 0.0L;  // the bubble vanishes at ±1 whatever P'
      else dP = legendre_deriv(j - 1, r);
      V[i * n + j] = 0.25L * (1 - r) * (1 + r) * dP;
    }
  }
  Vi = V;
  if (!invert(Vi, n)) throw std::runtime_error("filter Vandermonde is singular");
  std::vector<ld> sig(n, 1.0L);
  for (int i = ic + 1; i <= P; ++i) {
    ld frac = (ld)(i - ic) / (ld)(P - ic);
    ld e = (s != 0.0) ? std::pow(frac, (ld)s) : 1.0L;
    sig[i] = std::exp(-(ld)alpha * e);
  }
  for (int i = 0; i < n; ++i)
    for (int j = 0; j < n; ++j) {
      ld acc = 0.0L;
      for (int k = 0; k < n; ++k) acc += V[i * n + k] * sig[k] * Vi[k * n + j];
      F[i * n + j] = static_cast<double>(acc);
    }
  return F;
}

}  // namespace semgb
