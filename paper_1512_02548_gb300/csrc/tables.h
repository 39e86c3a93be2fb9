// Host-side one-dimensional tables for the nodal spectral element method
// (§3.1.4, §3.3, §3.4 of arXiv 1512.02548), computed in long double and stored
// as double.  Row-major matrices.
#pragma once
#include <vector>

namespace semgb {

struct Line {
  int P = 0;
  std::vector<double> r, w;  // GLL nodes (ascending) and weights, P+1
  std::vector<double> D;     // (P+1)²: D[i*(P+1)+j] = l_j'(r_i)
  std::vector<double> M;     // (P+1)²: exact mass ∫ l_i l_j on [-1,1]
};

// GLL nodes/weights, differentiation and exact mass of order P (1 ≤ P ≤ 24).
Line make_line(int P);

// Lagrange basis of the order-P GLL nodes evaluated at points x: out[q*(P+1)+j].
std::vector<double> lagrange_at(const Line& L, const std::vector<double>& x);

// Interpolation matrix from order-P to order-Pf GLL nodes, (Pf+1)×(P+1).
std::vector<double> interpolation(const Line& coarse, const Line& fine);

// Per-element modal filter F = V̂ S V̂⁻¹ in the boundary/bubble basis (§3.4), (P+1)².
std::vector<double> filter_matrix(const Line& L, double alpha, double s, int ic);

// Dense inverse (Gauss–Jordan with partial pivoting); returns false if singular.
bool invert(std::vector<long double>& a, int n);

// Eigen-decomposition of a symmetric n×n matrix (cyclic Jacobi rotations): on return
// evals[k] ascending and evecs[i*n+k] the orthonormal eigenvector k.
void sym_eig(std::vector<long double> a, int n, std::vector<long double>& evals,
             std::vector<long double>& evecs);

}  // namespace semgb
