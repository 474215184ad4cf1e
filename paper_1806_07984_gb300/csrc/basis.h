// One-dimensional nodal operators on the reference interval [0, 1] for the
// ADER-DG kernels, computed on the host in long double and rounded once to
// double (paper Sec. 2.1: Lagrange polynomials over Gauss-Legendre points,
// tensor-product space-time ansatz).
#pragma once

namespace ader {

constexpr int kMaxN = 8;  // nodes per direction (order N <= 7)

// All matrices are row-major [i][j] with n = N + 1 entries per side.
struct BasisTables {
  int n;
  double xi[kMaxN];           // GL nodes on [0, 1]
  double w[kMaxN];            // GL weights (sum 1)
  double D[kMaxN][kMaxN];     // D[i][j] = phi_j'(xi_i)
  double Mt[kMaxN][kMaxN];    // K1^{-1} diag(w): q_k = u - dt sum_l Mt[k][l] div_l
  double V[kMaxN][kMaxN];     // V[i][j] = w_j D[j][i] / w_i (weak volume term)
  double phi0[kMaxN];         // phi_j(0)
  double phi1[kMaxN];         // phi_j(1)
  double lift0[kMaxN];        // phi_i(0) / w_i
  double lift1[kMaxN];        // phi_i(1) / w_i
  double P[3][kMaxN][kMaxN];  // P[s][i][j] = phi_j((s + xi_i) / 3)
  double R[3][kMaxN][kMaxN];  // R[s][i][j] = P[s][j][i] w_j / (3 w_i)
};

// Fills the tables for n = N + 1 nodes (1 <= n <= kMaxN).
void make_basis(int n, BasisTables* out);

constexpr int kMaxS = 2 * kMaxN - 1;  // subcells per direction, S = 2N + 1

// Subcell operators of the a posteriori FV limiter (S = 2N + 1 equal
// subintervals per direction):
//   A[s][j]  mean of phi_j over [s/S, (s+1)/S]   (nodes -> subcell averages)
//   R[i][s]  (A^T A)^-1 A^T                        (averages -> nodes, least squares)
//   Pi[i][s] A[s][i] / (S w_i)                     (subface fluxes -> face nodes, L2)
struct SubcellTables {
  int n, S;
  double A[kMaxS][kMaxN];
  double R[kMaxN][kMaxS];
  double Pi[kMaxN][kMaxS];
};

void make_subcells(int n, SubcellTables* out);

}  // namespace ader
