// Host construction of the nodal operators in long double.
//
// * Gauss-Legendre nodes: Newton iteration on the three-term recurrence of the
//   Legendre polynomial P_n on [-1, 1], started from the Chebyshev-like guess
//   cos(pi (i + 3/4) / (n + 1/2)); weights 2 / ((1 - x^2) P_n'(x)^2); mapped to
//   [0, 1].
// * D by the barycentric formula with the negative-sum diagonal.
// * K1_kl = theta_k(1) theta_l(1) - w_l D_lk (time-weak form with upwind
//   inflow), inverted by Gauss-Jordan elimination with partial pivoting.
#include "basis.h"

#include <cmath>

namespace ader {

namespace {

typedef long double ld;

void legendre(int n, ld x, ld* p, ld* dp) {
  ld p0 = 1.0L, p1 = x;
  if (n == 0) {
    *p = 1.0L;
    *dp = 0.0L;
    return;
  }
  for (int k = 2; k <= n; ++k) {
    const ld p2 = ((2 * k - 1) * x * p1 - (k - 1) * p0) / k;
    p0 = p1;
    p1 = p2;
  }
  *p = p1;
  *dp = n * (x * p1 - p0) / (x * x - 1.0L);
}

ld lagrange(const ld* xi, int n, int j, ld x) {
  ld v = 1.0L;
  for (int k = 0; k < n; ++k)
    if (k != j) v *= (x - xi[k]) / (xi[j] - xi[k]);
  return v;
}

void gl_nodes(int n, ld* xi, ld* w) {
  const ld pi = 3.14159265358979323846264338327950288L;
  for (int i = 0; i < n; ++i) {
    ld x = std::cos(pi * (i + 0.75L) / (n + 0.5L));
    for (int it = 0; it < 100; ++it) {
      ld p, dp;
      legendre(n, x, &p, &dp);
      const ld dx = p / dp;
      x -= dx;
      if (std::fabs(dx) < 1e-19L) break;
    }
    ld p, dp;
    legendre(n, x, &p, &dp);
    // ascending order on [0, 1]: node i from the i-th largest root reversed
    xi[n - 1 - i] = 0.5L * (x + 1.0L);
    w[n - 1 - i] = 0.5L * 2.0L / ((1.0L - x * x) * dp * dp);
  }
}

// In-place Gauss-Jordan elimination with partial pivoting on [M | I]:
// afterwards columns n..2n-1 hold M^-1.
void gauss_jordan(ld (*A)[2 * kMaxN], int n) {
  for (int c = 0; c < n; ++c) {
    int piv = c;
    for (int r = c + 1; r < n; ++r)
      if (std::fabs(A[r][c]) > std::fabs(A[piv][c])) piv = r;
    if (piv != c)
      for (int j = 0; j < 2 * n; ++j) {
        const ld t = A[c][j];
        A[c][j] = A[piv][j];
        A[piv][j] = t;
      }
    const ld inv = 1.0L / A[c][c];
    for (int j = 0; j < 2 * n; ++j) A[c][j] *= inv;
    for (int r = 0; r < n; ++r) {
      if (r == c) continue;
      const ld f = A[r][c];
      if (f == 0.0L) continue;
      for (int j = 0; j < 2 * n; ++j) A[r][j] -= f * A[c][j];
    }
  }
}

}  // namespace

void make_basis(int n, BasisTables* out) {
  ld xi[kMaxN], w[kMaxN];
  gl_nodes(n, xi, w);
  ld lam[kMaxN];
  for (int j = 0; j < n; ++j) {
    lam[j] = 1.0L;
    for (int k = 0; k < n; ++k)
      if (k != j) lam[j] /= (xi[j] - xi[k]);
  }
  ld D[kMaxN][kMaxN];
  for (int i = 0; i < n; ++i) {
    ld diag = 0.0L;
    for (int j = 0; j < n; ++j) {
      if (i == j) continue;
      D[i][j] = (lam[j] / lam[i]) / (xi[i] - xi[j]);
      diag -= D[i][j];
    }
    D[i][i] = diag;
  }
  ld phi0[kMaxN], phi1[kMaxN];
  for (int j = 0; j < n; ++j) {
    phi0[j] = lagrange(xi, n, j, 0.0L);
    phi1[j] = lagrange(xi, n, j, 1.0L);
  }
  // K1 and its inverse times diag(w)
  ld A[kMaxN][2 * kMaxN];
  for (int k = 0; k < n; ++k) {
    for (int l = 0; l < n; ++l) {
      A[k][l] = phi1[k] * phi1[l] - w[l] * D[l][k];
      A[k][n + l] = (k == l) ? 1.0L : 0.0L;
    }
  }
  gauss_jordan(A, n);
  out->n = n;
  for (int i = 0; i < kMaxN; ++i) {
    out->xi[i] = out->w[i] = out->phi0[i] = out->phi1[i] = 0.0;
    out->lift0[i] = out->lift1[i] = 0.0;
    for (int j = 0; j < kMaxN; ++j) {
      out->D[i][j] = out->Mt[i][j] = out->V[i][j] = 0.0;
      for (int s = 0; s < 3; ++s) out->P[s][i][j] = out->R[s][i][j] = 0.0;
    }
  }
  for (int i = 0; i < n; ++i) {
    out->xi[i] = double(xi[i]);
    out->w[i] = double(w[i]);
    out->phi0[i] = double(phi0[i]);
    out->phi1[i] = double(phi1[i]);
    out->lift0[i] = double(phi0[i] / w[i]);
    out->lift1[i] = double(phi1[i] / w[i]);
    for (int j = 0; j < n; ++j) {
      out->D[i][j] = double(D[i][j]);
      out->Mt[i][j] = double(A[i][n + j] * w[j]);
      out->V[i][j] = double(w[j] * D[j][i] / w[i]);
      for (int s = 0; s < 3; ++s) {
        const ld Pij = lagrange(xi, n, j, (s + xi[i]) / 3.0L);
        const ld Pji = lagrange(xi, n, i, (s + xi[j]) / 3.0L);
        out->P[s][i][j] = double(Pij);
        out->R[s][i][j] = double(Pji * w[j] / (3.0L * w[i]));
      }
    }
  }
}

void make_subcells(int n, SubcellTables* out) {
  ld xi[kMaxN], w[kMaxN];
  gl_nodes(n, xi, w);
  const int S = 2 * n - 1;
  ld A[kMaxS][kMaxN];
  for (int s = 0; s < S; ++s)
    for (int j = 0; j < n; ++j) {
      // mean of phi_j over [s/S, (s+1)/S]: n-point GL is exact for degree n-1
      ld acc = 0.0L;
      for (int q = 0; q < n; ++q) acc += w[q] * lagrange(xi, n, j, (s + xi[q]) / S);
      A[s][j] = acc;
    }
  // R = (A^T A)^-1 A^T
  ld G[kMaxN][2 * kMaxN];
  for (int i = 0; i < n; ++i)
    for (int j = 0; j < n; ++j) {
      ld acc = 0.0L;
      for (int s = 0; s < S; ++s) acc += A[s][i] * A[s][j];
      G[i][j] = acc;
      G[i][n + j] = (i == j) ? 1.0L : 0.0L;
    }
  gauss_jordan(G, n);
  *out = SubcellTables{};
  out->n = n;
  out->S = S;
  for (int s = 0; s < S; ++s)
    for (int j = 0; j < n; ++j) out->A[s][j] = double(A[s][j]);
  for (int i = 0; i < n; ++i)
    for (int s = 0; s < S; ++s) {
      ld acc = 0.0L;
      for (int k = 0; k < n; ++k) acc += G[i][n + k] * A[s][k];
      out->R[i][s] = double(acc);
      out->Pi[i][s] = double(A[s][i] / (S * w[i]));
    }
}

}  // namespace ader
