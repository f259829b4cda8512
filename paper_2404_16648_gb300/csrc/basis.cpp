// Host construction of the LGL operators (FP64).
//
// LGL nodes: +-1 and the interior roots of q(x) = P_{N+1}(x) - P_{N-1}(x), whose derivative is
// q'(x) = (2N+1) P_N(x); Newton from the Chebyshev-Gauss-Lobatto points.  Weights
// 2 / (N (N+1) P_N(x_j)^2).  Derivative matrix from the LGL closed form
// D_ij = P_N(x_i) / (P_N(x_j) (x_i - x_j)), diagonal as minus the off-diagonal row sum.
// Half-interval interpolation P_c by the barycentric formula; the mortar->face / child->parent
// projection (1/2) M^{-1} S_c^T (Sec. 3.3) with exact (Gauss-Legendre, N+2 point) mass matrices.
#include "basis.hpp"

#include <cmath>
#include <stdexcept>

namespace dgl {
namespace {

// P_n(x) and P_n'(x) by the Bonnet recurrence.
void legendre(int n, double x, double* p, double* dp) {
  double p0 = 1.0, p1 = x, d0 = 0.0, d1 = 1.0;
  if (n == 0) { *p = 1.0; *dp = 0.0; return; }
  for (int k = 2; k <= n; ++k) {
    double p2 = ((2.0 * k - 1.0) * x * p1 - (k - 1.0) * p0) / k;
    double d2 = d0 + (2.0 * k - 1.0) * p1;
    p0 = p1; p1 = p2; d0 = d1; d1 = d2;
  }
  *p = p1; *dp = d1;
}

double legendre_p(int n, double x) { double p, dp; legendre(n, x, &p, &dp); return p; }

void gauss_legendre(int n, std::vector<double>& g, std::vector<double>& gw) {
  g.assign(n, 0.0); gw.assign(n, 0.0);
  for (int j = 0; j < n; ++j) {
    double x = -std::cos(M_PI * (j + 0.75) / (n + 0.5));
    for (int it = 0; it < 100; ++it) {
      double p, dp; legendre(n, x, &p, &dp);
      double dx = p / dp; x -= dx;
      if (std::fabs(dx) < 1e-16) break;
    }
    double p, dp; legendre(n, x, &p, &dp);
    g[j] = x; gw[j] = 2.0 / ((1.0 - x * x) * dp * dp);
  }
}

// Lagrange basis on nodes xs evaluated at t, barycentric second form (exact at nodes).
void lagrange_at(const std::vector<double>& xs, const std::vector<double>& lam, double t,
                 double* out) {
  const int n = (int)xs.size();
  for (int j = 0; j < n; ++j) {
    if (t == xs[j]) { for (int k = 0; k < n; ++k) out[k] = (k == j) ? 1.0 : 0.0; return; }
  }
  double den = 0.0;
  for (int j = 0; j < n; ++j) { out[j] = lam[j] / (t - xs[j]); den += out[j]; }
  for (int j = 0; j < n; ++j) out[j] /= den;
}

// Solves A X = B in place (A n x n, B n x m, row-major) with partial pivoting.
void solve(std::vector<double> A, std::vector<double>& B, int n, int m) {
  for (int c = 0; c < n; ++c) {
    int piv = c;
    for (int r = c + 1; r < n; ++r) if (std::fabs(A[r * n + c]) > std::fabs(A[piv * n + c])) piv = r;
    if (piv != c) {
      for (int k = 0; k < n; ++k) std::swap(A[c * n + k], A[piv * n + k]);
      for (int k = 0; k < m; ++k) std::swap(B[c * m + k], B[piv * m + k]);
    }
    for (int r = 0; r < n; ++r) {
      if (r == c) continue;
      double f = A[r * n + c] / A[c * n + c];
      if (f == 0.0) continue;
      for (int k = c; k < n; ++k) A[r * n + k] -= f * A[c * n + k];
      for (int k = 0; k < m; ++k) B[r * m + k] -= f * B[c * m + k];
    }
  }
  for (int r = 0; r < n; ++r) for (int k = 0; k < m; ++k) B[r * m + k] /= A[r * n + r];
}

}  // namespace

Basis1D make_basis(int N) {
  if (N < 1 || N > 8) throw std::invalid_argument("degree out of range");
  Basis1D b; b.N = N; const int n1 = N + 1;
  b.x.assign(n1, 0.0); b.w.assign(n1, 0.0);
  b.x[0] = -1.0; b.x[N] = 1.0;
  for (int j = 1; j < N; ++j) {
    double x = -std::cos(M_PI * j / N);
    for (int it = 0; it < 100; ++it) {
      double qa, dqa, qb, dqb;
      legendre(N + 1, x, &qa, &dqa); legendre(N - 1, x, &qb, &dqb);
      double q = qa - qb, dq = (2.0 * N + 1.0) * legendre_p(N, x);
      double dx = q / dq; x -= dx;
      if (std::fabs(dx) < 1e-16) break;
    }
    b.x[j] = x;
  }
  for (int j = 0; j < n1; ++j) {
    double p = legendre_p(N, b.x[j]);
    b.w[j] = 2.0 / (N * (N + 1.0) * p * p);
  }
  b.D.assign(n1 * n1, 0.0);
  for (int i = 0; i < n1; ++i) {
    double s = 0.0;
    for (int j = 0; j < n1; ++j) {
      if (i == j) continue;
      double v = legendre_p(N, b.x[i]) / (legendre_p(N, b.x[j]) * (b.x[i] - b.x[j]));
      b.D[i * n1 + j] = v; s += v;
    }
    b.D[i * n1 + i] = -s;
  }
  std::vector<double> lam(n1, 1.0);
  for (int j = 0; j < n1; ++j)
    for (int k = 0; k < n1; ++k) if (k != j) lam[j] /= (b.x[j] - b.x[k]);
  std::vector<double> g, gw; gauss_legendre(N + 2, g, gw);
  const int ng = N + 2;
  std::vector<double> Lg(ng * n1);
  for (int q = 0; q < ng; ++q) lagrange_at(b.x, lam, g[q], &Lg[q * n1]);
  std::vector<double> M(n1 * n1, 0.0);
  for (int i = 0; i < n1; ++i)
    for (int j = 0; j < n1; ++j) {
      double s = 0.0;
      for (int q = 0; q < ng; ++q) s += gw[q] * Lg[q * n1 + i] * Lg[q * n1 + j];
      M[i * n1 + j] = s;
    }
  std::vector<double> tmp(n1);
  for (int c = 0; c < 2; ++c) {
    b.G[c].assign(n1 * n1, 0.0);
    for (int i = 0; i < n1; ++i) {
      const bool mid = std::fabs(b.x[i]) < 1e-14;
      const bool inside = c == 0 ? b.x[i] < 0.0 : b.x[i] > 0.0;
      const double wt = mid ? 0.5 : (inside ? 1.0 : 0.0);
      if (wt == 0.0) continue;
      lagrange_at(b.x, lam, 2.0 * b.x[i] - (2.0 * c - 1.0), tmp.data());
      for (int j = 0; j < n1; ++j) b.G[c][i * n1 + j] = wt * tmp[j];
    }
  }
  for (int c = 0; c < 2; ++c) {
    const double off = 2.0 * c - 1.0;
    b.P[c].assign(n1 * n1, 0.0);
    for (int i = 0; i < n1; ++i) {
      lagrange_at(b.x, lam, (b.x[i] + off) * 0.5, tmp.data());
      for (int j = 0; j < n1; ++j) b.P[c][i * n1 + j] = tmp[j];
    }
    // S_c^T[j][i] = int l_i(x) l_j(xi_c(x)) dx, i child basis, j parent basis
    std::vector<double> St(n1 * n1, 0.0), Lp(ng * n1);
    for (int q = 0; q < ng; ++q) lagrange_at(b.x, lam, (g[q] + off) * 0.5, &Lp[q * n1]);
    for (int j = 0; j < n1; ++j)
      for (int i = 0; i < n1; ++i) {
        double s = 0.0;
        for (int q = 0; q < ng; ++q) s += gw[q] * Lg[q * n1 + i] * Lp[q * n1 + j];
        St[j * n1 + i] = 0.5 * s;
      }
    solve(M, St, n1, n1);
    b.C[c] = St;
  }
  return b;
}

}  // namespace dgl
