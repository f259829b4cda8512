"""Reference-element operators of the nodal dGSEM (oracle; test infrastructure only).

Restates, in plain FP64 numpy, the one-dimensional objects that arXiv 2404.16648 builds a
single time on the reference element and applies axis by axis as tensor products (Sec. 3.3):

* Legendre-Gauss-Lobatto (LGL) nodes and weights of degree N (the collocation points named
  in Sec. 3.3; the diagonal LGL mass matrix of Sec. 2.2);
* the collocation derivative D_ij = l_j'(x_i) used by the strong form (Sec. 2.2);
* the L2 projection matrices between a parent interval and its two halves: the
  face->mortar projection P = M^{-1} S (Sec. 3.3, first mortar projection), which on degree-N
  data is exact interpolation, and the mortar->face projection s M^{-1} S^T with s = 1/2
  (Sec. 3.3, second mortar projection).  The same matrices serve refinement (parent -> child)
  and coarsening (children -> parent), as Sec. 3.3 states.

Reading (ambiguity): Sec. 3.3 describes coarsening as an integration over the LGL points
while the mortar formulas use mass matrices M.  The oracle takes M as the *exact* mass matrix
(Gauss-Legendre with N+2 points), which makes coarsen(refine(q)) = q exactly and conserves the
LGL-discrete mass.

Pinned by tests/test_oracle_basis.py (closed-form nodes/weights for N = 2, 3, 4, exactness of D
on x^k, the SBP identity, sum_c C_c I_c = I, exactness of I_c on polynomials).
"""
import numpy as np

__all__ = [
    "legendre_and_derivative", "lgl_nodes_weights", "barycentric_weights", "derivative_matrix",
    "lagrange_matrix", "gauss_legendre", "exact_mass_matrix", "child_map", "interp_child",
    "mixed_mass_child", "prolong_matrix", "restrict_matrix", "Basis",
]


def legendre_and_derivative(n, x):
    """P_n(x) and P_n'(x) by the three-term recurrence (textbook definition)."""
    x = np.asarray(x, dtype=np.float64)
    p_prev = np.ones_like(x)
    dp_prev = np.zeros_like(x)
    if n == 0:
        return p_prev, dp_prev
    p = x.copy()
    dp = np.ones_like(x)
    for k in range(1, n):
        # (k+1) P_{k+1} = (2k+1) x P_k - k P_{k-1};  P'_{k+1} = P'_{k-1} + (2k+1) P_k
        p_next = ((2 * k + 1) * x * p - k * p_prev) / (k + 1)
        dp_next = dp_prev + (2 * k + 1) * p
        p_prev, p = p, p_next
        dp_prev, dp = dp, dp_next
    return p, dp


def lgl_nodes_weights(N):
    """LGL nodes (ascending) and weights for polynomial degree N >= 1.

    Nodes are -1, +1 and the N-1 roots of P_N'; weights w_j = 2 / (N (N+1) P_N(x_j)^2).
    Interior roots by Newton's method on P_N' (with P_N'' from Legendre's equation), started
    from the Chebyshev-Gauss-Lobatto points.
    """
    if N < 1:
        raise ValueError("N must be >= 1")
    x = -np.cos(np.pi * np.arange(N + 1) / N)
    interior = x[1:-1].copy()
    for _ in range(100):
        p, dp = legendre_and_derivative(N, interior)
        # Legendre's equation: (1-x^2) P'' = 2 x P' - N (N+1) P
        ddp = (2.0 * interior * dp - N * (N + 1) * p) / (1.0 - interior ** 2)
        step = dp / ddp
        interior = interior - step
        if np.all(np.abs(step) < 1e-16):
            break
    nodes = np.concatenate([[-1.0], np.sort(interior), [1.0]])
    pN, _ = legendre_and_derivative(N, nodes)
    weights = 2.0 / (N * (N + 1) * pN ** 2)
    return nodes, weights


def barycentric_weights(nodes):
    """lambda_j = 1 / prod_{k != j} (x_j - x_k)."""
    n = len(nodes)
    lam = np.ones(n)
    for j in range(n):
        for k in range(n):
            if k != j:
                lam[j] /= (nodes[j] - nodes[k])
    return lam


def derivative_matrix(nodes):
    """Collocation derivative D_ij = l_j'(x_i) of the Lagrange basis on ``nodes``.

    Off-diagonal (lambda_j / lambda_i) / (x_i - x_j); diagonal -sum of the row (l_j sum to 1).
    """
    n = len(nodes)
    lam = barycentric_weights(nodes)
    D = np.zeros((n, n))
    for i in range(n):
        for j in range(n):
            if i != j:
                D[i, j] = (lam[j] / lam[i]) / (nodes[i] - nodes[j])
        D[i, i] = -np.sum(D[i, :])
    return D


def lagrange_matrix(nodes, x):
    """L[p, j] = l_j(x_p), Lagrange basis on ``nodes`` by the product definition."""
    x = np.atleast_1d(np.asarray(x, dtype=np.float64))
    n = len(nodes)
    L = np.ones((len(x), n))
    for j in range(n):
        for k in range(n):
            if k != j:
                L[:, j] *= (x - nodes[k]) / (nodes[j] - nodes[k])
    return L


def gauss_legendre(n):
    """n-point Gauss-Legendre rule on [-1, 1] (library routine)."""
    return np.polynomial.legendre.leggauss(n)


def exact_mass_matrix(nodes):
    """M_ij = int_{-1}^{1} l_i l_j dx, integrated exactly (Gauss-Legendre, N+2 points)."""
    N = len(nodes) - 1
    g, gw = gauss_legendre(N + 2)
    L = lagrange_matrix(nodes, g)
    return L.T @ (gw[:, None] * L)


def child_map(c, x):
    """Parent coordinate of child/mortar coordinate x in [-1,1]; c = 0 lower half, 1 upper."""
    return (np.asarray(x) + (2 * c - 1)) / 2.0


def interp_child(nodes, c):
    """I_c[i, j] = l_j(xi_c(x_i)): parent basis evaluated at the child's nodes."""
    return lagrange_matrix(nodes, child_map(c, nodes))


def mixed_mass_child(nodes, c):
    """S_c[i, j] = int_{-1}^{1} l_i(x) l_j(xi_c(x)) dx (child/mortar basis i, parent basis j).

    This is the mixed mass matrix S^{Omega_L -> Xi_c} of Sec. 3.3, integrated exactly.
    """
    N = len(nodes) - 1
    g, gw = gauss_legendre(N + 2)
    Lm = lagrange_matrix(nodes, g)                 # mortar basis at GL points
    Lp = lagrange_matrix(nodes, child_map(c, g))   # parent basis at the same points
    return Lm.T @ (gw[:, None] * Lp)


def prolong_matrix(nodes, c):
    """Face -> mortar (or parent -> child) projection P_c = M^{-1} S_c (Sec. 3.3)."""
    M = exact_mass_matrix(nodes)
    return np.linalg.solve(M, mixed_mass_child(nodes, c))


def restrict_matrix(nodes, c, s=0.5):
    """Mortar -> face (or child -> parent) projection s M^{-1} S_c^T with s = 1/2 (Sec. 3.3)."""
    M = exact_mass_matrix(nodes)
    return s * np.linalg.solve(M, mixed_mass_child(nodes, c).T)


class Basis:
    """All 1D reference operators for degree N."""

    def __init__(self, N):
        self.N = N
        self.nodes, self.weights = lgl_nodes_weights(N)
        self.D = derivative_matrix(self.nodes)
        self.M = exact_mass_matrix(self.nodes)
        self.P = [prolong_matrix(self.nodes, c) for c in (0, 1)]
        self.C = [restrict_matrix(self.nodes, c) for c in (0, 1)]
