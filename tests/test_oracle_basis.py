"""Pins of the oracle's reference-element operators (closed forms, exactness, identities)."""
import math

import numpy as np
import pytest

from oracle import basis


@pytest.mark.parametrize("N,nodes,weights", [
    (1, [-1.0, 1.0], [1.0, 1.0]),
    (2, [-1.0, 0.0, 1.0], [1 / 3, 4 / 3, 1 / 3]),
    (3, [-1.0, -1 / math.sqrt(5), 1 / math.sqrt(5), 1.0], [1 / 6, 5 / 6, 5 / 6, 1 / 6]),
    (4, [-1.0, -math.sqrt(3 / 7), 0.0, math.sqrt(3 / 7), 1.0],
     [1 / 10, 49 / 90, 32 / 45, 49 / 90, 1 / 10]),
])
def test_lgl_closed_forms(N, nodes, weights):
    x, w = basis.lgl_nodes_weights(N)
    np.testing.assert_allclose(x, nodes, atol=1e-15)
    np.testing.assert_allclose(w, weights, rtol=1e-14)


@pytest.mark.parametrize("N", range(1, 9))
def test_lgl_quadrature_exactness(N):
    # LGL with N+1 points integrates polynomials of degree 2N-1 exactly, and not 2N
    x, w = basis.lgl_nodes_weights(N)
    assert abs(w.sum() - 2.0) < 1e-14
    for k in range(2 * N):
        exact = 0.0 if k % 2 else 2.0 / (k + 1)
        assert abs(np.dot(w, x ** k) - exact) < 1e-13
    k = 2 * N
    assert abs(np.dot(w, x ** k) - 2.0 / (k + 1)) > 1e-6


@pytest.mark.parametrize("N", range(1, 9))
def test_derivative_exact_on_polynomials(N):
    x, _ = basis.lgl_nodes_weights(N)
    D = basis.derivative_matrix(x)
    np.testing.assert_allclose(D @ np.ones(N + 1), 0.0, atol=1e-13)
    for k in range(1, N + 1):
        np.testing.assert_allclose(D @ x ** k, k * x ** (k - 1), atol=5e-13)


@pytest.mark.parametrize("N", range(1, 9))
def test_derivative_sbp(N):
    # summation by parts: W D + (W D)^T = diag(-1, 0, ..., 0, 1)
    x, w = basis.lgl_nodes_weights(N)
    Q = np.diag(w) @ basis.derivative_matrix(x)
    B = np.zeros((N + 1, N + 1))
    B[0, 0], B[-1, -1] = -1.0, 1.0
    np.testing.assert_allclose(Q + Q.T, B, atol=1e-13)


@pytest.mark.parametrize("N", range(1, 9))
def test_prolongation_is_exact_interpolation(N):
    b = basis.Basis(N)
    rng = np.random.default_rng(N)
    coef = rng.standard_normal(N + 1)
    p = np.polynomial.polynomial.polyval(b.nodes, coef)
    for c in (0, 1):
        child_x = (b.nodes + (2 * c - 1)) / 2.0
        np.testing.assert_allclose(b.P[c] @ p, np.polynomial.polynomial.polyval(child_x, coef),
                                   atol=1e-13)
        np.testing.assert_allclose(b.P[c], basis.interp_child(b.nodes, c), atol=1e-13)


@pytest.mark.parametrize("N", range(1, 9))
def test_restrict_after_prolong_is_identity(N):
    b = basis.Basis(N)
    np.testing.assert_allclose(b.C[0] @ b.P[0] + b.C[1] @ b.P[1], np.eye(N + 1), atol=2e-14)


@pytest.mark.parametrize("N", range(1, 9))
def test_restriction_conserves_lgl_mass(N):
    # sum_i w_i (C_0 f0 + C_1 f1)_i = (1/2) (sum w f0 + sum w f1): the s = 1/2 of Sec. 3.3
    b = basis.Basis(N)
    rng = np.random.default_rng(100 + N)
    f0, f1 = rng.standard_normal((2, N + 1))
    lhs = np.dot(b.weights, b.C[0] @ f0 + b.C[1] @ f1)
    rhs = 0.5 * (np.dot(b.weights, f0) + np.dot(b.weights, f1))
    assert abs(lhs - rhs) < 1e-13


@pytest.mark.parametrize("N", range(1, 9))
def test_prolongation_conserves_lgl_mass(N):
    b = basis.Basis(N)
    rng = np.random.default_rng(200 + N)
    f = rng.standard_normal(N + 1)
    lhs = 0.5 * (np.dot(b.weights, b.P[0] @ f) + np.dot(b.weights, b.P[1] @ f))
    assert abs(lhs - np.dot(b.weights, f)) < 1e-13


def test_lumped_restriction_is_not_identity():
    # the alternative reading (LGL-lumped mass) would not give an identity: keep the exact one
    b = basis.Basis(4)
    W = np.diag(b.weights)
    lumped = [0.5 * np.linalg.solve(W, b.P[c].T @ W) for c in (0, 1)]
    err = np.abs(lumped[0] @ b.P[0] + lumped[1] @ b.P[1] - np.eye(5)).max()
    assert err > 0.1


def test_legendre_closed_forms():
    """P_2..P_4 and their derivatives written out; P_n(1) = 1 and P_n'(1) = n (n+1) / 2."""
    x = np.linspace(-1.0, 1.0, 13)
    closed = {2: ((3 * x**2 - 1) / 2, 3 * x),
              3: ((5 * x**3 - 3 * x) / 2, (15 * x**2 - 3) / 2),
              4: ((35 * x**4 - 30 * x**2 + 3) / 8, (140 * x**3 - 60 * x) / 8)}
    for n, (p, dp) in closed.items():
        got_p, got_dp = basis.legendre_and_derivative(n, x)
        np.testing.assert_allclose(got_p, p, atol=1e-15)
        np.testing.assert_allclose(got_dp, dp, atol=1e-14)
    for n in range(0, 10):
        p1, dp1 = basis.legendre_and_derivative(n, np.array([1.0]))
        assert abs(p1[0] - 1.0) < 1e-15 and abs(dp1[0] - n * (n + 1) / 2) < 1e-12


def test_barycentric_weights_closed_form():
    """On {-1, 0, 1}: 1 / ((x_j - x_k)(x_j - x_l)) = 1/2, -1, 1/2."""
    np.testing.assert_allclose(basis.barycentric_weights(np.array([-1.0, 0.0, 1.0])), [0.5, -1.0, 0.5])


@pytest.mark.parametrize("N", range(1, 9))
def test_lagrange_matrix_cardinal_and_exact(N):
    """l_j(x_i) = delta_ij, and sum_j p(x_j) l_j(x) = p(x) for every polynomial of degree <= N."""
    x, _ = basis.lgl_nodes_weights(N)
    np.testing.assert_allclose(basis.lagrange_matrix(x, x), np.eye(N + 1), atol=1e-14)
    y = np.linspace(-1.0, 1.0, 17)
    L = basis.lagrange_matrix(x, y)
    for k in range(N + 1):
        np.testing.assert_allclose(L @ x**k, y**k, atol=1e-13)
    # degree N + 1 is not reproduced
    assert np.abs(L @ x**(N + 1) - y**(N + 1)).max() > 1e-6


@pytest.mark.parametrize("n", range(1, 10))
def test_gauss_legendre_exactness(n):
    """n points integrate x^k exactly for k <= 2n - 1."""
    g, gw = basis.gauss_legendre(n)
    for k in range(2 * n):
        exact = 0.0 if k % 2 else 2.0 / (k + 1)
        assert abs(np.dot(gw, g**k) - exact) < 1e-13


@pytest.mark.parametrize("N", range(1, 9))
def test_mass_matrices_row_and_column_sums(N):
    """M 1 = w (the LGL rule is exact on the degree-N l_i), 1^T M 1 = 2, M symmetric positive
    definite; the mixed matrices S_c 1 = w (the parent basis sums to 1) and
    sum_c 1^T S_c = 2 w^T (the two children cover the parent, each at half scale); the entries of
    M against a 30-point Gauss rule."""
    x, w = basis.lgl_nodes_weights(N)
    M = basis.exact_mass_matrix(x)
    np.testing.assert_allclose(M @ np.ones(N + 1), w, atol=1e-14)
    assert abs(M.sum() - 2.0) < 1e-13
    np.testing.assert_allclose(M, M.T, atol=1e-15)
    assert np.linalg.eigvalsh(M).min() > 0.0
    g, gw = np.polynomial.legendre.leggauss(30)
    L = basis.lagrange_matrix(x, g)
    np.testing.assert_allclose(M, L.T @ (gw[:, None] * L), atol=1e-14)
    S = [basis.mixed_mass_child(x, c) for c in (0, 1)]
    for Sc in S:
        np.testing.assert_allclose(Sc @ np.ones(N + 1), w, atol=1e-14)
    np.testing.assert_allclose(np.ones(N + 1) @ (S[0] + S[1]), 2 * w, atol=1e-13)
