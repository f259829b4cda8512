"""Pins of the oracle's small helpers that GPU tests use as references: the theta' refinement
indicator (Sec. 4.3) and its inverse map from a theta' field to the hydrostatic-pressure state,
the tracer indicator, the initial adaptation driver, and the error norm of the isentropic vortex
(Sec. 4.1).  Each is checked against what its definition fixes: a round trip through the
closed-form inverse, absolute values of negative fields, the closed form of the norm on a
constant error, and the invariants the adaptation loop must leave behind."""
import math

import numpy as np

from oracle import dg, forest as fo, tracer, vortex


def _mesh(d=2, N=3, base=(3, 2), lengths=(1500.0, 1000.0), max_level=0):
    return dg.Mesh(fo.Forest(base, max_level), N, lengths)


def test_theta_indicator_inverts_the_initial_state_map():
    """theta' of state_from_theta(theta) is theta itself: rho_bar + rho' = rho_bar theta0 /
    (theta0 + theta), so (Theta_bar + 0) / (rho_bar + rho') - theta0 = theta (Theta_bar =
    rho_bar theta0).  The indicator is the largest |theta| of each element, negative values
    included."""
    m = _mesh()
    rng = np.random.default_rng(7)
    th = rng.uniform(-3.0, 3.0, size=(m.E, m.np_))
    th[0, 5] = -9.5                      # the largest magnitude of element 0 is negative
    q = dg.state_from_theta(m, th)
    np.testing.assert_allclose(dg.theta_prime(m, q), th, rtol=0, atol=1e-11)
    ind = dg.indicator(m, q)
    np.testing.assert_allclose(ind, np.max(np.abs(th), axis=1), rtol=1e-12)
    assert abs(ind[0] - 9.5) <= 1e-11
    # a planted sign error in the inverse map breaks the round trip
    bad = q.copy()
    bad[0] = -bad[0]
    assert np.abs(dg.theta_prime(m, bad) - th).max() > 1e-3


def test_tracer_indicator_is_max_abs_per_element():
    C = np.array([[0.1, -0.7, 0.3], [0.0, 0.0, 0.0], [2.0, -2.5, 1.0]])
    np.testing.assert_array_equal(tracer.indicator(None, C), [0.7, 0.0, 2.5])


def test_vortex_norm_closed_form():
    """(1 / n) sqrt(sum e^2): a constant error c over n values gives |c| / sqrt(n)."""
    n_var, E, NP = 4, 6, 16
    q_exact = np.random.default_rng(3).standard_normal((n_var, E, NP))
    c = -0.0375
    n = n_var * E * NP
    assert abs(vortex.l2_paper(q_exact + c, q_exact) - abs(c) / math.sqrt(n)) <= 1e-16
    assert vortex.l2_paper(q_exact, q_exact) == 0.0


def test_adapt_initial_invariants():
    """The initial adaptation re-evaluates the analytic bubble on each new mesh, max_level
    times: with nothing above the threshold the mesh stays at the roots; with everything above
    it every leaf ends at max_level; for a bubble, every final element whose indicator exceeds
    the threshold is at max_level (it was tagged in every round), and coarse leaves lie where
    theta' is small."""
    N, base, lengths, L = 3, (4, 2), (4000.0, 2000.0), 2
    flat = dg.adapt_initial(fo.Forest(base, L), N, lengths, lambda m: np.zeros((m.E, m.np_)), 0.1, 1)
    assert flat.E == 8 and all(lev == 0 for lev, _ in flat.forest.leaves)
    hot = dg.adapt_initial(fo.Forest(base, L), N, lengths, lambda m: np.full((m.E, m.np_), 1.0), 0.1, 0)
    assert hot.E == 8 * 4 ** L and all(lev == L for lev, _ in hot.forest.leaves)

    def bell(m):
        return dg.bubble_theta(m, (1000.0, 900.0), (600.0, 600.0), 1.0)

    m = dg.adapt_initial(fo.Forest(base, L), N, lengths, bell, 0.05, 1)
    ind = dg.indicator(m, dg.state_from_theta(m, bell(m)))
    levels = np.array([lev for lev, _ in m.forest.leaves])
    assert np.all(levels[ind > 0.05] == L)
    assert levels.min() == 0 and levels.max() == L
    assert np.all(ind[levels == 0] <= 0.05)
