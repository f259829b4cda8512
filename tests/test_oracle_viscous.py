"""Pins of the oracle's BR1 viscous operator: exact zeros, conservation with flux-free walls,
convergence towards an independently differentiated exact operator."""
import math

import numpy as np
import pytest

from oracle import dg, forest as fo, physics

K = physics.Constants()
NU = 75.0


def _hanging(base, N, L, seed):
    f = fo.Forest(base, 1)
    rng = np.random.default_rng(seed)
    f, _ = f.regrid(rng.random(len(f)) < 0.3, 0)
    assert f.face_lists()[1]
    return dg.Mesh(f, N, L, K)


def test_rest_and_constant_primitives_give_zero():
    m = _hanging((3, 3), 3, (900.0, 900.0), 0)
    assert np.all(dg.viscous_rhs(m, np.zeros((4, m.E, m.np_)), NU) == 0.0)
    rb, _, _ = m.bg
    q = np.zeros((4, m.E, m.np_))
    q[1] = rb * 1.5          # u = 1.5, w = -0.5, theta' = 0.2 everywhere (rho' = 0)
    q[2] = rb * -0.5
    q[3] = rb * 0.2
    V = dg.viscous_rhs(m, q, NU)
    assert np.abs(V).max() <= 1e-10 * NU * np.abs(rb).max() / m.h.min() ** 2


@pytest.mark.parametrize("base,N,L", [((3, 3), 3, (900.0, 900.0)), ((2, 2, 2), 2, (800.0, 800.0, 800.0))])
def test_conservation_with_flux_free_walls(base, N, L):
    m = _hanging(base, N, L, 1)
    rng = np.random.default_rng(2)
    q = np.empty((m.nv, m.E, m.np_))
    q[0] = 1e-3 * rng.standard_normal(q[0].shape)
    q[1:1 + m.d] = rng.standard_normal(q[1:1 + m.d].shape)
    q[1 + m.d] = 0.2 * rng.standard_normal(q[0].shape)
    V = dg.viscous_rhs(m, q, NU)
    assert np.all(V[0] == 0.0)          # no viscous mass flux
    W = m.wnode[None, :] * m.J[:, None]
    for v in range(1, m.nv):
        assert abs(math.fsum((W * V[v]).ravel())) <= 1e-13 * math.fsum(np.abs(W * V[v]).ravel())


@pytest.mark.parametrize("N,order", [(2, 1), (3, 3), (4, 3)])
def test_convergence_against_exact_operator(N, order):
    # u = cos(kx) cos(kz) has zero normal derivative on the walls of [0, L]^2; rho' = 0 so
    # rho = rho_bar(z); exact nu [rho_bar (u_xx + u_zz) + rho_bar' u_z] with rho_bar' by complex step
    L = 1000.0
    k = np.pi / L
    errs = []
    for nb in (4, 8, 16):
        f = fo.Forest((nb, nb), 1)
        tag = np.zeros(nb * nb, dtype=bool)
        tag[nb * nb // 2 + nb // 2] = True
        f, _ = f.regrid(tag, 0)
        m = dg.Mesh(f, N, (L, L), K)
        x, z = m.x
        rb, _, _ = m.bg
        u = np.cos(k * x) * np.cos(k * z)
        q = np.stack([0 * x, rb * u, 0 * x, 0 * x])
        V = dg.viscous_rhs(m, q, NU)
        hstep = 1e-30
        drb = physics.background(z + 1j * hstep, K)[0].imag / hstep
        exact = NU * (rb * (-2 * k * k * u) + drb * (-k * np.cos(k * x) * np.sin(k * z)))
        errs.append(np.abs(V[1] - exact).max() / np.abs(exact).max())
    rate = math.log2(errs[-2] / errs[-1])
    assert rate >= order - 0.3, (errs, rate)


def test_viscous_primitives_against_their_definition():
    """phi = (U / rho, theta') with rho = rho_bar + rho' and theta' defined as
    (Theta_bar + Theta') / (rho_bar + rho') - theta0; the oracle's form (Theta' - theta0 rho') / rho
    is its rewriting for Theta_bar = rho_bar theta0, so both agree to rounding."""
    m = _hanging((3, 3), 3, (900.0, 900.0), 1)
    rb, Tb, _ = m.bg
    g = np.random.default_rng(5)
    q = np.empty((4, m.E, m.np_))
    q[0] = 1e-3 * g.standard_normal((m.E, m.np_))
    q[1:3] = 2.0 * g.standard_normal((2, m.E, m.np_))
    q[3] = 0.5 * g.standard_normal((m.E, m.np_))
    phi, rho = dg.viscous_primitives(m, q)
    np.testing.assert_allclose(rho, rb + q[0], rtol=1e-15)
    np.testing.assert_allclose(phi[:2], q[1:3] / (rb + q[0]), rtol=1e-14)
    theta = (Tb + q[3]) / (rb + q[0]) - K.theta0
    np.testing.assert_allclose(phi[2], theta, rtol=0, atol=1e-11)
