"""Pins of the oracle's tracer advection (linear-advection test of Sec. 4.2): the wind and the
bell, the upwind flux, conservation with mortars and its loss with point interpolation, the two
modes agreeing on conforming meshes, convergence against the exact tendency, and the return of
the bell after the time-reversing period."""
import math

import numpy as np
import pytest

import workloads
from oracle import dg as odg, forest as ofo, tracer as otr

T = 5.0


def _mesh(base, N, L=0, flags_p=0.0, seed=0):
    f = ofo.Forest(base, L)
    if L and flags_p:
        flags = workloads.random_flags(len(f), flags_p, seed)
        flags[0] = 1
        f, _ = f.regrid(flags.astype(bool), 0)
    return odg.Mesh(f, N, (1.0, 1.0))


def test_wind_is_divergence_free_and_vanishes_on_the_walls():
    rng = np.random.default_rng(1)
    x, y = rng.random(50), rng.random(50)
    h = 1e-20
    # complex step: d/dx u + d/dy v
    du = otr.leveque_wind(x + 1j * h, y, 0.7, T)[0].imag / h
    dv = otr.leveque_wind(x, y + 1j * h, 0.7, T)[1].imag / h
    assert np.abs(du + dv).max() <= 1e-13
    s = np.linspace(0.0, 1.0, 11)
    assert np.all(otr.leveque_wind(np.zeros(11), s, 0.3, T)[0] == 0.0)
    assert np.all(otr.leveque_wind(s, np.zeros(11), 0.3, T)[1] == 0.0)
    # reversal: g(T - t) = -g(t)
    u1 = otr.leveque_wind(x, y, 1.1, T)[0]
    u2 = otr.leveque_wind(x, y, T - 1.1, T)[0]
    np.testing.assert_allclose(u1, -u2, atol=1e-15)


def test_upwind_flux_takes_the_upwind_value():
    cm, cp = np.array([2.0, 2.0, 5.0]), np.array([3.0, 3.0, 5.0])
    un = np.array([0.5, -0.25, 0.0])
    np.testing.assert_allclose(otr.upwind(cm, cp, un), [1.0, -0.75, 0.0], rtol=0, atol=1e-15)


def test_bell_profile():
    m = _mesh((4, 4), 4)
    C = otr.bell(m, (0.25, 0.25), 0.25, 0.5)
    r = np.hypot(m.x[0] - 0.25, m.x[1] - 0.25) / 0.25
    inside = r <= 1.0
    np.testing.assert_allclose(C[inside], 0.5 * (1 + np.cos(np.pi * r[inside])), rtol=0, atol=1e-15)
    assert np.all(C[~inside] == 0.0)
    assert C.max() <= 1.0


@pytest.mark.parametrize("N", [2, 3, 4])
def test_modes_agree_on_conforming_meshes(N):
    m = _mesh((3, 4), N)
    C = workloads.random_scalar(m.E, m.np_, seed=5 + N)
    np.testing.assert_array_equal(otr.rhs(m, C, 0.4, T, "mortar"), otr.rhs(m, C, 0.4, T, "interp"))


@pytest.mark.parametrize("N", [2, 3, 4])
def test_mortar_conserves_and_interpolation_does_not(N):
    m = _mesh((3, 3), N, L=1, flags_p=0.4, seed=10 + N)
    assert len(m.forest.face_lists()[1]) > 0
    C = workloads.random_scalar(m.E, m.np_, seed=20 + N)
    W = m.wnode[None, :] * m.J[:, None]
    for t in (0.3, 1.9):
        r_m = otr.rhs(m, C, t, T, "mortar")
        r_i = otr.rhs(m, C, t, T, "interp")
        scale = np.abs(W * r_m).sum()
        assert abs(math.fsum((W * r_m).ravel())) <= 1e-14 * scale
        assert abs(math.fsum((W * r_i).ravel())) >= 1e-6 * scale
        # the fine sides of hanging faces and every other element see identical fluxes
        coarse = {g[0] for g in m.forest.face_lists()[1]}
        rest = [e for e in range(m.E) if e not in coarse]
        np.testing.assert_array_equal(r_m[rest], r_i[rest])


def _exact_tendency(mesh, t, fx, fy_unused=None):
    """-div(C u) of the smooth field C = fx(x, y) by complex step."""
    h = 1e-20
    x, y = mesh.x[0], mesh.x[1]

    def Cu(xx, yy):
        u, v = otr.leveque_wind(xx, yy, t, T)
        return fx(xx, yy) * u, fx(xx, yy) * v
    dx = Cu(x + 1j * h, y)[0].imag / h
    dy = Cu(x, y + 1j * h)[1].imag / h
    return -(dx + dy)


@pytest.mark.parametrize("N,refined", [(2, False), (3, False), (3, True), (4, True)])
def test_convergence_against_exact_tendency(N, refined):
    def field(x, y):
        return np.cos(1.3 * x + 0.4) * np.sin(2.1 * y + 0.2) + 0.3 * x * y

    errs = []
    bases = (2, 4, 8)
    for b in bases:
        f = ofo.Forest((b, b), 1 if refined else 0)
        if refined:
            flags = np.zeros(len(f), bool)
            flags[: len(f) // 3] = True
            f, _ = f.regrid(flags, 0)
        m = odg.Mesh(f, N, (1.0, 1.0))
        C = field(m.x[0], m.x[1])
        err = otr.rhs(m, C, 0.6, T, "mortar") - _exact_tendency(m, 0.6, field)
        errs.append(np.abs(err).max())
    rates = [math.log2(errs[i] / errs[i + 1]) for i in range(len(errs) - 1)]
    assert rates[-1] >= N - 0.5, (errs, rates)


def test_bell_returns_after_the_period():
    """The reversing flow brings the bell back after one period T = 5 (uniform grids, N = 4):
    the tracer total is kept to round-off and the return error shrinks under refinement
    (4 x 4: relative L2 error about 1.07, 8 x 8: 0.44; a 16 x 16 run gives 0.14)."""
    errs = []
    for b, nsteps in ((4, 250), (8, 500)):
        m = _mesh((b, b), 4)
        C0 = otr.bell(m, (0.25, 0.25), 0.25, 0.5)
        C = C0.copy()
        dt = T / nsteps
        for i in range(nsteps):
            C = otr.ssprk3_step(m, C, i * dt, dt, T)
        mass0 = otr.total(m, C0)
        assert abs(otr.total(m, C) - mass0) <= 1e-13 * mass0
        W = m.wnode[None, :] * m.J[:, None]
        errs.append(math.sqrt((W * (C - C0) ** 2).sum() / (W * C0 ** 2).sum()))
    assert errs[1] <= 0.5 * errs[0] and errs[1] <= 0.5, errs


@pytest.mark.parametrize("N", [2, 3, 4, 5])
def test_coarse_gather_evaluates_the_fine_polynomials(N):
    """Point-to-point interpolation: sum_c G[c] (fine face c values) is the fine polynomial at
    the coarse face nodes, exact for a common polynomial of degree N."""
    from oracle import basis as bmod
    nodes = bmod.lgl_nodes_weights(N)[0]
    coef = np.random.default_rng(N).standard_normal(N + 1)

    def p(x):
        return np.polyval(coef, x)
    G = otr.coarse_gather(nodes)
    fine = [p(bmod.child_map(c, nodes)) for c in (0, 1)]
    np.testing.assert_allclose(G[0] @ fine[0] + G[1] @ fine[1], p(nodes), rtol=0, atol=1e-13)
