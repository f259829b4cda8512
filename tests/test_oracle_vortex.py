"""Pins of the isentropic vortex (Sec. 4.1) and of the right-hand side on periodic meshes: the
isentropic relations, the free stream far away, exact preservation of a uniform stream across
periodic and hanging faces, conservation, the wrap-around of the exact solution, and
convergence of the right-hand side to the exact time derivative of the moving vortex."""
import math

import numpy as np
import pytest

import workloads
from oracle import dg as odg, forest as ofo, physics, vortex as ovx

K = ovx.constants()
L = (12.0, 12.0)
CENTER, BETA, UINF = (6.0, 6.0), 5.0, (1.0, 1.0)


def _mesh(base, N, level=0, p=0.0, seed=0):
    f = ofo.Forest(base, level, periodic=(True, True))
    if level:
        flags = workloads.random_flags(len(f), p, seed)
        flags[0] = 1
        f, _ = f.regrid(flags.astype(bool), 0)
    return odg.Mesh(f, N, L, K)


def test_constants_are_the_nondimensional_air():
    assert K.gamma == 1.4 and K.R == 1.0 and K.p0 == 1.0 and K.theta0 == 1.0 and K.g == 0.0
    m = _mesh((2, 2), 2)
    rb, Tb, pb = m.bg
    assert np.all(rb == 1.0) and np.all(Tb == 1.0) and np.all(pb == 1.0)


def test_isentropic_relations_and_far_field():
    m = _mesh((8, 8), 3)
    q = ovx.vortex_state(m, CENTER, BETA, UINF)
    rho = 1.0 + q[0]
    Theta = 1.0 + q[3]
    p = physics.eos_pressure(Theta, K)
    np.testing.assert_allclose(p, rho ** 1.4, rtol=1e-13)
    np.testing.assert_allclose(Theta / rho, 1.0, rtol=1e-15)
    r = np.hypot(m.x[0] - 6.0, m.x[1] - 6.0)
    far = r > 5.5
    assert np.abs(q[0][far]).max() <= 1e-9
    np.testing.assert_allclose(q[1][far] / rho[far], 1.0, atol=2e-6)
    # centre: T = 1 - 0.4 * 25 / (8 * 1.4 * pi^2) e
    T0 = 1.0 - 0.4 * 25.0 / (8.0 * 1.4 * math.pi ** 2) * math.e
    assert abs(rho.min() - T0 ** 2.5) <= 0.05


def test_exact_solution_wraps_around():
    m = _mesh((4, 4), 3)
    q0 = ovx.vortex_state(m, CENTER, BETA, UINF, 0.0)
    q12 = ovx.vortex_state(m, CENTER, BETA, UINF, 12.0)    # one box length in each direction
    np.testing.assert_allclose(q12, q0, rtol=0, atol=1e-12)


@pytest.mark.parametrize("N", [2, 3, 4])
def test_uniform_stream_is_preserved_on_periodic_hanging_meshes(N):
    m = _mesh((3, 3), N, level=1, p=0.4, seed=N)
    assert len(m.forest.face_lists()[1]) > 0 and len(m.forest.face_lists()[2]) == 0
    q = np.zeros((4, m.E, m.np_))
    q[1], q[2] = 1.0, -0.5
    r = odg.rhs(m, q)
    assert np.abs(r).max() <= 1e-13 * 2.0


@pytest.mark.parametrize("N", [2, 3])
def test_conservation_on_periodic_hanging_meshes(N):
    m = _mesh((3, 4), N, level=1, p=0.4, seed=10 + N)
    q = ovx.vortex_state(m, CENTER, BETA, UINF) + 0.01 * workloads.random_state(4, m.E, m.np_, seed=N)
    r = odg.rhs(m, q)
    W = m.wnode[None, :] * m.J[:, None]
    for v in range(4):
        scale = np.abs(W * r[v]).sum()
        # total mass, momentum (no gravity) and Theta' are conserved without walls
        assert abs(math.fsum((W * r[v]).ravel())) <= 1e-13 * scale


@pytest.mark.parametrize("N,refined", [(3, False), (3, True)])
def test_rhs_converges_to_the_moving_vortex(N, refined):
    errs = []
    for b in (8, 16, 32):
        f = ofo.Forest((b, b), 1 if refined else 0, periodic=(True, True))
        if refined:
            tag = np.array([abs(f.box(e)[0][0] - (b << (ofo.MAXL - 1))) < (b << ofo.MAXL) // 4
                            for e in range(len(f))])
            f, _ = f.regrid(tag, 0)
        m = odg.Mesh(f, N, L, K)
        q = ovx.vortex_state(m, CENTER, BETA, UINF, 0.3)
        dt = 1e-5
        dqdt = (ovx.vortex_state(m, CENTER, BETA, UINF, 0.3 + dt)
                - ovx.vortex_state(m, CENTER, BETA, UINF, 0.3 - dt)) / (2 * dt)
        errs.append(np.abs(odg.rhs(m, q) - dqdt).max())
    rates = [math.log2(errs[i] / errs[i + 1]) for i in range(2)]
    assert rates[-1] >= N - 0.5, (errs, rates)
