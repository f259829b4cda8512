"""Pins of the oracle's physics: paper values, closed forms, characteristic speeds."""
import json
import os

import mpmath
import numpy as np
import pytest

from oracle import physics

GOLDEN = json.load(open(os.path.join(os.path.dirname(__file__), "golden", "paper_values.json")))
K = physics.Constants()


def test_sound_speed_matches_paper():
    g = GOLDEN["sound_speed_surface"]
    rb, Tb, pb = physics.background(0.0, K)
    c = physics.sound_speed(pb, rb, K)
    assert abs(c - g["value_m_per_s"]) < g["rounding_m_per_s"]


def test_background_is_closed_form_hydrostatic():
    z = np.linspace(0.0, 10000.0, 41)
    rb, Tb, pb = physics.background(z, K)
    np.testing.assert_allclose(pb, physics.hydrostatic_pressure(z, K), rtol=2e-15)
    np.testing.assert_allclose(Tb / rb, K.theta0, rtol=1e-15)
    # ideal gas: p = rho R T with T = theta0 * pi
    np.testing.assert_allclose(pb, rb * K.R * K.theta0 * physics.exner(z, K), rtol=1e-14)


def test_background_satisfies_hydrostatic_balance():
    # dp_bar/dz = -rho_bar g, derivative by complex step (independent of any formula retyping)
    z = np.linspace(0.0, 10000.0, 21)
    hstep = 1e-20
    dp = physics.background(z + 1j * hstep, K)[2].imag / hstep
    rb = physics.background(z, K)[0]
    np.testing.assert_allclose(dp, -rb * K.g, rtol=1e-13)


def test_pressure_perturbation_against_high_precision():
    mpmath.mp.dps = 50
    rb, Tb, pb = physics.background(np.array([0.0, 3000.0, 9000.0]), K)
    for k in range(3):
        for tp in (-5.0, -1e-3, 1e-9, 0.02, 2.5):
            got = physics.pressure_perturbation(tp, Tb[k], pb[k], K)
            T0 = mpmath.mpf(Tb[k])
            P = lambda T: K.p0 * (mpmath.mpf(K.R) * T / K.p0) ** (mpmath.mpf(K.cp) / mpmath.mpf(K.cv))
            ref = P(T0 + mpmath.mpf(tp)) - P(T0)
            # the oracle's p_bar is the double-rounded P(Theta_bar); compare relative to p'
            assert abs(got - float(ref)) <= 1e-14 * abs(float(ref)) + 1e-12 * 1e-16 * float(P(T0))


def test_rest_has_zero_pressure_perturbation():
    rb, Tb, pb = physics.background(np.linspace(0, 5000, 11), K)
    assert np.all(physics.pressure_perturbation(np.zeros(11), Tb, pb, K) == 0.0)


def _jacobian(q, bg, axis):
    nv = q.shape[0]
    J = np.zeros((nv, nv))
    hstep = 1e-30
    for j in range(nv):
        qc = q.astype(complex)
        qc[j] += 1j * hstep
        J[:, j] = physics.flux(qc, bg, K, axis).imag / hstep
    return J


@pytest.mark.parametrize("d", [2, 3])
@pytest.mark.parametrize("axis", [0, 1, 2])
def test_flux_characteristic_speeds(d, axis):
    # the Euler flux Jacobian has eigenvalues u_a - c, u_a (d-fold), u_a + c
    if axis >= d:
        pytest.skip("axis beyond dimension")
    rng = np.random.default_rng(7 + d + axis)
    z = 1234.0
    bg = physics.background(np.array(z), K)
    q = np.zeros(d + 2)
    q[0] = 0.01 * rng.standard_normal()
    q[1:1 + d] = 20.0 * rng.standard_normal(d)
    q[1 + d] = 3.0 * rng.standard_normal()
    J = _jacobian(q, bg, axis)
    ev = np.sort(np.linalg.eigvals(J).real)
    rho, u, Theta, pp, P = physics.primitives(q, bg, K)
    c = physics.sound_speed(P, rho, K)
    want = np.sort([u[axis] - c] + [u[axis]] * d + [u[axis] + c])
    np.testing.assert_allclose(ev, want, rtol=1e-9, atol=1e-9)


@pytest.mark.parametrize("d", [2, 3])
def test_rusanov_consistency_and_dissipation(d):
    rng = np.random.default_rng(11)
    bg = physics.background(np.array([500.0]), K)
    q = np.zeros((d + 2, 1))
    q[0] = 1e-3
    q[1:1 + d, 0] = rng.standard_normal(d)
    q[1 + d] = 0.4
    for a in range(d):
        Fs, Fm, Fp = physics.rusanov(q, q, bg, bg, K, a)
        np.testing.assert_allclose(Fs, Fm, rtol=1e-15, atol=0)
    # fluid at rest with more Theta on the high side: dissipation moves Theta towards the low side
    qm = np.zeros((d + 2, 1))
    qp = np.zeros((d + 2, 1))
    qp[1 + d] = 1.0
    Fs, _, _ = physics.rusanov(qm, qp, bg, bg, K, 0)
    assert Fs[1 + d, 0] < 0.0


@pytest.mark.parametrize("d", [2, 3])
def test_wall_mirror_blocks_mass(d):
    rng = np.random.default_rng(3)
    bg = physics.background(np.array([200.0, 800.0]), K)
    q = rng.standard_normal((d + 2, 2))
    q[0] *= 1e-3
    for a in range(d):
        Fs, _, _ = physics.rusanov(q, physics.wall_mirror(q, a), bg, bg, K, a)
        assert np.all(Fs[0] == 0.0)
        assert np.all(Fs[1 + d] == 0.0)
