"""Pins of the oracle's dGSEM operator, time stepping, transfer and integrals.

Every check rests on something the mathematics fixes (exact zeros, conservation, convergence
towards an independently differentiated exact tendency, closed-form integrals, the RK3
stability polynomial), not on the oracle itself.
"""
import math

import numpy as np
import pytest
from scipy import integrate

from oracle import dg, forest as fo, physics

K = physics.Constants()


def _hanging_forest(base, max_level=2, seed=0):
    """A forest with hanging faces on every axis and both sub-face positions."""
    f = fo.Forest(base, max_level)
    rng = np.random.default_rng(seed)
    for _ in range(max_level):
        tag = rng.random(len(f)) < 0.25
        f, _ = f.regrid(tag, 0)
    return f


def _random_state(mesh, seed):
    rng = np.random.default_rng(seed)
    q = np.empty((mesh.nv, mesh.E, mesh.np_))
    q[0] = 1e-3 * rng.standard_normal(q[0].shape)
    q[1:1 + mesh.d] = 2.0 * rng.standard_normal(q[1:1 + mesh.d].shape)
    q[1 + mesh.d] = 0.3 * rng.standard_normal(q[0].shape)
    return q


MESHES = [((3, 3), (3000.0, 3000.0), 4), ((4, 2), (2000.0, 1000.0), 3),
          ((2, 2, 2), (2000.0, 2000.0, 2000.0), 2), ((2, 1, 2), (1000.0, 500.0, 1000.0), 3)]


@pytest.mark.parametrize("base,L,N", MESHES)
def test_rest_state_exactly_zero(base, L, N):
    mesh = dg.Mesh(_hanging_forest(base), N, L, K)
    assert any(True for _ in mesh.forest.face_lists()[1])
    r = dg.rhs(mesh, np.zeros((mesh.nv, mesh.E, mesh.np_)))
    assert np.all(r == 0.0)


@pytest.mark.parametrize("base,L,N", MESHES)
def test_free_stream_preserved_on_hanging_faces(base, L, N):
    K0 = physics.Constants(g=0.0)
    f = _hanging_forest(tuple(b + 2 for b in base), seed=1)
    mesh = dg.Mesh(f, N, L, K0)
    q = np.zeros((mesh.nv, mesh.E, mesh.np_))
    q[0] = 0.01
    q[1:1 + mesh.d] = np.array([3.0, -2.0, 1.5][:mesh.d])[:, None, None]
    q[1 + mesh.d] = 0.5
    r = dg.rhs(mesh, q)
    _, mort, bnd = f.face_lists()
    walls = {e for e, _, _ in bnd}
    inner = [e for e in range(mesh.E) if e not in walls]
    assert inner and any(m[0] in inner for m in mort)
    scale = max(np.abs(physics.flux(q[:, inner], dg._bg_at(mesh, inner), K0, a)).max()
                for a in range(mesh.d)) / min(mesh.h.min(), 1.0)
    assert np.abs(r[:, inner]).max() <= 1e-13 * scale


@pytest.mark.parametrize("base,L,N", MESHES)
def test_discrete_conservation_of_mass_and_theta(base, L, N):
    mesh = dg.Mesh(_hanging_forest(base, seed=2), N, L, K)
    q = _random_state(mesh, 3)
    r = dg.rhs(mesh, q)
    W = mesh.wnode[None, :] * mesh.J[:, None]
    for v in (0, mesh.d + 1):
        total = math.fsum((W * r[v]).ravel())
        scale = math.fsum(np.abs(W * r[v]).ravel())
        assert abs(total) <= 1e-14 * scale


def _smooth_q(x, L, d):
    """Smooth state with zero normal velocity on every wall of [0, L]^d."""
    c = [np.cos(np.pi * x[a] / L[a]) for a in range(d)]
    s = [np.sin(np.pi * x[a] / L[a]) for a in range(d)]
    zrel = x[d - 1] / L[d - 1]
    rp = 1e-3 * c[0] * np.cos(2 * np.pi * zrel) + 2e-4 * s[d - 1]
    U = []
    for a in range(d):
        val = (2.0 - 0.5 * a) * s[a]
        for b in range(d):
            if b != a:
                val = val * c[b]
        U.append(val)
    Tp = 0.3 * c[0] * np.sin(2 * np.pi * zrel) + 0.1
    if d == 3:
        Tp = Tp + 0.2 * c[1]
    return np.stack([rp] + U + [Tp])


def _exact_tendency(qfun, x, Kc):
    """-div F + S of the analytic field, derivatives by complex step."""
    d = len(x)
    out = physics.source(qfun(x), Kc).astype(complex)
    hstep = 1e-30
    for a in range(d):
        xc = [xi.astype(complex) for xi in x]
        xc[a] = xc[a] + 1j * hstep
        q = qfun(xc)
        F = physics.flux(q, physics.background(xc[d - 1], Kc), Kc, a)
        out = out - F.imag / hstep
    return out.real


def _convergence(N, d, refine, qfun_of_L, L, Kc, bases):
    errs = []
    for nb in bases:
        f = fo.Forest((nb,) * d, 1)
        if refine:
            tag = np.zeros(len(f), dtype=bool)
            tag[len(f) // 2] = True
            tag[len(f) // 4 + 1] = True
            f, _ = f.regrid(tag, 0)
            assert f.face_lists()[1]
        mesh = dg.Mesh(f, N, L, Kc)
        qf = qfun_of_L
        r = dg.rhs(mesh, qf(list(mesh.x)))
        ex = _exact_tendency(qf, list(mesh.x), Kc)
        # mass, momentum (one scale for all components), Theta
        groups = [[0], list(range(1, 1 + d)), [1 + d]]
        errs.append(max(np.abs(r[g] - ex[g]).max() / np.abs(ex[g]).max() for g in groups))
    return np.log2(np.array(errs[:-1]) / np.array(errs[1:])), errs


@pytest.mark.parametrize("N", [2, 3, 4])
@pytest.mark.parametrize("refine", [False, True])
def test_convergence_order_2d(N, refine):
    L = (1000.0, 1000.0)
    rates, errs = _convergence(N, 2, refine, lambda x: _smooth_q(x, L, 2), L, K, (4, 8, 16))
    assert rates[-1] >= N - 0.35, (rates, errs)


def test_convergence_order_3d():
    L = (1000.0, 1000.0, 1000.0)
    rates, errs = _convergence(3, 3, True, lambda x: _smooth_q(x, L, 3), L, K, (2, 4, 8))
    assert rates[-1] >= 3 - 0.35, (rates, errs)


@pytest.mark.parametrize("refine", [False, True])
def test_other_hydrostatic_atmosphere_converges_to_rest(refine):
    # a neutral atmosphere with theta = theta0 + 5 K is also at rest; expressed as a perturbation
    # of the theta0 background its tendency must vanish as h -> 0 (pins gravity's sign and size)
    L = (1000.0, 2000.0)
    th2 = K.theta0 + 5.0

    def q_alt(x):
        z = x[1]
        pi2 = 1.0 - K.g * z / (K.cp * th2)
        rho2 = K.p0 * pi2 ** (K.cv / K.R) / (K.R * th2)
        rb, Tb, _ = physics.background(z, K)
        zero = 0.0 * z
        return np.stack([rho2 - rb, zero, zero, rho2 * th2 - Tb])

    N = 3
    errs = []
    for nb in (2, 4, 8):
        f = fo.Forest((nb, nb), 1)
        if refine:
            tag = np.zeros(len(f), dtype=bool)
            tag[len(f) // 2] = True
            f, _ = f.regrid(tag, 0)
        mesh = dg.Mesh(f, N, L, K)
        r = dg.rhs(mesh, q_alt(list(mesh.x)))
        # scale: the buoyancy term rho' g
        scale = np.abs(q_alt(list(mesh.x))[0]).max() * K.g
        errs.append(np.abs(r[2]).max() / scale)
    rate = math.log2(errs[-2] / errs[-1])
    assert errs[-1] < 1e-5 and rate >= N - 0.5, errs


def test_mirror_symmetry_of_centred_bubble():
    f = fo.Forest((6, 4), 1)
    mesh = dg.Mesh(f, 4, (1200.0, 800.0), K)
    th = dg.bubble_theta(mesh, (600.0, 300.0), (250.0, 250.0), 0.25)
    q = dg.state_from_theta(mesh, th)
    q[1] = 0.3 * np.sin(np.pi * (mesh.x[0] - 600.0) / 600.0)   # odd in x about the centre
    r = dg.rhs(mesh, q)
    # mirror map x -> 1200 - x: element (ix, iz) -> (5 - ix, iz), node i -> N - i
    n1 = mesh.n1
    err = 0.0
    for e, (l, c) in enumerate(f.leaves):
        em = f.index(l, (5 - c[0], c[1]))
        a = r[:, e].reshape(mesh.nv, n1, n1)
        b = r[:, em].reshape(mesh.nv, n1, n1)[:, :, ::-1]
        sgn = np.array([1, -1, 1, 1])[:, None, None]
        err = max(err, np.abs(a - sgn * b).max() / (np.abs(r).max()))
    assert err < 1e-12


def test_ssprk3_stability_polynomial():
    for lam_dt in (-0.3, -1.0, 0.5 + 0.7j, -2.0 + 1.0j):
        y = dg.ssprk3_step(np.array([1.0 + 0j]), 1.0, lambda s: lam_dt * s)
        z = lam_dt
        assert abs(y[0] - (1 + z + z * z / 2 + z ** 3 / 6)) < 1e-15


def test_rusanov_dissipation_keeps_noise_bounded():
    # white noise of small amplitude on the rising-bubble mesh; anti-dissipation would blow up
    f = fo.Forest((10, 10), 0)
    mesh = dg.Mesh(f, 4, (1000.0, 1000.0), K)
    rng = np.random.default_rng(0)
    q = np.zeros((mesh.nv, mesh.E, mesh.np_))
    q[1:3] = 1e-3 * rng.standard_normal(q[1:3].shape)
    e0 = np.abs(q).max()
    q = dg.step(mesh, q, 0.02, 20)
    assert np.all(np.isfinite(q)) and np.abs(q[1:3]).max() < 2 * e0


@pytest.mark.parametrize("base,N", [((3, 3), 4), ((2, 2, 2), 3)])
def test_transfer_refine_coarsen_identity_and_mass(base, N):
    L = tuple(1000.0 for _ in base)
    f = fo.Forest(base, 2)
    m0 = dg.Mesh(f, N, L, K)
    q0 = _random_state(m0, 4)
    tag = np.zeros(len(f), dtype=bool)
    tag[[0, len(f) - 1]] = True
    f1, t1 = f.regrid(tag, 0)
    m1 = dg.Mesh(f1, N, L, K)
    q1 = dg.transfer(q0, m0, m1, t1)
    W0 = m0.wnode[None, :] * m0.J[:, None]
    W1 = m1.wnode[None, :] * m1.J[:, None]
    for v in range(m0.nv):
        a = math.fsum((W0 * q0[v]).ravel())
        b = math.fsum((W1 * q1[v]).ravel())
        assert abs(a - b) <= 1e-13 * math.fsum(np.abs(W0 * q0[v]).ravel())
    f2, t2 = f1.regrid(np.zeros(len(f1), dtype=bool), 0)
    assert f2.leaves == f.leaves
    q2 = dg.transfer(q1, m1, dg.Mesh(f2, N, L, K), t2)
    np.testing.assert_allclose(q2, q0, rtol=0, atol=1e-13 * np.abs(q0).max())
    # coarsening an arbitrary (non-polynomial) fine field also conserves the discrete mass
    q1r = _random_state(m1, 5)
    q2r = dg.transfer(q1r, m1, dg.Mesh(f2, N, L, K), t2)
    W2 = W0
    for v in range(m0.nv):
        a = math.fsum((W1 * q1r[v]).ravel())
        b = math.fsum((W2 * q2r[v]).ravel())
        assert abs(a - b) <= 1e-13 * math.fsum(np.abs(W1 * q1r[v]).ravel())


def test_integrals_of_rest_atmosphere_closed_form():
    Lx, H = 1000.0, 10000.0
    mesh = dg.Mesh(_hanging_forest((2, 5), seed=4), 5, (Lx, H), K)
    I = dg.integrals(mesh, np.zeros((mesh.nv, mesh.E, mesh.np_)))
    p = lambda z: physics.hydrostatic_pressure(z, K)
    # hydrostatic: int rho dz = (p(0) - p(H)) / g
    assert abs(I[0] - Lx * (p(0.0) - p(H)) / K.g) <= 1e-12 * I[0]
    # energy: int (p cv/R + rho g z) dz = (cv/R + 1) int p dz - p(H) H   (integration by parts)
    ip, _ = integrate.quad(p, 0.0, H, epsabs=0, epsrel=1e-13)
    e_ref = Lx * ((K.cv / K.R + 1.0) * ip - p(H) * H)
    assert abs(I[1] - e_ref) <= 1e-11 * e_ref
    assert I[2] == 0.0 and I[4] == 0.0
    assert abs(I[3] - Lx * H) <= 1e-12 * Lx * H


def test_bubble_initial_state_round_trip():
    f = fo.Forest((10, 10), 0)
    mesh = dg.Mesh(f, 4, (1000.0, 1000.0), K)
    th = dg.bubble_theta(mesh, (500.0, 350.0), (250.0, 250.0), 0.25)
    q = dg.state_from_theta(mesh, th)
    np.testing.assert_allclose(dg.theta_prime(mesh, q), th, rtol=0, atol=1e-12)
    assert abs(dg.theta_prime(mesh, q).max() - 0.5) < 1e-3      # theta_c = 0.5 K (Sec. 4.3)
    rb, Tb, pb = mesh.bg
    assert np.all(physics.pressure_perturbation(q[3], Tb, pb, K) == 0.0)


def test_rhs_subset_equals_full():
    mesh = dg.Mesh(_hanging_forest((3, 3), seed=6), 3, (900.0, 900.0), K)
    q = _random_state(mesh, 7)
    full = dg.rhs(mesh, q)
    sub = np.array([0, 3, mesh.E - 1])
    part = dg.rhs(mesh, q, elems=sub)
    np.testing.assert_array_equal(part[:, sub], full[:, sub])


@pytest.mark.parametrize("base,N,L", [((4, 4), 3, (1200.0, 1200.0)), ((3, 2, 3), 2, (900.0, 600.0, 900.0))])
def test_step_on_sampled_elements_equals_the_full_step(base, N, L):
    """step_on restricts one SSP-RK3 step to the elements a sample needs (two face hops for
    stage 1, one for stage 2): on the sample it gives the full step's values bit for bit, also
    for elements whose neighbourhood crosses hanging faces."""
    mesh = dg.Mesh(_hanging_forest(base, seed=8), N, L, K)
    q = 1e-2 * _random_state(mesh, 9)
    full = dg.step(mesh, q, 0.01, 1)
    _, mort, _ = mesh.forest.face_lists()
    sample = np.unique([0, mesh.E // 2, mesh.E - 1] + [int(mort[0][0])])
    part = dg.step_on(mesh, q, 0.01, sample)
    np.testing.assert_array_equal(part[:, sample], full[:, sample])
    others = np.setdiff1d(np.arange(mesh.E), sample)
    assert np.all(np.isnan(part[:, others]))
    # a stage short of the two-hop neighbourhood would not be exact: drop the second hop
    hop1 = set(sample.tolist())
    for e in sample:
        hop1 |= set(mesh.forest.face_neighbors(int(e)))
    s1 = np.array(sorted(hop1))
    q1 = q.copy()
    q1[:, s1] = q[:, s1] + 0.01 * dg.rhs(mesh, q, elems=s1)[:, s1]
    q2 = q.copy()
    q2[:, s1] = 0.75 * q[:, s1] + 0.25 * (q1[:, s1] + 0.01 * dg.rhs(mesh, q1, elems=s1)[:, s1])
    short = (1.0 / 3.0) * q + (2.0 / 3.0) * (q2 + 0.01 * dg.rhs(mesh, q2, elems=sample))
    assert not np.array_equal(short[:, sample], full[:, sample])
