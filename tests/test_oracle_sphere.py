"""Pins of the oracle's cubed-sphere transfer (oracle/sphere.py) against what geometry and the
method fix: the octant's area, an independent form of the spherical excess, the sphere's total
area, convergence of the isoparametric metrics to the analytic area element of the gnomonic
map, conservation through refinement and coarsening, the closed-form action on constants, and
the reduction to the reference transfer when all children have equal volumes."""
import math

import numpy as np
import pytest

import workloads
from oracle import forest as fo, sphere

R = 6.371e6


def _forest(n, rounds, p, seed, max_level=3):
    f = fo.Forest((6 * n, n), max_level)
    tmaps = []
    for k in range(rounds):
        f2, tm = f.regrid(workloads.random_flags(len(f), p, seed + k).astype(bool), 0)
        tmaps.append((f, f2, tm))
        f = f2
    return f, tmaps


def test_octant_area_is_an_eighth_of_the_sphere():
    a = sphere.spherical_excess([R, 0, 0], [0, R, 0], [0, 0, R], R)
    assert abs(a - 4 * math.pi * R * R / 8) <= 1e-15 * 4 * math.pi * R * R


def test_excess_equals_van_oosterom_strackee_form():
    rng = np.random.default_rng(3)
    for _ in range(200):
        p = rng.standard_normal((3, 3))
        p /= np.linalg.norm(p, axis=1, keepdims=True)
        a, b, c = p
        got = sphere.spherical_excess(a, b, c, 1.0)
        # tan(E/2) = |a . (b x c)| / (1 + a.b + b.c + c.a)
        want = 2.0 * math.atan2(abs(np.dot(a, np.cross(b, c))), 1.0 + a @ b + b @ c + c @ a)
        assert abs(got - want) <= 1e-12


@pytest.mark.parametrize("n,rounds", [(1, 0), (2, 2), (3, 3)])
def test_total_area_is_the_sphere_at_any_refinement(n, rounds):
    f, _ = _forest(n, rounds, 0.3, seed=10 + n)
    m = sphere.SphereMesh(f, 3, n, R)
    total = 4 * math.pi * R * R
    assert abs(m.area.sum() - total) <= 1e-12 * total
    for t in range(6):
        assert abs(m.area[m.tile == t].sum() - total / 6) <= 1e-12 * total


def test_isoparametric_metrics_converge_to_the_gnomonic_area_element():
    """J of the interpolated surface against the analytic metric of the equiangular map,
    r^2 sec^2(a) sec^2(b) / (1 + tan^2 a + tan^2 b)^(3/2) (d alpha/d xi)(d beta/d eta)."""
    n = 2
    f = fo.Forest((6 * n, n), 0)
    errs = []
    for N in (2, 4, 6, 8):
        m = sphere.SphereMesh(f, N, n, R)
        a, b = m.alpha, m.beta
        X, Y = np.tan(a), np.tan(b)
        h = (math.pi / 2) / n / 2.0          # d alpha / d xi on a level-0 element
        exact = R * R / (np.cos(a) ** 2 * np.cos(b) ** 2) / (1 + X * X + Y * Y) ** 1.5 * h * h
        errs.append(np.abs(m.J - exact).max() / exact.max())
        iso = m.W.sum()
        assert abs(iso - 4 * math.pi * R * R) <= 10 * errs[-1] * 4 * math.pi * R * R
    assert errs[-1] < 1e-6 and all(errs[k + 1] < 0.05 * errs[k] for k in range(3))


def _fields(m, seed):
    """Positive smooth fields (a tracer-like total) plus a sign-changing one."""
    rng = np.random.default_rng(seed)
    x = m.x / R
    q = np.empty((3, len(m.forest), m.np_))
    q[0] = 2.0 + np.sin(3 * x[..., 0]) * np.cos(2 * x[..., 1]) + x[..., 2]
    q[1] = 1.0 + 0.5 * np.exp(-4 * ((x[..., 0] - 0.6) ** 2 + x[..., 1] ** 2))
    q[2] = np.sin(2 * x[..., 2]) + 0.3 + 0.01 * rng.standard_normal(q[2].shape)
    return q


@pytest.mark.parametrize("N", [3, 4])
def test_transfer_conserves_every_integral(N):
    n = 2
    f0 = fo.Forest((6 * n, n), 3)
    m = sphere.SphereMesh(f0, N, n, R)
    q = _fields(m, 1)
    I0 = m.integrals(q)
    rng = np.random.default_rng(4)
    for k in range(5):
        # refine at random, then coarsen everywhere it is allowed, alternately
        tag = rng.random(len(m.forest)) < (0.4 if k % 2 == 0 else 0.0)
        f2, tm = m.forest.regrid(tag, 0)
        m2 = sphere.SphereMesh(f2, N, n, R)
        q = sphere.transfer(q, m, m2, tm)
        m = m2
        np.testing.assert_allclose(m.integrals(q), I0, rtol=2e-14, atol=0)
    assert max(lf[0] for lf in m.forest.leaves) > 0


def test_constant_scales_by_the_isoparametric_area_ratio():
    """Refinement of a constant c: P_c keeps c, the scale factor makes each child c A_p / sum A_c
    with A = sum W the isoparametric areas (the geometry of the children differs from the
    parent's).  Coarsening maps constant children to that constant times the inverse ratio."""
    n, N = 1, 3
    f0 = fo.Forest((6 * n, n), 2)
    m0 = sphere.SphereMesh(f0, N, n, R)
    tag = np.zeros(len(f0), bool)
    tag[[0, 3]] = True
    f1, tm = f0.regrid(tag, 0)
    m1 = sphere.SphereMesh(f1, N, n, R)
    q0 = np.full((1, len(f0), m0.np_), 5.0)
    q1 = sphere.transfer(q0, m0, m1, tm)
    for k, entry in enumerate(tm):
        if entry[0] == "child":
            kids = [kk for kk, e in enumerate(tm) if e[0] == "child" and e[1] == entry[1]]
            ratio = m0.W[entry[1]].sum() / m1.W[kids].sum()
            np.testing.assert_allclose(q1[0, k], 5.0 * ratio, rtol=1e-14)
        elif entry[0] == "keep":
            assert np.all(q1[0, k] == 5.0)
    assert not np.allclose(q1, 5.0)   # the curved geometry does change on refinement
    f2, tm2 = f1.regrid(np.zeros(len(f1), bool), 0)
    m2 = sphere.SphereMesh(f2, N, n, R)
    q2 = sphere.transfer(np.full((1, len(f1), m1.np_), 5.0), m1, m2, tm2)
    for k, entry in enumerate(tm2):
        if entry[0] == "parent":
            ratio = m1.W[list(entry[1])].sum() / m2.W[k].sum()
            np.testing.assert_allclose(q2[0, k], 5.0 * ratio, rtol=1e-13)


def test_equal_volumes_reduce_coarsening_to_the_reference_restriction():
    """With the reference weights the restriction is the box transfer's parent formula up to
    the scale factor; the volume weights give the same result where the children's areas are
    equal and a different one where they are not (two roots per tile: no root is symmetric)."""
    n, N = 2, 3
    f0 = fo.Forest((6 * n, n), 1)
    f1, _ = f0.regrid(np.ones(len(f0), bool), 0)
    m1 = sphere.SphereMesh(f1, N, n, R)
    q1 = _fields(m1, 2)
    f2, tm = f1.regrid(np.zeros(len(f1), bool), 0)
    m2 = sphere.SphereMesh(f2, N, n, R)
    ref = sphere.transfer(q1, m1, m2, tm, volume_weights=False)
    vol = sphere.transfer(q1, m1, m2, tm, volume_weights=True)
    B = m1.basis
    differ = 0
    for k, entry in enumerate(tm):
        assert entry[0] == "parent"
        kids = list(entry[1])
        acc = sum(m1.apply_1d(B.C[(ci >> 1) & 1], m1.apply_1d(B.C[ci & 1], q1[:, e], 0), 1)
                  for ci, e in enumerate(kids))
        s = ref[:, k, 0] / acc[:, 0]
        np.testing.assert_allclose(ref[:, k], acc * s[:, None], rtol=1e-14)
        V = m1.area[kids]
        if np.ptp(V) <= 1e-12 * V.mean():
            np.testing.assert_allclose(vol[:, k], ref[:, k], rtol=1e-11)
        else:
            assert not np.allclose(vol[:, k], ref[:, k], rtol=1e-6)
            differ += 1
    assert differ > 0


def test_planted_mistakes_break_conservation():
    """A copy of the transfer without the scale factor no longer conserves.  (A uniform error in
    the volume weights would be absorbed by that factor; their shape is pinned above.)"""
    n, N = 1, 3
    f0 = fo.Forest((6 * n, n), 2)
    m0 = sphere.SphereMesh(f0, N, n, R)
    q0 = _fields(m0, 5)
    f1, tm = f0.regrid(np.ones(len(f0), bool), 0)
    m1 = sphere.SphereMesh(f1, N, n, R)
    orig = sphere._scale
    try:
        sphere._scale = lambda q_new, W_new, I_old: np.ones(q_new.shape[0])
        q1 = sphere.transfer(q0, m0, m1, tm)
    finally:
        sphere._scale = orig
    err = np.abs(m1.integrals(q1) - m0.integrals(q0)) / np.abs(m0.integrals(q0))
    assert err.max() > 1e-6


def test_tile_points_lie_on_the_sphere_and_cover_it_once():
    """Every tile point has norm r; tile t's centre is its axis (+x, +y, -x, -y, +z, -z); inside
    a tile the axis of the centre is the point's dominant one (the six tiles do not overlap);
    along the equator belt the edge alpha = pi/4 of tile t is the edge alpha = -pi/4 of tile
    t + 1 (mod 4) at the same beta."""
    axes = np.array([[1, 0, 0], [0, 1, 0], [-1, 0, 0], [0, -1, 0], [0, 0, 1], [0, 0, -1]], float)
    g = np.random.default_rng(3)
    a, b = g.uniform(-math.pi / 4, math.pi / 4, (2, 200)) * 0.999
    for t in range(6):
        p = sphere.tile_point(t, a, b, R)
        np.testing.assert_allclose(np.linalg.norm(p, axis=-1), R, rtol=1e-15)
        np.testing.assert_allclose(sphere.tile_point(t, 0.0, 0.0, R), R * axes[t], atol=1e-9)
        dom = np.argmax(np.abs(p), axis=-1)
        sgn = np.sign(p[np.arange(len(dom)), dom])
        np.testing.assert_array_equal(dom, np.argmax(np.abs(axes[t])))
        np.testing.assert_array_equal(sgn, axes[t].sum())
    for t in range(4):
        edge = np.full_like(b, math.pi / 4)
        np.testing.assert_allclose(sphere.tile_point(t, edge, b, R),
                                   sphere.tile_point((t + 1) % 4, -edge, b, R), atol=1e-8)
