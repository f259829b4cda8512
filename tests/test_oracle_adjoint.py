"""Pins of the oracle's discrete adjoint: complex-step derivatives against central finite
differences of the same oracle, the local-support shortcut, the real-input equivalence of the
complex-step-safe |.| and max."""
import numpy as np
import pytest

from oracle import adjoint, dg, forest as fo, physics


def _mesh(base, N, L, seed=0):
    f = fo.Forest(base, 1)
    rng = np.random.default_rng(seed)
    f, _ = f.regrid(rng.random(len(f)) < 0.4, 0)
    return dg.Mesh(f, N, L)


def _state(mesh, seed):
    rng = np.random.default_rng(seed)
    q = np.empty((mesh.nv, mesh.E, mesh.np_))
    q[0] = 1e-3 * rng.standard_normal(q[0].shape)
    q[1:1 + mesh.d] = rng.standard_normal(q[1:1 + mesh.d].shape)
    q[1 + mesh.d] = 0.2 * rng.standard_normal(q[0].shape)
    return q


def test_cs_helpers_equal_numpy_on_real_input():
    rng = np.random.default_rng(1)
    a, b = rng.standard_normal((2, 50))
    a[0] = 0.0
    assert np.array_equal(physics.abs_cs(a), np.abs(a))
    assert np.array_equal(physics.max_cs(a, b), np.maximum(a, b))


@pytest.mark.parametrize("base,N,L", [((2, 2), 2, (1000.0, 1000.0)), ((2, 1, 2), 1, (800.0, 400.0, 800.0))])
def test_rhs_vjp_inner_product_against_finite_differences(base, N, L):
    m = _mesh(base, N, L)
    q = _state(m, 2)
    rng = np.random.default_rng(3)
    lam = rng.standard_normal(q.shape)
    v = rng.standard_normal(q.shape)
    jt = adjoint.rhs_vjp(m, q, lam)
    h = 1e-7
    fd = (dg.rhs(m, q + h * v) - dg.rhs(m, q - h * v)) / (2 * h)
    lhs, rhs = np.sum(lam * fd), np.sum(jt * v)
    assert abs(lhs - rhs) <= 1e-7 * abs(rhs)


def test_rhs_vjp_local_support_matches_full_evaluation():
    m = _mesh((2, 2), 2, (1000.0, 1000.0), seed=4)
    q = _state(m, 5)
    lam = np.random.default_rng(6).standard_normal(q.shape)
    a = adjoint.rhs_vjp(m, q, lam, local=True)
    b = adjoint.rhs_vjp(m, q, lam, local=False)
    np.testing.assert_allclose(a, b, rtol=0, atol=1e-13 * np.abs(b).max())


def test_ke_functional_is_the_integral():
    m = _mesh((2, 2), 3, (1000.0, 1000.0), seed=7)
    q = _state(m, 8)
    assert abs(adjoint.ke_functional(m, q) - dg.integrals(m, q)[2]) <= 1e-12 * dg.integrals(m, q)[2]


def test_final_ke_gradient_against_finite_differences():
    m = _mesh((2, 2), 2, (1000.0, 1000.0), seed=9)
    rng = np.random.default_rng(10)
    theta = 0.5 * rng.standard_normal((m.E, m.np_))
    nodes = [3, 17, m.E * m.np_ - 2]
    g = adjoint.final_ke_gradient(m, theta, 0.01, 3, nodes)
    for k, j in enumerate(nodes):
        h = 1e-4
        tp, tm = theta.copy(), theta.copy()
        tp.flat[j] += h
        tm.flat[j] -= h
        fd = (adjoint.final_ke(m, tp, 0.01, 3) - adjoint.final_ke(m, tm, 0.01, 3)) / (2 * h)
        assert abs(fd - g[k]) <= 1e-6 * np.abs(g).max()


# ---- step_vjp: the transpose of one SSP-RK3 step (Shu-Osher form of the three stages), pinned
# by the adjoint identity <lam, J v> = <J^T lam, v> with J v taken by central differences of
# dg.step itself.  Meshes carry hanging faces so the mortar terms enter the step.

def _step_vjp_gap(m, vjp_fn, seed, dt=0.01):
    q = _state(m, seed)
    rng = np.random.default_rng(seed + 1)
    lam = rng.standard_normal(q.shape)
    v = rng.standard_normal(q.shape)
    jt = vjp_fn(m, q, dt, lam)
    h = 1e-7
    fd = (dg.step(m, q + h * v, dt, 1) - dg.step(m, q - h * v, dt, 1)) / (2 * h)
    lhs, rhs = np.sum(lam * fd), np.sum(jt * v)
    return abs(lhs - rhs) / abs(lhs)


def _hanging_mesh(base, N, L, seed):
    f = fo.Forest(base, 1)
    rng = np.random.default_rng(seed)
    flags = rng.random(len(f)) < 0.4
    flags[0] = True
    f, _ = f.regrid(flags, 0)
    assert len(f.face_lists()[1]) > 0, "mesh must carry hanging faces"
    return dg.Mesh(f, N, L)


@pytest.mark.parametrize("base,N,L", [((2, 2), 2, (1000.0, 1000.0)), ((1, 1, 2), 1, (600.0, 600.0, 800.0))])
def test_step_vjp_inner_product_against_finite_differences(base, N, L):
    m = _hanging_mesh(base, N, L, seed=11)
    assert _step_vjp_gap(m, adjoint.step_vjp, seed=12) <= 1e-7


def _step_vjp_planted(mistake):
    """Copies of step_vjp with one plausible mistake each (planted here, on the CPU)."""
    def fn(mesh, q, dt, lam):
        out = np.zeros(q.size)
        for j in range(q.size):
            qc = q.astype(complex)
            qc.flat[j] += 1j * adjoint.H
            if mistake == "half_dt":
                y = dg.step(mesh, qc, 0.5 * dt, 1)
            else:
                y = dg.step(mesh, qc, dt, 1)
            if mistake == "transposed_pairing":   # lambda paired with the wrong variable plane
                out[j] = np.sum(np.roll(lam, 1, axis=0) * y.imag) / adjoint.H
            else:
                out[j] = np.sum(lam * y.imag) / adjoint.H
        if mistake == "element_order":             # columns assigned to the wrong element
            return np.roll(out.reshape(q.shape), 1, axis=1)
        return out.reshape(q.shape)
    return fn


@pytest.mark.parametrize("mistake", ["half_dt", "transposed_pairing", "element_order"])
def test_step_vjp_pin_rejects_planted_mistakes(mistake):
    m = _hanging_mesh((2, 2), 2, (1000.0, 1000.0), seed=11)
    assert _step_vjp_gap(m, _step_vjp_planted(mistake), seed=12) > 1e-3
