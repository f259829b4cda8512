"""Refinement indicator of Sec. 4.3: per element the largest |theta'| over its nodes.  The kernel
takes the FP64 division only at the nodes an FP32 estimate cannot rule out; its result must be
the value of the FP64 division at every node bit for bit.  That reference is the library's
per-node theta' (dg_primitives, the same FP64 expression, one node per thread), reduced here
with numpy.  Cases: random and bubble states on refined 2D/3D meshes for FP32 and FP64
storage, perturbations below FP32 resolution (every node a candidate), and elements that take
the division at every node (NaN, negative density), whose maximum ignores NaN."""
import numpy as np
import pytest

import workloads

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def pkg():
    import torch
    assert torch.cuda.is_available()
    from paper_2404_16648_gb300 import build as b
    b.build()
    import paper_2404_16648_gb300 as p
    return p


def _mesh(pkg, dim, N, precision, rounds=2, theta0=300.0):
    base = (6, 4) if dim == 2 else (3, 3, 2)
    length = (6000.0, 4000.0) if dim == 2 else (3000.0, 3000.0, 2000.0)
    lm = pkg.Mesh(dim, N, base, length, max_level=2, precision=precision, theta0=theta0)
    for r in range(rounds):
        lm.adapt(flags=workloads.random_flags(lm.num_elements, 0.3, seed=17 * r + N + dim), buffer=1)
    return lm


def _per_node_max(lm):
    th = lm.primitives()[lm.dim].cpu().numpy()          # theta' at every node, FP64 division
    return np.fmax.reduce(np.abs(th), axis=1, initial=0.0)


def _set(lm, q):
    lm.set_state(q.astype(lm.np_dtype))


@pytest.mark.parametrize("dim,N,precision,theta0", [(2, 4, "fp64", 300.0), (2, 7, "fp32", 300.0),
                                                    (2, 8, "fp64", 287.3), (3, 1, "fp32", 300.0),
                                                    (3, 3, "fp64", 300.0), (3, 7, "fp32", 300.0),
                                                    (3, 8, "fp32", 301.7)])
def test_indicator_equals_division_at_every_node(pkg, dim, N, precision, theta0):
    # theta0 = 287.3 and 301.7 have no exact FP32 form
    lm = _mesh(pkg, dim, N, precision, theta0=theta0)
    E, NP = lm.num_elements, (N + 1) ** dim
    for seed, kw in ((1, {}), (2, dict(theta_scale=3.0)),
                     (3, dict(rho_scale=1e-12, theta_scale=1e-9))):   # below FP32 resolution
        _set(lm, workloads.random_state(dim + 2, E, NP, seed=seed, **kw))
        np.testing.assert_array_equal(lm.indicator(), _per_node_max(lm))
    lm.set_bubble(center=(3000.0, 1500.0, 1000.0)[:dim], radius=(1500.0,) * dim, amp=2.0)
    np.testing.assert_array_equal(lm.indicator(), _per_node_max(lm))
    _set(lm, np.zeros(lm.state_shape))                  # the background alone
    np.testing.assert_array_equal(lm.indicator(), _per_node_max(lm))


@pytest.mark.parametrize("precision", ["fp32", "fp64"])
def test_indicator_elements_outside_the_fast_range(pkg, precision):
    lm = _mesh(pkg, 3, 5, precision)
    E, NP = lm.num_elements, 216
    q = workloads.random_state(5, E, NP, seed=9)
    q[4, 3, 17] = np.nan                                 # NaN Theta' at one node
    q[0, 5, :] = np.nan                                  # NaN density everywhere: result 0
    q[0, 7, 40] = -50.0                                  # negative density at one node
    q[4, 9, 2] = 1e35                                    # quotient far above the FP32 range
    _set(lm, q)
    got = lm.indicator()
    want = _per_node_max(lm)
    np.testing.assert_array_equal(got, want)
    assert got[5] == 0.0 and np.isfinite(got[3]) and got[9] > 1e30
    assert np.all(np.isfinite(np.delete(got, [9])))


def _twins(pkg, dim, N, precision, theta0):
    base = (6, 4) if dim == 2 else (3, 3, 2)
    length = (6000.0, 4000.0) if dim == 2 else (3000.0, 3000.0, 2000.0)
    return [pkg.Mesh(dim, N, base, length, max_level=1, precision=precision, theta0=theta0) for _ in range(2)]


@pytest.mark.parametrize("dim,N,precision,theta0", [(2, 4, "fp64", 300.0), (2, 7, "fp32", 301.7),
                                                    (3, 3, "fp64", 287.3), (3, 7, "fp32", 300.0)])
def test_adapt_threshold_tags_equal_indicator_comparison(pkg, dim, N, precision, theta0):
    """dg_adapt's theta' criterion decides `indicator > threshold` on the device without forming
    the indicator where FP32 intervals settle it.  Against the same comparison made on the
    host from dg_indicator: roots at level 0 with one level to go and no buffer, so every tag
    shows in the leaves.  Thresholds: a typical one, every tenth element's indicator value
    itself (that element is not tagged) and the next double below it (it is), on random,
    bubble, below-FP32-resolution and NaN / negative-density states."""
    a, b = _twins(pkg, dim, N, precision, theta0)
    E, NP = a.num_elements, (N + 1) ** dim
    states = [workloads.random_state(dim + 2, E, NP, seed=41, theta_scale=0.05),
              workloads.random_state(dim + 2, E, NP, seed=42, rho_scale=1e-12, theta_scale=1e-9)]
    # elements outside the intervals' range: a NaN node (left out, as the indicator leaves it
    # out) and a negative density (every node of that element takes the division)
    odd = workloads.random_state(dim + 2, E, NP, seed=43, theta_scale=0.05)
    odd[dim + 1, 3, 0] = np.nan
    odd[0, 5, :] = -3.0
    states.append(odd)
    for q in states + [None]:
        for m in (a, b):
            if q is None:
                m.set_bubble(center=(3000.0, 1500.0, 1000.0)[:dim], radius=(1500.0,) * dim, amp=0.05)
            else:
                _set(m, q)
        ind = a.indicator()
        edges = sorted(set(range(0, E, 10)) | {3, 5})
        thrs = [0.05] + [float(ind[e]) for e in edges] + [float(np.nextafter(ind[e], -np.inf)) for e in edges]
        for thr in thrs:
            want = (ind > thr).astype(np.uint8)
            ra = a.adapt(threshold=thr, buffer=0)
            rb = b.adapt(flags=want, buffer=0)
            assert ra == rb
            np.testing.assert_array_equal(a.leaves(), b.leaves())
            # back to the roots for the next threshold
            for m in (a, b):
                m.adapt(flags=np.zeros(m.num_elements, np.uint8), buffer=0)
            assert a.num_elements == E
            if q is None:
                for m in (a, b):
                    m.set_bubble(center=(3000.0, 1500.0, 1000.0)[:dim], radius=(1500.0,) * dim, amp=0.05)
            else:
                for m in (a, b):
                    _set(m, q)
