"""The regrid's error path, through the C ABI, with failures made on the host
(DG_OPT_FAIL_NEXT_ADAPT; no device fault is involved).

- A failure before the new tree is committed leaves the mesh as it was: same elements, same
  state, and it steps and regrids afterwards exactly like an untouched copy.
- A failure after the commit leaves device tables of mixed sizes; every later call on the mesh
  is refused with DG_ERR_STATE instead of launching kernels on them.
"""
import ctypes

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


def _mesh(pkg):
    m = pkg.Mesh(2, 3, (3, 3), (900.0, 900.0), max_level=2)
    q = workloads.random_state(m.nv, m.num_elements, m.np_, seed=71, rho_scale=1e-4, u_scale=0.5,
                               theta_scale=0.05)
    m.set_state(q)
    return m, q


def test_failure_before_commit_leaves_the_mesh_usable(pkg):
    m, q = _mesh(pkg)
    ref, _ = _mesh(pkg)
    flags = workloads.random_flags(m.num_elements, 0.5, seed=72)
    m.fail_next_adapt(1)
    with pytest.raises(pkg.DGError) as ex:
        m.adapt(flags=flags, buffer=0)
    assert ex.value.status == 4
    assert m.num_elements == 9
    np.testing.assert_array_equal(m.get_state(), q)
    for mm in (m, ref):
        mm.adapt(flags=flags, buffer=0)
        mm.step(0.01, 3)
    assert m.num_elements == ref.num_elements > 9
    np.testing.assert_array_equal(m.get_state(), ref.get_state())
    np.testing.assert_array_equal(m.integrals(), ref.integrals())


def test_failure_after_commit_refuses_every_later_call(pkg):
    import torch
    m, q = _mesh(pkg)
    flags = workloads.random_flags(m.num_elements, 0.5, seed=73)
    m.fail_next_adapt(2)
    with pytest.raises(pkg.DGError) as ex:
        m.adapt(flags=flags, buffer=0)
    assert ex.value.status == 3
    lib = m.lib
    calls = [
        lambda: m.step(0.01, 1),
        lambda: m.get_state(),
        lambda: m.set_state(q),
        lambda: m.integrals(),
        lambda: m.rhs(torch.zeros(m.nv * 9 * m.np_, dtype=torch.float64, device="cuda")),
        lambda: m.adapt(flags=np.zeros(m.num_elements, np.uint8), buffer=0),
        lambda: m.indicator(),
        lambda: m.leaves(),
    ]
    for c in calls:
        with pytest.raises(pkg.DGError) as ex:
            c()
        assert ex.value.status == 4
    assert b"unusable" in lib.dg_last_error(m.h)
    h = ctypes.c_void_p()
    arr = (ctypes.c_void_p * 1)(m.h.value)
    assert lib.dg_batch_create(arr, 1, ctypes.byref(h)) == 4
    m.close()   # destroying an unusable mesh is allowed
