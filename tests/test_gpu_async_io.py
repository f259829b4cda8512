"""The asynchronous state copies and integrals (dg_set_state_async, dg_get_state_async,
dg_integrals_async) give the bits of the synchronous calls: a step after an asynchronous copy
in equals a step after dg_set_state, the copy out on a second stream equals dg_get_state, and
the device-side combination of the integrals equals the host's, including the non-finite flag."""
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


@pytest.mark.parametrize("precision", ["fp64", "fp32"])
def test_async_io_equals_sync(pkg, precision):
    import torch
    a = pkg.Mesh(3, 3, (2, 2, 2), (2000.0,) * 3, max_level=1, precision=precision)
    b = pkg.Mesh(3, 3, (2, 2, 2), (2000.0,) * 3, max_level=1, precision=precision)
    f = workloads.random_flags(a.num_elements, 0.4, seed=81)
    for m in (a, b):
        m.adapt(flags=f, buffer=0)
    dtype = np.float64 if precision == "fp64" else np.float32
    q = workloads.random_state(a.nv, a.num_elements, a.np_, seed=82, rho_scale=1e-4, u_scale=0.2,
                               theta_scale=0.02, dtype=dtype)
    host = torch.from_numpy(q).pin_memory()
    out = torch.empty_like(host).pin_memory()
    integ = torch.full((6,), -1.0, dtype=torch.float64).pin_memory()
    side = torch.cuda.Stream()
    for step in range(2):
        a.set_state(q)
        a.step(0.002, 1)
        want_q = a.get_state()
        want_i = a.integrals()
        b.set_state_async(host)
        b.step(0.002, 1)
        b.get_state_async(out, stream=side)
        b.integrals_async(integ)
        torch.cuda.synchronize()
        assert np.array_equal(out.numpy(), want_q)
        assert np.array_equal(integ.numpy()[:5], want_i) and integ[5].item() == 0.0
        q = want_q.copy()
        host.copy_(torch.from_numpy(q))
    bad = q.copy()
    bad[0, 0, 0] = np.nan
    b.set_state(bad)
    b.integrals_async(integ)
    torch.cuda.synchronize()
    assert integ[5].item() == 1.0


@pytest.mark.parametrize("precision", ["fp64", "fp32"])
def test_state_layout_flags(pkg, precision):
    """dg_set_state / dg_get_state with DG_LAYOUT_ELEMENTS take and give q[e][v][n]: in from host
    and device arrays it equals the planes layout of the transposed array, out it is the
    transpose of the planes, bit for bit; an unknown flag is an argument error."""
    import ctypes
    import torch
    m = pkg.Mesh(3, 3, (2, 2, 1), (1000.0, 1000.0, 1000.0), max_level=1, precision=precision)
    m.adapt(flags=workloads.random_flags(m.num_elements, 0.5, seed=91), buffer=0)
    dtype = np.float64 if precision == "fp64" else np.float32
    q = workloads.random_state(m.nv, m.num_elements, m.np_, seed=92, dtype=dtype)
    qe = np.ascontiguousarray(q.transpose(1, 0, 2))
    m.set_state(qe, layout="elements")                           # host, element-major
    assert np.array_equal(m.get_state(), q)
    assert np.array_equal(m.get_state(layout="elements"), qe)
    m.set_state(np.zeros_like(q))
    m.set_state(torch.from_numpy(qe).cuda(), layout="elements")  # device, element-major
    assert np.array_equal(m.get_state(), q)
    out = torch.empty(qe.shape, dtype=torch.float64 if precision == "fp64" else torch.float32, device="cuda")
    m.get_state(out, layout="elements")
    assert np.array_equal(out.cpu().numpy(), qe)
    lib = m.lib
    assert lib.dg_set_state(m.h, ctypes.c_void_p(qe.ctypes.data), 2, 0) == 1
    assert lib.dg_get_state(m.h, ctypes.c_void_p(qe.ctypes.data), -1, 0) == 1
