"""The allocation-free integrals entry point against dg_integrals, through the C ABI.

dg_integrals_noalloc serves callers that cannot allocate device memory (stream capture,
externally owned device memory, real-time loops); it keeps its reduction scratch in a static
device array.  This file is collected last so that a failure here comes after every other test
has run; it must also pass when run alone in a fresh process.
"""
import ctypes

import numpy as np
import pytest

import workloads

@pytest.fixture(scope="module")
def pkg():
    import torch
    assert torch.cuda.is_available()
    from paper_2404_16648_gb300 import build as b
    b.build()
    import paper_2404_16648_gb300 as p
    return p


@pytest.mark.gpu
@pytest.mark.parametrize("precision", ["fp64", "fp32"])
def test_noalloc_integrals_match_dg_integrals_twice(pkg, precision):
    import torch
    lib = pkg.load_library()
    m = pkg.Mesh(3, 4, (2, 2, 3), (2000.0, 2000.0, 3000.0), max_level=1, precision=precision)
    m.adapt(flags=workloads.random_flags(m.num_elements, 0.4, seed=41), buffer=0)
    elem = torch.from_numpy(np.ascontiguousarray(m.leaves()[:, 1:5])).cuda()
    out = torch.full((6,), -1.0, dtype=torch.float64, device="cuda")
    for call in range(2):
        dtype = np.float64 if precision == "fp64" else np.float32
        q = workloads.random_state(m.nv, m.num_elements, m.np_, seed=42 + call, dtype=dtype)
        m.set_state(q)
        want = m.integrals()
        qd = torch.from_numpy(q).cuda()
        st = lib.dg_integrals_noalloc(ctypes.byref(m.desc), ctypes.c_void_p(elem.data_ptr()),
                                      m.num_elements, ctypes.c_void_p(qd.data_ptr()),
                                      ctypes.c_void_p(out.data_ptr()), None)
        assert st == 0
        torch.cuda.synchronize()
        got = out.cpu().numpy()
        assert got[5] == 0.0
        np.testing.assert_allclose(got[[0, 1, 3]], want[[0, 1, 3]], rtol=1e-13)
        np.testing.assert_allclose(got[[2, 4]], want[[2, 4]], rtol=1e-11)


@pytest.mark.gpu
def test_noalloc_rejects_sizes_beyond_the_scratch(pkg):
    lib = pkg.load_library()
    m = pkg.Mesh(3, 8, (1, 1, 1), (1000.0, 1000.0, 1000.0))
    # 729 nodes per element: 100,000 elements exceed the 67,108,864-node limit
    st = lib.dg_integrals_noalloc(ctypes.byref(m.desc), ctypes.c_void_p(16), 100000,
                                  ctypes.c_void_p(16), ctypes.c_void_p(16), None)
    assert st == 1


# The argument checks below return before any device call, so they run without a GPU.

@pytest.fixture(scope="module")
def hostlib():
    from paper_2404_16648_gb300 import build as b
    b.build()
    import paper_2404_16648_gb300 as p
    return p


def test_noalloc_rejects_an_element_count_whose_node_count_wraps(hostlib):
    lib = hostlib.load_library()
    d = hostlib.make_desc(3, 7, (1, 1, 1), (1000.0, 1000.0, 1000.0))
    # 512 nodes per element: 2^55 elements give 2^64 nodes, which wraps to 0 in int64
    st = lib.dg_integrals_noalloc(ctypes.byref(d), ctypes.c_void_p(16), 1 << 55,
                                  ctypes.c_void_p(16), ctypes.c_void_p(16), None)
    assert st == 1


def test_noalloc_rejects_a_box_above_the_neutral_atmosphere(hostlib):
    lib = hostlib.load_library()
    # cp theta0 / g = 1004.5 * 300 / 9.81 = 30,718 m: a 40 km column has no background at its top
    d = hostlib.make_desc(2, 3, (2, 2), (1000.0, 40000.0))
    st = lib.dg_integrals_noalloc(ctypes.byref(d), ctypes.c_void_p(16), 4,
                                  ctypes.c_void_p(16), ctypes.c_void_p(16), None)
    assert st == 1
