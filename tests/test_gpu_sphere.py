"""Cubed-sphere transfer on the GPU (Sec. 3.4, App. B) against the oracle (oracle/sphere.py), through
the C ABI: per-node isoparametric weights and spherical-excess areas, then a sequence of
refinements and coarsenings with the library's host forest, the fields transferred on the
device and by the oracle.  Tolerances: weights 1e-12 and areas 1e-11 relative (the angle sum of
a small spherical triangle loses digits to the subtraction of pi on either side); transferred
fields 1e-11 of max|q| per field after every one of six regrids (the coarsening's volume
weights 4 V_c / sum V carry the areas' 1e-11 and the fields are carried from regrid to regrid);
integrals conserved to 1e-13 and the total area kept at 4 pi r^2 to 1e-12 (the volume-loss
metric)."""
import math

import numpy as np
import pytest

from oracle import forest as fo, sphere

pytestmark = pytest.mark.gpu

R = 6.371e6


@pytest.fixture(scope="module")
def pkg():
    import torch
    assert torch.cuda.is_available()
    from paper_2404_16648_gb300 import build as b
    b.build()
    import paper_2404_16648_gb300 as p
    return p


def _fields(m):
    x = m.x / R
    q = np.empty((3, len(m.forest), m.np_))
    q[0] = 2.0 + np.sin(3 * x[..., 0]) * np.cos(2 * x[..., 1]) + x[..., 2]
    q[1] = 1.0 + 0.5 * np.exp(-4 * ((x[..., 0] - 0.6) ** 2 + x[..., 1] ** 2))
    q[2] = np.sin(2 * x[..., 2]) + 0.3
    return q


@pytest.mark.parametrize("n,N", [(2, 3), (3, 5), (1, 8)])
def test_sphere_geometry_and_transfer_against_the_oracle(pkg, n, N):
    import torch
    lf = pkg.Forest(2, (6 * n, n), 3)
    of = fo.Forest((6 * n, n), 3)
    om = sphere.SphereMesh(of, N, n, R)
    W, area = pkg.sphere_geometry(N, n, R, lf.leaves())
    np.testing.assert_allclose(W.cpu().numpy(), om.W, rtol=1e-12, atol=0)
    np.testing.assert_allclose(area.cpu().numpy(), om.area, rtol=1e-11, atol=0)
    q_o = _fields(om)
    q_g = torch.from_numpy(q_o).cuda()
    I0 = np.einsum("en,ven->v", om.W, q_o)
    rng = np.random.default_rng(10 * n + N)
    for k in range(6):
        p = 0.35 if k % 3 != 2 else 0.0
        flags = (rng.random(len(of)) < p).astype(np.uint8)
        tm = lf.regrid(flags, 0)
        of2, otm = of.regrid(flags.astype(bool), 0)
        assert np.array_equal(lf.leaves()[:, 1:4], np.array([[l, c[0], c[1]] for l, c in of2.leaves]))
        om2 = sphere.SphereMesh(of2, N, n, R)
        W2, area2 = pkg.sphere_geometry(N, n, R, lf.leaves())
        q_g = pkg.sphere_transfer(N, n, q_g, tm, W, area, W2)
        q_o = sphere.transfer(q_o, om, om2, otm)
        got = q_g.cpu().numpy()
        for v in range(3):
            assert np.abs(got[v] - q_o[v]).max() <= 1e-11 * np.abs(q_o[v]).max()
        Wn = W2.cpu().numpy()
        np.testing.assert_allclose(np.einsum("en,ven->v", Wn, got), I0, rtol=1e-13, atol=0)
        assert abs(area2.cpu().numpy().sum() - 4 * math.pi * R * R) <= 1e-12 * 4 * math.pi * R * R
        of, om, W, area = of2, om2, W2, area2
    assert max(l for l, _ in of.leaves) >= 1


def test_sphere_transfer_rejects_a_broken_map(pkg):
    import ctypes
    import torch
    lib = pkg.load_library()
    N, n = 3, 1
    lf = pkg.Forest(2, (6 * n, n), 2)
    W, area = pkg.sphere_geometry(N, n, R, lf.leaves())
    q = torch.zeros((1, len(lf), (N + 1) ** 2), dtype=torch.float64, device="cuda")
    tm = lf.regrid(np.ones(len(lf), np.uint8), 0)
    bad = tm.copy()
    bad[1, 2] = 3                      # a family whose children are out of order
    out = torch.empty((1, tm.shape[0], (N + 1) ** 2), dtype=torch.float64, device="cuda")
    st = lib.dg_sphere_transfer(N, n, 1, np.ascontiguousarray(bad).ctypes.data_as(ctypes.POINTER(ctypes.c_int32)),
                                tm.shape[0], ctypes.c_void_p(W.data_ptr()), ctypes.c_void_p(area.data_ptr()),
                                ctypes.c_void_p(q.data_ptr()), len(W), ctypes.c_void_p(W.data_ptr()),
                                ctypes.c_void_p(out.data_ptr()), None)
    assert st == 1
    bad = tm.copy()
    bad[0, 1] = 10 ** 6                # an old element out of range
    st = lib.dg_sphere_transfer(N, n, 1, np.ascontiguousarray(bad).ctypes.data_as(ctypes.POINTER(ctypes.c_int32)),
                                tm.shape[0], ctypes.c_void_p(W.data_ptr()), ctypes.c_void_p(area.data_ptr()),
                                ctypes.c_void_p(q.data_ptr()), len(W), ctypes.c_void_p(W.data_ptr()),
                                ctypes.c_void_p(out.data_ptr()), None)
    assert st == 1
