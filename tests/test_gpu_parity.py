"""GPU parity: the CUDA path (through the C ABI) against the FP64 oracle, element by element.

Tolerances: FP64 RHS within 1e-12 of max|rhs| per variable (the relative-per-RHS target);
FP64 steps, transfers and integrals within 1e-12 / 1e-13 relative; the FP32 perturbation path
within the bound stated in each test (FP32 rounding of the state and fluxes).
"""
import math

import numpy as np
import pytest

import workloads
from oracle import dg as odg, forest as ofo, physics

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def pkg():
    import torch
    assert torch.cuda.is_available()
    from paper_2404_16648_gb300 import build as b
    b.build()
    import paper_2404_16648_gb300 as p
    return p


def _pair(pkg, dim, N, base, length, max_level=2, flags_rounds=(), precision="fp64", B=1):
    """Library mesh and oracle mesh built independently with the same explicit flags."""
    lm = pkg.Mesh(dim, N, base, length, max_level=max_level, precision=precision)
    of = ofo.Forest(base, max_level)
    for p, seed in flags_rounds:
        flags = workloads.random_flags(len(of), p, seed)
        lm.adapt(flags=flags, buffer=B)
        of, _ = of.regrid(flags.astype(bool), B)
    om = odg.Mesh(of, N, length)
    lv = lm.leaves()
    assert lv.shape[0] == om.E
    np.testing.assert_array_equal(lv[:, 1], [l for l, _ in of.leaves])
    return lm, om


def _rel_err(got, want):
    errs = []
    for v in range(want.shape[0]):
        scale = np.abs(want[v]).max()
        errs.append(np.abs(got[v] - want[v]).max() / (scale if scale > 0 else 1.0))
    return max(errs)


def _gpu_rhs(lm, q):
    import torch
    qt = torch.from_numpy(q).cuda()
    out = lm.rhs(qt)
    torch.cuda.synchronize()
    return out.cpu().numpy()


MESHES = [
    (2, 4, (10, 10), (1000.0, 1000.0), ()),
    (2, 4, (4, 3), (1200.0, 900.0), ((0.3, 1), (0.3, 2))),
    (2, 7, (3, 3), (3000.0, 3000.0), ((0.3, 3),)),
    (3, 3, (2, 2, 2), (2000.0, 2000.0, 2000.0), ((0.3, 4), (0.2, 5))),
    (3, 7, (2, 2, 2), (2000.0, 2000.0, 2000.0), ((0.3, 6),)),
    (2, 1, (3, 2), (300.0, 200.0), ((0.5, 7),)),
    (3, 8, (1, 2, 1), (1000.0, 2000.0, 1000.0), ((0.5, 8),)),
    (3, 5, (2, 1, 2), (2000.0, 1000.0, 2000.0), ((0.4, 9),)),
    (3, 1, (2, 2, 3), (2000.0, 2000.0, 3000.0), ((0.3, 10), (0.3, 11))),
]


@pytest.mark.parametrize("layout", [0, 1, 2, 3, 4, 5])
@pytest.mark.parametrize("dim,N,base,length,rounds", MESHES)
def test_rhs_parity_fp64(pkg, dim, N, base, length, rounds, layout):
    lm, om = _pair(pkg, dim, N, base, length, flags_rounds=rounds)
    lm.set_stage_kernel(layout)
    q = workloads.random_state(om.nv, om.E, om.np_, seed=N + 10 * dim)
    got = _gpu_rhs(lm, q)
    want = odg.rhs(om, q)
    assert _rel_err(got, want) <= 1e-12


@pytest.mark.parametrize("precision", ["fp64", "fp32"])
def test_rest_state_exactly_zero(pkg, precision):
    lm, om = _pair(pkg, 3, 4, (2, 2, 2), (2000.0,) * 3, flags_rounds=((0.3, 9),), precision=precision)
    import torch
    q = torch.zeros(lm.state_shape, dtype=torch.float64 if precision == "fp64" else torch.float32,
                    device="cuda")
    out = lm.rhs(q)
    torch.cuda.synchronize()
    assert torch.count_nonzero(out).item() == 0


@pytest.mark.parametrize("layout", [0, 1, 2, 3, 4, 5])
@pytest.mark.parametrize("dim,N,base,length,rounds", MESHES)
def test_rhs_parity_fp32_perturbation(pkg, dim, N, base, length, rounds, layout):
    # FP32 state and flux arithmetic, FP64 background and pressure perturbation.  Bound: the
    # oracle evaluated on the FP32-rounded input, error <= 2e-5 of max|rhs| per variable.
    lm, om = _pair(pkg, dim, N, base, length, flags_rounds=rounds, precision="fp32")
    lm.set_stage_kernel(layout)
    q32 = workloads.random_state(om.nv, om.E, om.np_, seed=N + 10 * dim, dtype=np.float32)
    got = _gpu_rhs(lm, q32).astype(np.float64)
    want = odg.rhs(om, q32.astype(np.float64))
    assert _rel_err(got, want) <= 2e-5


def test_bubble_initial_state_and_indicator(pkg):
    cfg = workloads.RTB_2D
    lm, om = _pair(pkg, 2, cfg["N"], cfg["base"], cfg["length"], max_level=0)
    lm.set_bubble(**cfg["bubble"])
    got = lm.get_state()
    b = cfg["bubble"]
    want = odg.state_from_theta(om, odg.bubble_theta(om, b["center"], b["radius"], b["amp"]))
    np.testing.assert_allclose(got, want, rtol=0, atol=1e-15 * np.abs(want).max() + 1e-300)
    np.testing.assert_allclose(lm.indicator(), odg.indicator(om, want), rtol=0, atol=1e-12)


def test_step_parity_rising_bubble(pkg):
    cfg = workloads.RTB_2D
    lm, om = _pair(pkg, 2, cfg["N"], cfg["base"], cfg["length"], max_level=0)
    lm.set_bubble(**cfg["bubble"])
    q0 = lm.get_state()
    nsteps = 10
    lm.step(cfg["dt"], nsteps)
    got = lm.get_state()
    want = odg.step(om, q0, cfg["dt"], nsteps)
    # compare the tendency-carrying part: state change over the steps
    assert _rel_err(got - q0, want - q0) <= 1e-11


@pytest.mark.parametrize("layout", [0, 1, 2, 3, 4, 5])
def test_step_parity_hanging_3d(pkg, layout):
    lm, om = _pair(pkg, 3, 3, (2, 2, 2), (2000.0,) * 3, flags_rounds=((0.3, 11),))
    lm.set_stage_kernel(layout)
    q0 = workloads.random_state(om.nv, om.E, om.np_, seed=11, rho_scale=1e-4, u_scale=0.1,
                                theta_scale=0.01)
    lm.set_state(q0)
    lm.step(0.002, 3)
    got = lm.get_state()
    want = odg.step(om, q0, 0.002, 3)
    assert _rel_err(got - q0, want - q0) <= 1e-11


@pytest.mark.parametrize("dim,N,base", [(2, 4, (3, 3)), (3, 3, (2, 2, 2))])
def test_adapt_transfer_parity(pkg, dim, N, base):
    length = tuple(1000.0 for _ in base)
    lm, om = _pair(pkg, dim, N, base, length, flags_rounds=((0.4, 12),))
    q = workloads.random_state(om.nv, om.E, om.np_, seed=13)
    lm.set_state(q)
    flags = workloads.random_flags(om.E, 0.3, 14)
    flags[: om.E // 2] = 0
    rep = lm.adapt(flags=flags, buffer=0)
    of2, tmap = om.forest.regrid(flags.astype(bool), 0)
    om2 = odg.Mesh(of2, N, length)
    assert rep["after"] == om2.E
    np.testing.assert_array_equal(lm.leaves()[:, 1], [l for l, _ in of2.leaves])
    want = odg.transfer(q, om, om2, tmap)
    got = lm.get_state()
    np.testing.assert_allclose(got, want, rtol=0, atol=1e-13 * np.abs(q).max())


@pytest.mark.parametrize("precision", ["fp64", "fp32"])
def test_noop_adapt_keeps_mesh_and_state(pkg, precision):
    """A regrid pass that refines and coarsens nothing (level-0 roots, no flags) leaves the
    leaves and the state as they were, bit for bit, and the next steps equal those of a twin
    mesh that never adapted; the oracle's regrid agrees that nothing changes."""
    base, length = (3, 2, 2), (1500.0, 1000.0, 1000.0)
    a = pkg.Mesh(3, 3, base, length, max_level=2, precision=precision)
    b = pkg.Mesh(3, 3, base, length, max_level=2, precision=precision)
    for m in (a, b):
        m.set_bubble(center=(700.0, 500.0, 400.0), radius=(300.0,) * 3, amp=0.5)
    leaves0, q0 = a.leaves().copy(), a.get_state().copy()
    rep = a.adapt(flags=np.zeros(a.num_elements, np.uint8), buffer=1)
    of2, _ = ofo.Forest(base, 2).regrid(np.zeros(len(q0[0]), bool), 1)
    assert rep["before"] == rep["after"] == len(of2.leaves) == a.num_elements
    np.testing.assert_array_equal(a.leaves(), leaves0)
    assert np.array_equal(a.get_state(), q0)
    a.step(0.004, 3)
    b.step(0.004, 3)
    assert np.array_equal(a.get_state(), b.get_state())


def test_integrals_parity(pkg):
    lm, om = _pair(pkg, 3, 4, (2, 2, 3), (2000.0, 2000.0, 3000.0), flags_rounds=((0.3, 15),))
    q = workloads.random_state(om.nv, om.E, om.np_, seed=16)
    lm.set_state(q)
    got = lm.integrals()
    want = odg.integrals(om, q)
    np.testing.assert_allclose(got[[0, 1, 3]], want[[0, 1, 3]], rtol=1e-14)
    np.testing.assert_allclose(got[[2, 4]], want[[2, 4]], rtol=1e-12)


def test_mass_conserved_through_steps_and_adapts(pkg):
    # total mass conserved to 1e-13 relative over a run with regrids (FP64); finest h = 50 m,
    # so dt = 0.004 s keeps RK3 inside its stability limit
    lm = pkg.Mesh(2, 4, (5, 5), (1000.0, 1000.0), max_level=2)
    bub = dict(center=(500.0, 350.0), radius=(250.0, 250.0), amp=0.25)
    pkg.adapt_initial(lm, bub, threshold=0.05, buffer=1)
    m0 = lm.integrals()
    for _ in range(4):
        lm.step(0.004, 5)
        lm.adapt(threshold=0.05, buffer=1)
    m1 = lm.integrals()
    assert abs(m1[0] - m0[0]) <= 1e-13 * m0[0]
    assert abs(m1[4] - m0[4]) <= 1e-13 * m0[0]


def test_full_size_octree_sampled_parity(pkg):
    """The benchmark's 3D octree workload at full size (16^3 roots, N = 7, two levels), GPU
    RHS on every element against the oracle on a seeded sample of elements."""
    cfg = workloads.BUBBLE_3D
    b = cfg["bubble"]
    lm = pkg.Mesh(3, cfg["N"], cfg["base"], cfg["length"], max_level=cfg["max_level"])
    pkg.adapt_initial(lm, b, cfg["threshold"], cfg["buffer"])
    om = odg.adapt_initial(ofo.Forest(cfg["base"], cfg["max_level"]), cfg["N"], cfg["length"],
                           lambda m: odg.bubble_theta(m, b["center"], b["radius"], b["amp"]),
                           cfg["threshold"], cfg["buffer"])
    np.testing.assert_array_equal(lm.leaves()[:, 1:5][:, 0], [l for l, _ in om.forest.leaves])
    assert om.E > 8000 and len(om.forest.face_lists()[1]) > 0
    q = workloads.random_state(om.nv, om.E, om.np_, seed=21, rho_scale=1e-3, u_scale=1.0,
                               theta_scale=0.2)
    got = _gpu_rhs(lm, q)
    sample = workloads.sample_elements(om.E, 48, seed=22)
    _, mort, _ = om.forest.face_lists()
    coarse = sorted({m[0] for m in mort})[:8]
    sample = np.unique(np.concatenate([sample, coarse]))
    want = odg.rhs(om, q, elems=sample)
    assert _rel_err(got[:, sample], want[:, sample]) <= 1e-12


_FULL = {}


def _full_size_pair(pkg, precision):
    """The 3D octree workload at full size (16^3 roots, N = 7, two levels where |theta'| > 0.05 K):
    a library mesh in the given precision and the oracle mesh, built independently."""
    if precision not in _FULL:
        cfg = workloads.BUBBLE_3D
        b = cfg["bubble"]
        lm = pkg.Mesh(3, cfg["N"], cfg["base"], cfg["length"], max_level=cfg["max_level"],
                      precision=precision)
        pkg.adapt_initial(lm, b, cfg["threshold"], cfg["buffer"])
        if "oracle" not in _FULL:
            _FULL["oracle"] = odg.adapt_initial(
                ofo.Forest(cfg["base"], cfg["max_level"]), cfg["N"], cfg["length"],
                lambda m: odg.bubble_theta(m, b["center"], b["radius"], b["amp"]),
                cfg["threshold"], cfg["buffer"])
        om = _FULL["oracle"]
        np.testing.assert_array_equal(lm.leaves()[:, 1], [l for l, _ in om.forest.leaves])
        _FULL[precision] = lm
    return _FULL[precision], _FULL["oracle"]


def _full_size_sample(om, count, seed):
    """Seeded sample of elements plus coarse mortar elements, and elements from the far end of
    the leaf order (the last resident wave: no element ahead of them for the L2 lookahead)."""
    sample = workloads.sample_elements(om.E, count, seed=seed)
    _, mort, _ = om.forest.face_lists()
    coarse = sorted({m[0] for m in mort})[:8]
    return np.unique(np.concatenate([sample, coarse, [om.E - 1, om.E - 7 * 152 - 1]]))


def test_full_size_octree_sampled_parity_fp32(pkg):
    """The benchmarked FP32 path at full size: the default line layout (4) with its programmatic
    dependent launch after the mortar kernel and its L2 lookahead one resident wave ahead, GPU
    RHS of every element against the oracle on the FP32-rounded input at a seeded sample.
    Bound: 2e-5 of max|rhs| per variable, as for the small FP32 meshes."""
    lm, om = _full_size_pair(pkg, "fp32")
    assert om.E > 7 * 152 * 10 and len(om.forest.face_lists()[1]) > 0
    q32 = workloads.random_state(om.nv, om.E, om.np_, seed=23, rho_scale=1e-3, u_scale=1.0,
                                 theta_scale=0.2, dtype=np.float32)
    got = _gpu_rhs(lm, q32).astype(np.float64)
    sample = _full_size_sample(om, 48, seed=24)
    want = odg.rhs(om, q32.astype(np.float64), elems=sample)
    assert _rel_err(got[:, sample], want[:, sample]) <= 2e-5


@pytest.mark.parametrize("precision,tol", [("fp64", 1e-11), ("fp32", 4e-5)])
def test_full_size_octree_step_sampled(pkg, precision, tol):
    """One SSP-RK3 step of the full-size octree through dg_step (three fused stage launches,
    each after its mortar kernel) against the oracle's step restricted to a seeded sample
    (odg.step_on).  Compared on the state change per variable: FP64 1e-11 as for the small
    meshes; FP32 4e-5, twice the per-RHS bound (three FP32 tendencies combined, each within
    2e-5, plus the FP32 rounding of the stage states)."""
    lm, om = _full_size_pair(pkg, precision)
    dt = np.float64 if precision == "fp64" else np.float32
    q0 = workloads.random_state(om.nv, om.E, om.np_, seed=25, rho_scale=1e-4, u_scale=0.2,
                                theta_scale=0.02, dtype=dt)
    lm.set_state(q0)
    lm.step(workloads.BUBBLE_3D["dt"], 1)
    got = lm.get_state().astype(np.float64)
    sample = _full_size_sample(om, 12, seed=26)
    q64 = q0.astype(np.float64)
    want = odg.step_on(om, q64, workloads.BUBBLE_3D["dt"], sample)
    assert _rel_err(got[:, sample] - q64[:, sample], want[:, sample] - q64[:, sample]) <= tol


@pytest.mark.parametrize("precision,tol", [("fp64", 1e-12), ("fp32", 2e-5)])
def test_rhs_parity_large_theta_uses_fallback_branch(pkg, precision, tol):
    # |Theta'| ~ 20 makes |Theta'/Theta_bar| exceed 2^-5 at many nodes, so the pressure
    # perturbation takes the expm1/log1p branch there and the series elsewhere
    lm, om = _pair(pkg, 3, 3, (2, 2, 2), (2000.0,) * 3, flags_rounds=((0.3, 31),), precision=precision)
    dt = np.float64 if precision == "fp64" else np.float32
    q = workloads.random_state(om.nv, om.E, om.np_, seed=32, theta_scale=20.0, dtype=dt)
    rb, Tb, pb = om.bg
    assert np.mean(np.abs(q[-1] / Tb) > 2 ** -5) > 0.2
    got = _gpu_rhs(lm, q).astype(np.float64)
    want = odg.rhs(om, q.astype(np.float64))
    assert _rel_err(got, want) <= tol


@pytest.mark.parametrize("precision,tol", [("fp64", 1e-12), ("fp32", 2e-5)])
@pytest.mark.parametrize("dim,N,base", [(2, 3, (1, 1)), (3, 3, (1, 1, 1)), (3, 7, (1, 1, 1))])
@pytest.mark.parametrize("layout", [1, 2, 3, 4, 5])
def test_single_element_mesh(pkg, precision, tol, dim, N, base, layout):
    """One element with walls on every face: the smallest mesh the method has."""
    import torch
    lm = pkg.Mesh(dim, N, base, (800.0,) * dim, precision=precision)
    lm.set_stage_kernel(layout)
    om = odg.Mesh(ofo.Forest(base, 0), N, (800.0,) * dim)
    assert lm.num_elements == 1 and lm.num_mortars == 0
    q = workloads.random_state(om.nv, om.E, om.np_, seed=200 + N + dim)
    dt = torch.float64 if precision == "fp64" else torch.float32
    qt = torch.from_numpy(q).to(dt)
    got = lm.rhs(qt.cuda()).double().cpu().numpy()
    want = odg.rhs(om, qt.double().numpy())
    assert _rel_err(got, want) <= tol


@pytest.mark.parametrize("dim,N", [(2, 3), (3, 2)])
def test_deep_refinement_chain(pkg, dim, N):
    """Refining the corner element six times (a 2:1 ripple towards the coarse roots): levels
    0 .. 6 on one mesh, every level's 2/h from the per-level tables."""
    base = (2,) * dim
    lm = pkg.Mesh(dim, N, base, (16000.0,) * dim, max_level=6)
    of = ofo.Forest(base, 6)
    for _ in range(6):
        flags = np.zeros(len(of), np.uint8)
        flags[0] = 1                       # the leaf at the origin corner, Morton-first
        lm.adapt(flags=flags, buffer=0)
        of, _ = of.regrid(flags.astype(bool), 0)
    om = odg.Mesh(of, N, (16000.0,) * dim)
    levels = [l for l, _ in of.leaves]
    assert max(levels) == 6 and min(levels) <= 1 and lm.num_elements == om.E
    assert of.is_balanced()
    q = workloads.random_state(om.nv, om.E, om.np_, seed=300 + dim)
    assert _rel_err(_gpu_rhs(lm, q), odg.rhs(om, q)) <= 1e-12


def test_box_above_the_neutral_atmosphere_is_rejected(pkg):
    """The neutral background ends where the Exner function reaches zero, z = cp theta0 / g
    (30.7 km for the default constants); a taller box has no background and is refused."""
    from paper_2404_16648_gb300.dg import DGError
    with pytest.raises(DGError):
        pkg.Mesh(2, 3, (2, 2), (10000.0, 31000.0))
    pkg.Mesh(2, 3, (2, 2), (10000.0, 30000.0)).close()


def test_mesh_beyond_32_bit_state_offsets_is_rejected(pkg):
    """The kernels index a state buffer (NV + 1 planes of E (N+1)^d values) with 32-bit offsets:
    a mesh whose buffer would reach 2^31 values is refused before anything is allocated (80^3
    roots at N = 8: 6 x 512,000 x 729 > 2^31), and a mesh of the same degree well inside the
    limit is accepted."""
    from paper_2404_16648_gb300.dg import DGError
    with pytest.raises(DGError) as ex:
        pkg.Mesh(3, 8, (80, 80, 80), (8000.0, 8000.0, 8000.0), precision="fp32")
    assert ex.value.status == 6
    pkg.Mesh(3, 8, (8, 8, 8), (8000.0, 8000.0, 8000.0), precision="fp32").close()
