"""GPU tracer advection (linear-advection test of Sec. 4.2) against the oracle: right-hand side
and steps with mortar and point-interpolation hanging faces, the initial bell, conservation with
mortars and its loss with interpolation, and the swirling-flow workload with 80 regrids."""
import numpy as np
import pytest

import workloads
from oracle import dg as odg, forest as ofo, tracer as otr

pytestmark = pytest.mark.gpu
T = 5.0


@pytest.fixture(scope="module")
def pkg():
    import torch
    assert torch.cuda.is_available()
    from paper_2404_16648_gb300 import build as b
    b.build()
    import paper_2404_16648_gb300 as p
    return p


def _pair(pkg, N, base, mode, p=0.4, seed=0):
    lm = pkg.Mesh(2, N, base, (1.0, 1.0), max_level=1, equations="tracer", face_mode=mode,
                  wind_period=T)
    of = ofo.Forest(base, 1)
    flags = workloads.random_flags(len(of), p, seed)
    flags[0] = 1
    lm.adapt(flags=flags, buffer=0)
    of, _ = of.regrid(flags.astype(bool), 0)
    om = odg.Mesh(of, N, (1.0, 1.0))
    assert lm.num_elements == om.E and len(of.face_lists()[1]) > 0
    return lm, om


@pytest.mark.parametrize("mode", ["mortar", "interp"])
@pytest.mark.parametrize("N,base", [(2, (3, 3)), (3, (4, 3)), (4, (3, 2)), (5, (2, 3))])
def test_tracer_rhs_matches_oracle(pkg, mode, N, base):
    import torch
    lm, om = _pair(pkg, N, base, mode, seed=N)
    C = workloads.random_scalar(om.E, om.np_, seed=30 + N)
    for t in (0.0, 1.7, 3.9):
        lm.set_time(t)
        got = lm.rhs(torch.from_numpy(C[None]).cuda()).cpu().numpy()[0]
        want = otr.rhs(om, C, t, T, mode)
        assert np.abs(got - want).max() <= 1e-12 * np.abs(want).max()


@pytest.mark.parametrize("mode", ["mortar", "interp"])
def test_tracer_steps_match_oracle(pkg, mode):
    import torch
    lm, om = _pair(pkg, 4, (3, 3), mode, seed=7)
    C0 = otr.bell(om, (0.25, 0.25), 0.25, 0.5) + 0.1 * workloads.random_scalar(om.E, om.np_, seed=8)
    lm.set_state(torch.from_numpy(C0[None]).cuda())
    lm.set_time(0.2)
    dt = 0.004
    lm.step(dt, 5)
    C = C0
    for i in range(5):
        C = otr.ssprk3_step(om, C, 0.2 + i * dt, dt, T, mode)
    got = lm.get_state()[0]
    assert np.abs((got - C0) - (C - C0)).max() <= 1e-11 * np.abs(C - C0).max()
    assert abs(lm.get_time() - (0.2 + 5 * dt)) <= 1e-15


def test_tracer_bell_and_total(pkg):
    lm, om = _pair(pkg, 4, (4, 4), "mortar", seed=9)
    lm.set_bubble(center=(0.25, 0.25), radius=(0.25, 0.25), amp=0.5)
    C = otr.bell(om, (0.25, 0.25), 0.25, 0.5)
    np.testing.assert_allclose(lm.get_state()[0], C, rtol=0, atol=1e-14)
    I = lm.integrals()
    assert abs(I[0] - otr.total(om, C)) <= 1e-14 * otr.total(om, C)
    assert abs(I[3] - 1.0) <= 1e-14 and I[4] == I[0]
    np.testing.assert_allclose(lm.indicator(), otr.indicator(om, C), rtol=0, atol=1e-15)


@pytest.mark.parametrize("mode", ["mortar", "interp"])
def test_tracer_conservation_through_steps_and_regrids(pkg, mode):
    """Mortars keep the tracer total to round-off through steps and regrids; point-to-point
    interpolation on the hanging faces does not (the comparison of Sec. 4.2)."""
    cfg = workloads.LEVEQUE_2D
    lm = pkg.Mesh(2, cfg["N"], cfg["base"], cfg["length"], max_level=1, equations="tracer",
                  face_mode=mode, wind_period=cfg["period"])
    pkg.adapt_initial(lm, cfg["bubble"], cfg["threshold"], cfg["buffer"])
    m0 = lm.integrals()[0]
    for _ in range(8):
        lm.step(cfg["dt"], cfg["regrid_every"])
        lm.adapt(threshold=cfg["threshold"], buffer=cfg["buffer"])
    assert lm.num_mortars > 0
    drift = abs(lm.integrals()[0] - m0) / m0
    if mode == "mortar":
        assert drift <= 1e-13
    else:
        assert drift >= 1e-9


def test_tracer_rejects_unsupported(pkg):
    from paper_2404_16648_gb300.dg import DGError
    with pytest.raises(DGError):
        pkg.Mesh(3, 3, (2, 2, 2), (1.0, 1.0, 1.0), equations="tracer", wind_period=T)
    with pytest.raises(DGError):
        pkg.Mesh(2, 3, (2, 2), (1.0, 1.0), equations="tracer", wind_period=T, precision="fp32")
    with pytest.raises(DGError):
        pkg.Mesh(2, 3, (2, 2), (1.0, 1.0), equations="tracer", wind_period=0.0)
    with pytest.raises(DGError):
        pkg.Mesh(2, 3, (2, 2), (1.0, 1.0), face_mode="interp")       # Euler meshes use mortars
    m = pkg.Mesh(2, 3, (2, 2), (1.0, 1.0), equations="tracer", wind_period=T)
    with pytest.raises(DGError):
        m.primitives()


def _leveque_error(pkg, mode, max_level):
    """Run the swirling flow for one period; tracer drift and relative L2 distance from the
    initial bell, both on the final mesh (integrals of C, (C - C0)^2 and C0^2 by the library)."""
    import torch
    cfg = workloads.LEVEQUE_2D
    lm = pkg.Mesh(2, cfg["N"], cfg["base"], cfg["length"], max_level=max_level, equations="tracer",
                  face_mode=mode, wind_period=cfg["period"])
    if max_level:
        pkg.adapt_initial(lm, cfg["bubble"], cfg["threshold"], cfg["buffer"])
    else:
        lm.set_bubble(**cfg["bubble"])
    m0 = lm.integrals()[0]
    regrids = 0
    for done in range(cfg["regrid_every"], cfg["steps"] + 1, cfg["regrid_every"]):
        lm.step(cfg["dt"], cfg["regrid_every"])
        if max_level:
            lm.adapt(threshold=cfg["threshold"], buffer=cfg["buffer"])
            regrids += 1
    torch.cuda.synchronize()
    drift = abs(lm.integrals()[0] - m0) / m0
    C = lm.get_state()
    lm.set_bubble(**cfg["bubble"])
    C0 = lm.get_state()
    lm.set_state((C - C0) ** 2)
    e2 = lm.integrals()[0]
    lm.set_state(C0 ** 2)
    n2 = lm.integrals()[0]
    return drift, float(np.sqrt(e2 / n2)), regrids, lm.num_elements


def test_swirling_flow_workload(pkg):
    """16 x 16 roots, N = 4, one level where |C| > 0.05, buffer 2, T = 5 in 2000 steps with 80
    regrids.  Mortars conserve the tracer to round-off while interpolation loses it; after the
    period the AMR bell is closer to the initial one than on the uniform 16 x 16 grid."""
    d_m, e_m, regrids, E = _leveque_error(pkg, "mortar", 1)
    d_i, e_i, _, _ = _leveque_error(pkg, "interp", 1)
    d_u, e_u, _, _ = _leveque_error(pkg, "mortar", 0)
    print("mortar drift %.2e err %.4f | interp drift %.2e err %.4f | uniform 16x16 drift %.2e err %.4f "
          "| %d regrids, %d elements at T" % (d_m, e_m, d_i, e_i, d_u, e_u, regrids, E))
    assert regrids == 80
    # 2000 steps leave about 8e-14 of round-off on the uniform grid as well
    assert d_m <= 2e-13 and d_u <= 2e-13
    assert d_i >= 100 * max(d_m, 1e-16)
    assert e_m < e_u
