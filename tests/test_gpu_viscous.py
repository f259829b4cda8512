"""GPU BR1 viscous term against the oracle, and the 2D cold-bubble AMR workload with viscosity."""
import numpy as np
import pytest

import workloads
from oracle import dg as odg, forest as ofo

pytestmark = pytest.mark.gpu
NU = 75.0


@pytest.fixture(scope="module")
def pkg():
    import torch
    assert torch.cuda.is_available()
    from paper_2404_16648_gb300 import build as b
    b.build()
    import paper_2404_16648_gb300 as p
    return p


def _pair(pkg, dim, N, base, length, seed, nu=NU):
    lm = pkg.Mesh(dim, N, base, length, max_level=1, nu=nu)
    of = ofo.Forest(base, 1)
    flags = workloads.random_flags(len(of), 0.35, seed)
    flags[0] = 1
    lm.adapt(flags=flags, buffer=0)
    of, _ = of.regrid(flags.astype(bool), 0)
    return lm, odg.Mesh(of, N, length)


def _rel(got, want):
    return max(np.abs(got[v] - want[v]).max() / max(np.abs(want[v]).max(), 1e-300)
               for v in range(want.shape[0]))


@pytest.mark.parametrize("dim,N,base,length", [(2, 3, (3, 3), (900.0, 900.0)),
                                               (2, 5, (4, 2), (1600.0, 800.0)),
                                               (3, 2, (2, 2, 2), (1000.0,) * 3)])
def test_viscous_rhs_parity(pkg, dim, N, base, length):
    import torch
    lm, om = _pair(pkg, dim, N, base, length, seed=20 + N)
    q = workloads.random_state(om.nv, om.E, om.np_, seed=21 + N)
    got = lm.rhs(torch.from_numpy(q).cuda()).cpu().numpy()
    want = odg.rhs(om, q) + odg.viscous_rhs(om, q, NU)
    assert _rel(got, want) <= 1e-12


def test_viscous_step_parity(pkg):
    lm, om = _pair(pkg, 2, 4, (3, 3), (900.0, 900.0), seed=30)
    q = workloads.random_state(om.nv, om.E, om.np_, seed=31, rho_scale=1e-4, u_scale=0.5, theta_scale=0.05)
    lm.set_state(q)
    lm.step(0.002, 3)
    got = lm.get_state()
    want = odg.step(om, q, 0.002, 3, nu=NU)
    assert _rel(got - q, want - q) <= 1e-11


def test_viscous_is_fp64_only(pkg):
    from paper_2404_16648_gb300.dg import DGError
    with pytest.raises(DGError):
        pkg.Mesh(2, 3, (2, 2), (1000.0, 1000.0), precision="fp32", nu=NU)


def test_cold_bubble_amr_with_viscosity_conserves_mass(pkg):
    """The 2D cold-bubble workload (32 x 8 roots on 25.6 x 6.4 km, N = 5, up to 3 levels,
    nu = 75, regrid every 10 steps where |theta'| > 0.1 K): 60 steps conserve mass to 1e-13."""
    cfg = workloads.COLD_2D
    m = pkg.Mesh(2, cfg["N"], cfg["base"], cfg["length"], max_level=cfg["max_level"], nu=NU)
    pkg.adapt_initial(m, cfg["bubble"], cfg["threshold"], cfg["buffer"])
    assert m.num_mortars > 0
    m0 = m.integrals()
    for _ in range(6):
        m.step(cfg["dt"], cfg["regrid_every"])
        m.adapt(threshold=cfg["threshold"], buffer=cfg["buffer"])
    m1 = m.integrals()
    assert np.all(np.isfinite(m.get_state()))
    assert abs(m1[0] - m0[0]) <= 1e-13 * m0[0]
    assert abs(m1[4] - m0[4]) <= 1e-13 * m0[0]
