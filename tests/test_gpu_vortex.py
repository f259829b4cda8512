"""GPU isentropic vortex (Sec. 4.1) on periodic meshes: the device initial condition and the
right-hand side against the oracle, and the 32 x 32, N = 3 AMR run against the exact solution
with the error norm and value the paper prints (tests/golden/paper_values.json)."""
import json
import os

import numpy as np
import pytest

import workloads
from oracle import dg as odg, forest as ofo, vortex as ovx

pytestmark = pytest.mark.gpu
HERE = os.path.dirname(os.path.abspath(__file__))
K = ovx.constants()
L = (12.0, 12.0)
CENTER, BETA, UINF = (6.0, 6.0), 5.0, (1.0, 1.0)


@pytest.fixture(scope="module")
def pkg():
    import torch
    assert torch.cuda.is_available()
    from paper_2404_16648_gb300 import build as b
    b.build()
    import paper_2404_16648_gb300 as p
    return p


def _lib_mesh(pkg, N, base, max_level=1, precision="fp64"):
    return pkg.Mesh(2, N, base, L, max_level=max_level, precision=precision, theta0=1.0, p0=1.0,
                    g=0.0, R=1.0, cp=3.5, periodic=(True, True))


def _pair(pkg, N, base, precision="fp64", p=0.4, seed=0):
    lm = _lib_mesh(pkg, N, base, precision=precision)
    of = ofo.Forest(base, 1, periodic=(True, True))
    flags = workloads.random_flags(len(of), p, seed)
    flags[0] = 1
    lm.adapt(flags=flags, buffer=0)
    of, _ = of.regrid(flags.astype(bool), 0)
    om = odg.Mesh(of, N, L, K)
    assert lm.num_elements == om.E and len(of.face_lists()[1]) > 0
    return lm, om


@pytest.mark.parametrize("t", [0.0, 4.5])
def test_vortex_state_matches_oracle(pkg, t):
    lm, om = _pair(pkg, 3, (6, 6), seed=1)
    lm.set_vortex(CENTER, BETA, UINF, t)
    np.testing.assert_allclose(lm.get_state(), ovx.vortex_state(om, CENTER, BETA, UINF, t),
                               rtol=0, atol=1e-13)


@pytest.mark.parametrize("precision,tol", [("fp64", 1e-12), ("fp32", 2e-5)])
@pytest.mark.parametrize("N,base", [(3, (4, 4)), (4, (3, 5))])
def test_periodic_rhs_matches_oracle(pkg, precision, tol, N, base):
    import torch
    lm, om = _pair(pkg, N, base, precision=precision, seed=N)
    q = ovx.vortex_state(om, CENTER, BETA, UINF, 0.7) + 0.01 * workloads.random_state(4, om.E, om.np_, seed=N)
    dt = torch.float64 if precision == "fp64" else torch.float32
    qt = torch.from_numpy(q).to(dt)
    got = lm.rhs(qt.cuda()).double().cpu().numpy()
    want = odg.rhs(om, qt.double().numpy())
    for v in range(4):
        assert np.abs(got[v] - want[v]).max() <= tol * np.abs(want[v]).max()


def vortex_run(pkg, precision="fp64", t_end=3.0, dt=0.0025, regrid_every=40, thr=1e-3, max_level=1):
    """32 x 32 periodic roots on [0, 12]^2, N = 3, one level where max |rho'| > thr (flags from
    the state on the host), SSP-RK3; returns the paper's error norm at t_end, the mass drift
    and the element count."""
    m = _lib_mesh(pkg, 3, (32, 32), max_level=max_level, precision=precision)
    NP = 16
    for _ in range(max_level):
        m.set_vortex(CENTER, BETA, UINF, 0.0)
        flags = (np.abs(m.get_state()[0]).reshape(-1, NP).max(axis=1) > thr).astype(np.uint8)
        m.adapt(flags=flags, buffer=1)
    m.set_vortex(CENTER, BETA, UINF, 0.0)
    m0 = m.integrals()[0]
    nsteps = int(round(t_end / dt))
    done = 0
    while done < nsteps:
        k = min(regrid_every, nsteps - done)
        m.step(dt, k)
        done += k
        if max_level and done < nsteps:
            flags = (np.abs(m.get_state()[0]).reshape(-1, NP).max(axis=1) > thr).astype(np.uint8)
            m.adapt(flags=flags, buffer=1)
    q = m.get_state().astype(np.float64)
    drift = abs(m.integrals()[0] - m0) / m0
    m.set_vortex(CENTER, BETA, UINF, t_end)
    exact = m.get_state().astype(np.float64)
    return ovx.l2_paper(q, exact), drift, m.num_elements


def test_vortex_amr_run_against_exact_solution(pkg):
    gold = json.load(open(os.path.join(HERE, "golden", "paper_values.json")))["isentropic_vortex"]
    err, drift, E = vortex_run(pkg)
    err_u, drift_u, _ = vortex_run(pkg, max_level=0)
    print("isentropic vortex: AMR L2 %.3e (paper %.3e), uniform 32x32 L2 %.3e, mass drift %.1e, "
          "%d elements" % (err, gold["l2_error_at_t3"], err_u, drift, E))
    assert E > 32 * 32
    assert drift <= 1e-13 and drift_u <= 1e-13
    assert err <= gold["l2_error_at_t3"]
    assert err < err_u
