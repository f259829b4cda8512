"""GPU adjoint: the hand-written VJPs against the oracle's complex-step discrete adjoint, and the
checkpointed gradient of the final kinetic energy against central finite differences."""
import time

import numpy as np
import pytest

import workloads
from oracle import adjoint as oadj, dg as odg, forest as ofo

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def pkg():
    import torch
    assert torch.cuda.is_available()
    from paper_2404_16648_gb300 import build as b
    b.build()
    import paper_2404_16648_gb300 as p
    return p


def _pair(pkg, dim, N, base, length, seed, p=0.4):
    lm = pkg.Mesh(dim, N, base, length, max_level=1)
    of = ofo.Forest(base, 1)
    flags = workloads.random_flags(len(of), p, seed)
    flags[0] = 1
    lm.adapt(flags=flags, buffer=0)
    of, _ = of.regrid(flags.astype(bool), 0)
    om = odg.Mesh(of, N, length)
    assert lm.num_elements == om.E and len(of.face_lists()[1]) > 0
    return lm, om


def _rel(got, want):
    return np.abs(got - want).max() / np.abs(want).max()


@pytest.mark.parametrize("dim,N,base,length", [
    (2, 3, (2, 2), (1000.0, 1000.0)),
    (2, 2, (3, 2), (1500.0, 1000.0)),
    (3, 2, (2, 1, 2), (1000.0, 500.0, 1000.0)),
])
def test_rhs_vjp_matches_oracle(pkg, dim, N, base, length):
    import torch
    lm, om = _pair(pkg, dim, N, base, length, seed=N + dim)
    q = workloads.random_state(om.nv, om.E, om.np_, seed=50 + N, rho_scale=1e-3, u_scale=1.0,
                               theta_scale=0.3)
    lam = workloads.random_state(om.nv, om.E, om.np_, seed=60 + N, rho_scale=1.0, u_scale=1.0,
                                 theta_scale=1.0)
    got = lm.rhs_vjp(torch.from_numpy(q).cuda(), torch.from_numpy(lam).cuda()).cpu().numpy()
    want = oadj.rhs_vjp(om, q, lam)
    assert _rel(got, want) <= 1e-11


def test_rhs_vjp_with_zero_velocity_ties(pkg):
    # fluid at rest with theta' jumps: u = 0 everywhere (sign(0) = 0) and equal wave speeds on
    # walls (ties to the low side)
    import torch
    lm, om = _pair(pkg, 2, 2, (2, 2), (1000.0, 1000.0), seed=70)
    q = workloads.random_state(om.nv, om.E, om.np_, seed=71)
    q[1:3] = 0.0
    lam = workloads.random_state(om.nv, om.E, om.np_, seed=72, rho_scale=1.0, u_scale=1.0, theta_scale=1.0)
    got = lm.rhs_vjp(torch.from_numpy(q).cuda(), torch.from_numpy(lam).cuda()).cpu().numpy()
    want = oadj.rhs_vjp(om, q, lam)
    assert _rel(got, want) <= 1e-11


def test_step_vjp_matches_oracle(pkg):
    import torch
    lm, om = _pair(pkg, 2, 2, (2, 2), (1000.0, 1000.0), seed=80)
    q = workloads.random_state(om.nv, om.E, om.np_, seed=81, rho_scale=1e-4, u_scale=0.5,
                               theta_scale=0.05)
    lam = workloads.random_state(om.nv, om.E, om.np_, seed=82, rho_scale=1.0, u_scale=1.0, theta_scale=1.0)
    dt = 0.005
    got = lm.step_vjp(torch.from_numpy(q).cuda(), dt, torch.from_numpy(lam).cuda()).cpu().numpy()
    want = oadj.step_vjp(om, q, dt, lam)
    assert _rel(got, want) <= 1e-11


def test_step_state_matches_step(pkg):
    import torch
    lm, om = _pair(pkg, 3, 3, (2, 2, 2), (2000.0,) * 3, seed=90)
    q = workloads.random_state(om.nv, om.E, om.np_, seed=91, rho_scale=1e-4, u_scale=0.1, theta_scale=0.01)
    out = lm.step_state(torch.from_numpy(q).cuda(), torch.empty(lm.state_shape, dtype=torch.float64,
                                                                device="cuda"), 0.002, 3).cpu().numpy()
    want = odg.step(om, q, 0.002, 3)
    assert _rel(out - q, want - q) <= 1e-11


def test_bubble_theta_matches_oracle(pkg):
    cfg = workloads.ADJOINT_3D
    lm = pkg.Mesh(3, 2, (3, 3, 3), cfg["length"])
    om = odg.Mesh(ofo.Forest((3, 3, 3), 0), 2, cfg["length"])
    r = cfg["rff"]
    sigma, k, ph = workloads.rff_draws(3, r["sigma"], r["length"], 64)
    b = cfg["bubble"]
    got = lm.bubble_theta(**b, rff=(sigma, k, ph)).cpu().numpy()
    want = odg.bubble_theta(om, b["center"], b["radius"], b["amp"]) + odg.rff_theta(om, sigma, k, ph)
    np.testing.assert_allclose(got, want, rtol=0, atol=1e-12)


def test_gradient_matches_oracle_complex_step(pkg):
    from paper_2404_16648_gb300 import adjoint as ladj
    lm, om = _pair(pkg, 3, 2, (2, 2, 2), (2000.0,) * 3, seed=100, p=0.3)
    rng = np.random.default_rng(101)
    theta = 0.5 * rng.standard_normal((om.E, om.np_))
    import torch
    dt, nsteps = 0.01, 6
    J, g = ladj.ke_gradient(lm, torch.from_numpy(theta).cuda(), dt, nsteps, every=4)
    g = g.cpu().numpy().ravel()
    assert abs(J - oadj.final_ke(om, theta, dt, nsteps)) <= 1e-12 * J
    nodes = list(workloads.sample_elements(theta.size, 8, seed=102))
    want = oadj.final_ke_gradient(om, theta, dt, nsteps, nodes)
    assert np.abs(g[nodes] - want).max() <= 1e-9 * np.abs(want).max()


def test_adjoint_gradient_against_finite_differences(pkg):
    """The 3D adjoint workload: 12^3 elements, N = 5, warm bubble plus a Gaussian random theta'
    (sigma 0.05 K, correlation length 300 m), 200 steps with a checkpoint every 20; gradient of the
    final kinetic energy against central differences (h = 1e-6 K) at 64 random nodes."""
    import torch
    from paper_2404_16648_gb300 import adjoint as ladj
    cfg = workloads.ADJOINT_3D
    m = pkg.Mesh(3, cfg["N"], cfg["base"], cfg["length"])
    r = cfg["rff"]
    rff = workloads.rff_draws(3, r["sigma"], r["length"], r["features"])
    theta = m.bubble_theta(**cfg["bubble"], rff=rff)
    dt, nsteps = cfg["dt"], cfg["steps"]
    t0 = time.perf_counter()
    J0 = ladj.final_ke(m, theta, dt, nsteps)
    torch.cuda.synchronize()
    t_fwd = time.perf_counter() - t0
    t0 = time.perf_counter()
    J, g = ladj.ke_gradient(m, theta, dt, nsteps, every=20)
    torch.cuda.synchronize()
    t_adj = time.perf_counter() - t0
    assert abs(J - J0) <= 1e-12 * abs(J0)
    g = g.cpu().numpy().ravel()
    nodes = workloads.sample_elements(theta.numel(), 64, seed=110)
    h = 1e-6
    fd = []
    flat = theta.view(-1)
    for j in nodes:
        tp = flat.clone(); tp[j] += h
        tm = flat.clone(); tm[j] -= h
        fd.append((ladj.final_ke(m, tp.view_as(theta), dt, nsteps) -
                   ladj.final_ke(m, tm.view_as(theta), dt, nsteps)) / (2 * h))
    fd = np.array(fd)
    err = np.abs(g[nodes] - fd).max() / np.abs(fd).max()
    print("adjoint vs FD: max rel %.2e; adjoint/forward time %.2f" % (err, t_adj / t_fwd))
    assert err <= 1e-6


def test_recorded_step_equals_recomputed_step(pkg):
    """dg_step_record keeps the stage inputs of a step; its output equals dg_step_state and the
    transpose from the record equals dg_step_vjp (which recomputes the stages), bit for bit."""
    import torch
    lm, om = _pair(pkg, 3, 3, (2, 2, 2), (2000.0,) * 3, seed=130, p=0.4)
    q = torch.from_numpy(workloads.random_state(om.nv, om.E, om.np_, seed=131, rho_scale=1e-4,
                                                u_scale=0.5, theta_scale=0.05)).cuda()
    lam = torch.from_numpy(workloads.random_state(om.nv, om.E, om.np_, seed=132, rho_scale=1.0,
                                                  u_scale=1.0, theta_scale=1.0)).cuda()
    dt = 0.004
    rec = torch.empty(lm.record_shape, dtype=torch.float64, device="cuda")
    out_rec = lm.step_record(q, torch.empty_like(q), rec, dt)
    out_ref = lm.step_state(q, torch.empty_like(q), dt)
    assert torch.equal(out_rec, out_ref)
    assert torch.equal(rec[0, :om.nv].reshape(q.shape), q)
    g_rec = lm.step_vjp_record(rec, dt, lam)
    g_ref = lm.step_vjp(q, dt, lam)
    assert torch.equal(g_rec, g_ref)        # dg_step_vjp itself is checked against the oracle above
