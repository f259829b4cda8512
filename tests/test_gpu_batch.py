"""Batched solves: one graph-captured launch per (precision, N) group against the same meshes
advanced one launch at a time (bit-identical with the same kernel layout)."""
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


def _make(pkg, inst, refine=False):
    ms = []
    for k, d in enumerate(inst):
        m = pkg.Mesh(2, d["N"], d["base"], (1000.0, 1000.0), max_level=1, precision=d["precision"])
        if refine:
            m.adapt(flags=workloads.random_flags(m.num_elements, 0.2, seed=300 + k), buffer=0)
        m.set_bubble(**d["bubble"])
        ms.append(m)
    return ms


def _small(count, seed):
    return workloads.batch_instances(count, seed=seed, meshes=((4, 4), (6, 3), (8, 5)))


@pytest.mark.parametrize("refine", [False, True])
def test_batch_matches_one_at_a_time(pkg, refine):
    inst = _small(14, seed=11)
    a = _make(pkg, inst, refine)
    b = _make(pkg, inst, refine)
    # one refinement level halves h, so dt is halved to stay inside the RK3 limit
    dts = [d["dt"] * (0.5 if refine else 1.0) for d in inst]
    batch = pkg.Batch(a, dts)
    layouts = batch.autotune(reps=2)
    assert set(layouts) <= {1, 2, 5}
    for m, layout in zip(b, layouts):
        m.set_stage_kernel(int(layout))
    batch.run(6, graph=True)
    for m, dt in zip(b, dts):
        m.step(dt, 6)
    for ma, mb in zip(a, b):
        x = ma.get_state()
        assert np.all(np.isfinite(x))
        assert np.array_equal(x, mb.get_state())


def test_batch_graph_equals_eager_and_continues(pkg):
    inst = _small(6, seed=12)
    a = _make(pkg, inst)
    b = _make(pkg, inst)
    ba = pkg.Batch(a, [d["dt"] for d in inst])
    bb = pkg.Batch(b, [d["dt"] for d in inst])
    ba.run(3, graph=True)
    ba.run(2, graph=True)
    bb.run(5, graph=False)
    for ma, mb in zip(a, b):
        assert np.array_equal(ma.get_state(), mb.get_state())
        assert np.all(np.isfinite(ma.get_state()))


def test_batch_rejects_a_regridded_member(pkg):
    from paper_2404_16648_gb300.dg import DGError
    inst = _small(3, seed=13)
    ms = _make(pkg, inst)
    batch = pkg.Batch(ms, [d["dt"] for d in inst])
    ms[1].adapt(flags=np.ones(ms[1].num_elements, np.uint8), buffer=0)
    with pytest.raises(DGError):
        batch.run(1)


@pytest.mark.parametrize("refine", [False, True])
def test_batch_members_against_the_oracle(pkg, refine):
    """Batch members checked against the oracle itself, not only against single-mesh runs: two
    FP64 and two FP32 members of different degree, each stepped three times in the batch and
    compared with oracle.dg.step on its own (independently built) forest.  Bounds on the state
    change per variable: FP64 1e-11, FP32 1e-4 (three steps of FP32 tendencies, each stage
    within 2e-5 of max|rhs|)."""
    from oracle import dg as odg, forest as ofo
    pool = workloads.batch_instances(64, seed=15, meshes=((4, 4), (6, 3), (5, 5)))
    picked, seen = [], set()
    for d in pool:
        key = (d["precision"], d["N"])
        if key not in seen and sum(p["precision"] == d["precision"] for p in picked) < 2:
            picked.append(d)
            seen.add(key)
    assert len(picked) == 4
    ms = _make(pkg, picked, refine)
    dts = [d["dt"] * (0.5 if refine else 1.0) for d in picked]
    q0s, oms = [], []
    for k, (m, d) in enumerate(zip(ms, picked)):
        of = ofo.Forest(d["base"], 1)
        if refine:
            of, _ = of.regrid(workloads.random_flags(len(of), 0.2, seed=300 + k).astype(bool), 0)
        om = odg.Mesh(of, d["N"], (1000.0, 1000.0))
        assert om.E == m.num_elements
        dtype = np.float64 if d["precision"] == "fp64" else np.float32
        q0 = workloads.random_state(om.nv, om.E, om.np_, seed=400 + k, rho_scale=1e-4, u_scale=0.2,
                                    theta_scale=0.02, dtype=dtype)
        m.set_state(q0)
        q0s.append(q0.astype(np.float64))
        oms.append(om)
    batch = pkg.Batch(ms, dts)
    batch.run(3, graph=True)
    for m, om, q0, dt, d in zip(ms, oms, q0s, dts, picked):
        got = m.get_state().astype(np.float64) - q0
        want = odg.step(om, q0, dt, 3) - q0
        err = max(np.abs(got[v] - want[v]).max() / np.abs(want[v]).max() for v in range(om.nv))
        assert err <= (1e-11 if d["precision"] == "fp64" else 1e-4), (d["precision"], d["N"], err)


def test_batch_persistent_launch_shape_and_mixed_dimensions(pkg):
    """2D members run through the persistent launch (work items of every degree and precision
    in one kernel); a 3D member in the same batch takes the grouped launch.  Every member still
    matches its single-mesh run bit for bit with the chosen layout."""
    inst = _small(8, seed=16)
    a = _make(pkg, inst, refine=True)
    b = _make(pkg, inst, refine=True)
    for ms in (a, b):
        m3 = pkg.Mesh(3, 3, (2, 2, 2), (1000.0,) * 3, max_level=1)
        m3.adapt(flags=workloads.random_flags(m3.num_elements, 0.4, seed=17), buffer=0)
        m3.set_bubble(center=(500.0, 500.0, 350.0), radius=(250.0,) * 3, amp=0.5)
        ms.append(m3)
    dts = [d["dt"] * 0.5 for d in inst] + [0.002]
    batch = pkg.Batch(a, dts)
    layouts = batch.autotune(reps=2)
    shape = batch.shape()
    assert shape["grid"] > 0 and shape["items_per_stage"] > 0
    assert shape["ctas_per_sm_budget"] in (2, 4) and shape["tiles_per_item"] in (1, 2, 4, 8)
    for m, layout in zip(b, layouts):
        m.set_stage_kernel(int(layout))
    batch.run(4, graph=True)
    for m, dt in zip(b, dts):
        m.step(dt, 4)
    for ma, mb in zip(a, b):
        x = ma.get_state()
        assert np.all(np.isfinite(x))
        assert np.array_equal(x, mb.get_state())


@pytest.mark.parametrize("layout", [1, 2, 5])
def test_batch_every_degree_both_precisions(pkg, layout):
    """One persistent launch over members of every degree N = 1..8 in both precisions, each with
    hanging faces, against the same meshes stepped one launch at a time with the same layout
    (layout 5, face work items beside the mortar items, is for FP64 members; FP32 members take
    layout 2 there)."""
    def make():
        ms = []
        for k, (N, prec) in enumerate([(N, p) for N in range(1, 9) for p in ("fp64", "fp32")]):
            m = pkg.Mesh(2, N, (3, 2), (900.0, 600.0), max_level=1, precision=prec)
            m.set_stage_kernel(layout if (prec == "fp64" or layout != 5) else 2)
            m.adapt(flags=workloads.random_flags(m.num_elements, 0.5, seed=500 + k), buffer=0)
            q = workloads.random_state(m.nv, m.num_elements, m.np_, seed=600 + k, rho_scale=1e-4,
                                       u_scale=0.2, theta_scale=0.02,
                                       dtype=np.float64 if prec == "fp64" else np.float32)
            m.set_state(q)
            ms.append(m)
        return ms
    a, b = make(), make()
    batch = pkg.Batch(a, 0.002)
    batch.run(3, graph=True)
    for m in b:
        m.step(0.002, 3)
    for ma, mb in zip(a, b):
        assert ma.num_mortars > 0
        assert np.array_equal(ma.get_state(), mb.get_state())
