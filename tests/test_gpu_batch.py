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
    assert set(layouts) <= {1, 2}
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
