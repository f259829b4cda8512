"""Multi-rank path on CPU: the space-filling-curve partition and halo lists of the host tree
(Sec. 3.1 names SFC partitioning), checked against brute force over the oracle's neighbour
search, and a two-rank gloo run in which each rank evaluates the right-hand side of its own
leaf range from its own elements plus the face traces received from the other rank.  The result
must equal the single-process oracle right-hand side bit for bit: a trace missing from the halo
lists would leave a NaN in it.  The benchmark's max-over-ranks timing helper runs on the same
process group."""
import os
import socket
import sys

import numpy as np
import pytest

import workloads
from oracle import dg as odg, forest as fo

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def pkg():
    from paper_2404_16648_gb300 import build as b
    b.build()
    import paper_2404_16648_gb300 as p
    return p


def _adapted_pair(pkg, base, max_level, rounds, seed, p=0.3, B=1):
    lf = pkg.Forest(len(base), base, max_level)
    of = fo.Forest(base, max_level)
    for r in range(rounds):
        flags = workloads.random_flags(len(of), p, seed=seed + r)
        lf.regrid(flags, B)
        of, _ = of.regrid(flags.astype(bool), B)
    return lf, of


def _brute_halo(of, starts, part):
    owner = np.searchsorted(starts, np.arange(len(of)), side="right") - 1
    rows = []
    for e in range(starts[part], starts[part + 1]):
        for a in range(of.d):
            for s in (0, 1):
                kind, nb = of.neighbor(e, a, s)
                nbs = [] if kind == "boundary" else (nb if kind == "fine" else [nb])
                for n in nbs:
                    if owner[n] != part:
                        rows.append((e, a, s, n, owner[n]))
    return np.array(rows, dtype=np.int32).reshape(-1, 5)


@pytest.mark.parametrize("base,max_level,rounds", [((4, 3), 3, 3), ((3, 2, 2), 2, 2), ((5, 5), 0, 0)])
@pytest.mark.parametrize("nparts", [1, 2, 3, 7])
def test_partition_and_halo_match_brute_force(pkg, base, max_level, rounds, nparts):
    lf, of = _adapted_pair(pkg, base, max_level, rounds, seed=40 + len(base))
    starts = lf.partition(nparts)
    E = len(of)
    assert starts[0] == 0 and starts[-1] == E
    sizes = np.diff(starts)
    assert sizes.min() >= 0 and sizes.max() - sizes.min() <= 1
    for part in range(nparts):
        np.testing.assert_array_equal(lf.halo(nparts, part), _brute_halo(of, starts, part))
    # every cross-part face appears once from each side
    seen = set()
    for part in range(nparts):
        for e, a, s, n, op in lf.halo(nparts, part):
            seen.add((int(e), int(n)))
    assert all((n, e) in seen for (e, n) in seen)


def test_partition_rejects_bad_arguments(pkg):
    from paper_2404_16648_gb300.dg import DGError
    f = pkg.Forest(2, (2, 2), 1)
    with pytest.raises(DGError):
        f.partition(0)
    with pytest.raises(DGError):
        f.halo(2, 2)


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


CASE = dict(base=(3, 2), max_level=2, rounds=2, N=3, length=(1500.0, 1000.0), seed=61)


def _rank_main(rank, world, port, out_q):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank),
                      WORLD_SIZE=str(world))
    sys.path.insert(0, ROOT)
    import torch
    import torch.distributed as dist
    import paper_2404_16648_gb300 as pkg
    import bench
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        c = CASE
        lf, of = _adapted_pair(pkg, c["base"], c["max_level"], c["rounds"], seed=c["seed"])
        mesh = odg.Mesh(of, c["N"], c["length"])
        q_full = workloads.random_state(mesh.nv, mesh.E, mesh.np_, seed=62, rho_scale=1e-3,
                                        u_scale=1.0, theta_scale=0.3)
        starts = lf.partition(world)
        lo, hi = int(starts[rank]), int(starts[rank + 1])
        # this rank holds only its own elements; everything else is unknown
        q = np.full_like(q_full, np.nan)
        q[:, lo:hi] = q_full[:, lo:hi]
        # the host tree is replicated, so each rank knows what every other rank needs from it
        sends, recvs = [], []
        for peer in range(world):
            if peer == rank:
                continue
            need = [r for r in lf.halo(world, rank) if r[4] == peer]
            give = [r for r in lf.halo(world, peer) if r[4] == rank]
            # a trace is the neighbour's face on the opposite side of the same axis
            out = np.stack([q[:, n, mesh.trace_index(a, 1 - s)] for (_, a, s, n, _) in give]) \
                if give else np.zeros((0,))
            buf = torch.empty((len(need), mesh.nv, len(mesh.trace_index(0, 0))), dtype=torch.float64)
            sends.append(dist.isend(torch.from_numpy(np.ascontiguousarray(out)), dst=peer))
            recvs.append((dist.irecv(buf, src=peer), buf, need))
        for w in sends:
            w.wait()
        for req, buf, need in recvs:
            req.wait()
            for k, (_, a, s, n, _) in enumerate(need):
                q[:, n, mesh.trace_index(a, 1 - s)] = buf[k].numpy()
        mine = odg.rhs(mesh, q, elems=np.arange(lo, hi))[:, lo:hi]
        parts = [None] * world
        dist.all_gather_object(parts, (lo, hi, mine))
        t = bench._barrier_max(0.5 + rank, world, device="cpu")
        if rank == 0:
            full = odg.rhs(mesh, q_full)
            got = np.full_like(full, np.nan)
            for lo_, hi_, m in parts:
                got[:, lo_:hi_] = m
            out_q.put((bool(np.array_equal(got, full)), float(t), len(lf.halo(world, 0))))
    finally:
        dist.destroy_process_group()


def test_two_rank_gloo_rhs_equals_single_process(pkg):
    import multiprocessing as mp
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_rank_main, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    try:
        equal, tmax, nhalo = q.get(timeout=240)
    finally:
        for p in procs:
            p.join(timeout=60)
    assert all(p.exitcode == 0 for p in procs)
    assert nhalo > 0
    assert equal
    assert tmax == 1.5
