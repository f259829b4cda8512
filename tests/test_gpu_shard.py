"""Sharded meshes on the device: each part computes only its SFC range of the leaf order, with the
face traces it shares with other parts (conforming faces and both sides of mortars) packed,
exchanged and unpacked by the library's halo kernels.  The owned ranges of the parts' results
must equal the unsharded result bit for bit.  Every element a part does not own starts as NaN,
so a trace missing from the halo lists, or a stage that reads beyond its range, shows up as a
NaN in the comparison.

- self-exchange: all parts of the mesh live on one device in one process; the exchange is a
  device copy between the parts' buffers (no kernel waits on another);
- two processes with the gloo backend on host copies of the packed slots (the transport a
  multi-GPU run would do with NCCL on device buffers)."""
import os
import socket

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


CASES = [(3, 3, (2, 2, 2), (2000.0,) * 3, "fp64", 2), (3, 7, (2, 2, 2), (2000.0,) * 3, "fp32", 3),
         (2, 4, (4, 3), (1200.0, 900.0), "fp64", 3), (3, 3, (2, 2, 2), (2000.0,) * 3, "fp32", 2)]


def _mesh(pkg, dim, N, base, length, precision, flags):
    m = pkg.Mesh(dim, N, base, length, max_level=2, precision=precision)
    if precision == "fp64":
        # a partitioned mesh runs layout 2 in place of the FP64 default 5 (whose face kernel
        # works on the whole mesh's face lists): the reference takes the same layout
        m.set_stage_kernel(2)
    for f in flags:
        m.adapt(flags=f, buffer=1)
    return m


def _flags(pkg, dim, N, base, length, precision):
    m = pkg.Mesh(dim, N, base, length, max_level=2, precision=precision)
    out = []
    for r in range(2):
        f = workloads.random_flags(m.num_elements, 0.3, seed=700 + r)
        out.append(f)
        m.adapt(flags=f, buffer=1)
    assert m.num_mortars > 0
    m.close()
    return out


def _exchange_local(parts, bufs):
    """The transport between parts living on one device: receiver p gets, from each sender q in
    increasing order, the slice of q's send buffer addressed to p."""
    import torch
    infos = [m.partition() for m in parts]
    per = infos[0][3]
    sends = []
    for m, (q, pp) in zip(parts, bufs):
        snd = infos[parts.index(m)][1]
        sb = torch.empty(sum(snd) * per, dtype=torch.float64 if m.precision == "fp64" else torch.float32,
                         device="cuda")
        m.halo_pack(q, pp, sb)
        sends.append(sb)
    torch.cuda.synchronize()
    for p, (m, (q, pp)) in enumerate(zip(parts, bufs)):
        pieces = []
        for s, sb in enumerate(sends):
            if s == p:
                continue
            snd = infos[s][1]
            off = sum(snd[:p])
            pieces.append(sb[off * per:(off + snd[p]) * per])
        rb = torch.cat(pieces) if pieces else sends[p][:0]
        assert rb.numel() == sum(infos[p][2]) * per
        m.halo_unpack(rb, q, pp)
    torch.cuda.synchronize()


def _nan_outside(q, lo, hi):
    x = q.copy()
    x[:, :lo] = np.nan
    x[:, hi:] = np.nan
    return x


@pytest.mark.parametrize("dim,N,base,length,precision,nparts", CASES)
def test_sharded_rhs_and_steps_equal_unsharded(pkg, dim, N, base, length, precision, nparts):
    import torch
    flags = _flags(pkg, dim, N, base, length, precision)
    ref = _mesh(pkg, dim, N, base, length, precision, flags)
    dtype = np.float64 if precision == "fp64" else np.float32
    q0 = workloads.random_state(ref.nv, ref.num_elements, ref.np_, seed=710, rho_scale=1e-4, u_scale=0.2,
                                theta_scale=0.02, dtype=dtype)
    parts = [_mesh(pkg, dim, N, base, length, precision, flags) for _ in range(nparts)]
    for p, m in enumerate(parts):
        m.set_partition(nparts, p)
    ranges = [m.partition()[0] for m in parts]
    assert ranges[0][0] == 0 and ranges[-1][1] == ref.num_elements
    assert all(ranges[i][1] == ranges[i + 1][0] for i in range(nparts - 1))
    assert any(sum(m.partition()[1]) > 0 for m in parts)
    # right-hand side of a caller's state (state planes exchanged, P' recomputed by dg_rhs)
    want = ref.rhs(torch.from_numpy(q0).cuda()).cpu().numpy()
    got = np.full_like(want, np.nan)
    qs = [torch.from_numpy(_nan_outside(q0, *r)).cuda() for r in ranges]
    _exchange_local(parts, [(q.data_ptr(), 0) for q in qs])
    for m, q, (lo, hi) in zip(parts, qs, ranges):
        out = torch.full_like(q, float("nan"))
        m.rhs(q, out)
        got[:, lo:hi] = out.cpu().numpy()[:, lo:hi]
    assert np.array_equal(got, want)
    # two SSP-RK3 steps, stage by stage, with the halo of each stage input (state and P')
    dt = 0.002
    ref.set_state(q0)
    ref.step(dt, 2)
    want = ref.get_state()
    for m, r in zip(parts, ranges):
        m.set_state(_nan_outside(q0, *r))
    for _ in range(2):
        for st in range(3):
            bufs = [m.stage_buffer(st) for m in parts]
            _exchange_local(parts, bufs)
            for m in parts:
                m.stage(st, dt)
    got = np.full_like(want, np.nan)
    for m, (lo, hi) in zip(parts, ranges):
        got[:, lo:hi] = m.get_state()[:, lo:hi]
    assert np.array_equal(got, want)


def test_partitioned_mesh_refuses_whole_mesh_calls(pkg):
    from paper_2404_16648_gb300.dg import DGError
    m = pkg.Mesh(2, 3, (4, 4), (1000.0, 1000.0), max_level=1)
    m.set_partition(2, 1)
    for call in (lambda: m.step(0.01, 1), lambda: m.integrals(),
                 lambda: m.adapt(flags=np.zeros(m.num_elements, np.uint8), buffer=0)):
        with pytest.raises(DGError):
            call()
    with pytest.raises(DGError):
        pkg.Batch([m], 0.01)
    m.set_partition(1, 0)
    m.step(0.01, 1)
    assert m.partition()[0] == (0, m.num_elements)


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    port = s.getsockname()[1]
    s.close()
    return port


def _rank_main(rank, world, port, flags, q0, out_path):
    import torch
    import torch.distributed as dist
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    import paper_2404_16648_gb300 as pkg
    from paper_2404_16648_gb300 import shard
    torch.cuda.set_device(0)
    dim, N, base, length, precision, _ = CASES[0]
    m = _mesh(pkg, dim, N, base, length, precision, flags)
    m.set_partition(world, rank)
    lo, hi = m.partition()[0]
    m.set_state(_nan_outside(q0, lo, hi))
    shard.sharded_step(m, 0.002, nsteps=2)
    np.save(out_path % rank, m.get_state()[:, lo:hi])
    dist.barrier()
    dist.destroy_process_group()


@pytest.mark.timeout(600)
def test_two_processes_gloo_exchange(pkg, tmp_path):
    import torch.multiprocessing as tmp
    dim, N, base, length, precision, _ = CASES[0]
    flags = _flags(pkg, dim, N, base, length, precision)
    ref = _mesh(pkg, dim, N, base, length, precision, flags)
    q0 = workloads.random_state(ref.nv, ref.num_elements, ref.np_, seed=711, rho_scale=1e-4, u_scale=0.2,
                                theta_scale=0.02)
    ref.set_state(q0)
    ref.step(0.002, 2)
    want = ref.get_state()
    out = str(tmp_path / "part%d.npy")
    tmp.spawn(_rank_main, args=(2, _free_port(), flags, q0, out), nprocs=2, join=True)
    got = np.concatenate([np.load(out % r) for r in range(2)], axis=1)
    assert np.array_equal(got, want)
