"""Halo exchange of a sharded mesh between processes (argument marshalling and transport only).

Each rank owns part `rank` of the SFC partition of a replicated tree (Mesh.set_partition).  The
library packs the face traces other parts need and unpacks the ones received (dg_halo_pack /
dg_halo_unpack, CUDA kernels); this module moves the packed slots between ranks with
torch.distributed point-to-point calls: on the device with the NCCL backend, through host copies
with gloo.  No arithmetic of the method happens here.
"""
import torch
import torch.distributed as dist


def exchange(mesh, q, pp, group=None):
    """Exchanges the halo traces of the device state at address q (full-size layout) and its P'
    plane at address pp (0/None: state planes only) with every other part."""
    (lo, hi), snd, rcv, per = mesh.partition()
    nparts = len(snd)
    if nparts <= 1:
        return
    dtype = torch.float64 if mesh.precision == "fp64" else torch.float32
    send = torch.empty(sum(snd) * per, dtype=dtype, device="cuda")
    recv = torch.empty(sum(rcv) * per, dtype=dtype, device="cuda")
    mesh.halo_pack(q, pp, send)
    torch.cuda.synchronize()
    on_device = dist.get_backend(group) == "nccl"
    sbuf = send if on_device else send.cpu()
    rbuf = recv if on_device else torch.empty(recv.shape, dtype=dtype)
    ops = []
    off = 0
    for p in range(nparts):
        if snd[p]:
            ops.append(dist.P2POp(dist.isend, sbuf[off * per:(off + snd[p]) * per], p, group))
        off += snd[p]
    off = 0
    for p in range(nparts):
        if rcv[p]:
            ops.append(dist.P2POp(dist.irecv, rbuf[off * per:(off + rcv[p]) * per], p, group))
        off += rcv[p]
    if ops:
        for r in dist.batch_isend_irecv(ops):
            r.wait()
    if not on_device:
        recv.copy_(rbuf)
    mesh.halo_unpack(recv, q, pp)


def sharded_step(mesh, dt, nsteps=1, group=None):
    """nsteps SSP-RK3 steps of a partitioned mesh: before each of the three stages the halo of
    that stage's input (state and P') is exchanged."""
    for _ in range(nsteps):
        for st in range(3):
            q, pp = mesh.stage_buffer(st)
            exchange(mesh, q, pp, group)
            mesh.stage(st, dt)
