"""Sensitivity of a forecast diagnostic to the initial theta' field, behind torch.autograd.

J(theta') = kinetic-energy integral after `nsteps` SSP-RK3 steps from the hydrostatic-pressure
state of the nodal field theta' (the use case of variational data assimilation).  The forward
pass steps through the C ABI a segment at a time and keeps a checkpoint of the state every
`every` steps, and the stage inputs of every step of the last segment (dg_step_record); the
backward pass recomputes each earlier segment once from its checkpoint, keeping every step's
stage inputs, runs the hand-written step transposes on them (dg_step_vjp_record) in reverse,
then the transpose of the initial-state map (dg_theta_vjp).  Every operation runs in the library's kernels; this module only orders calls.
"""
import torch


def _final_state(mesh, theta, dt, nsteps, every, keep_last=False):
    """Final state, the checkpoint at the start of every segment of `every` steps, and (with
    keep_last) the step records of the last segment, which the backward pass then needs not
    recompute."""
    mesh.set_theta(theta)
    q = torch.empty(mesh.state_shape, dtype=torch.float64, device=theta.device)
    mesh.get_state(q)
    checkpoints = []
    last = None
    for start in range(0, nsteps, every):
        stop = min(start + every, nsteps)
        checkpoints.append(q.clone())
        if keep_last and stop == nsteps:
            last = []
            for _ in range(start, stop):
                rec = torch.empty(mesh.record_shape, dtype=torch.float64, device=theta.device)
                mesh.step_record(q, q, rec, dt)
                last.append(rec)
        else:
            mesh.step_state(q, q, dt, stop - start)
    return q, checkpoints, last


def final_ke(mesh, theta, dt, nsteps):
    """J(theta') without gradient bookkeeping."""
    mesh.set_theta(theta)
    mesh.step(dt, nsteps)
    return float(mesh.integrals()[2])


class FinalKineticEnergy(torch.autograd.Function):
    """J = KE(state after nsteps) as a differentiable function of theta' (device, FP64)."""

    @staticmethod
    def forward(ctx, theta, mesh, dt, nsteps, every):
        q, checkpoints, last = _final_state(mesh, theta, dt, nsteps, every, keep_last=True)
        mesh.set_state(q)
        J = float(mesh.integrals()[2])
        ctx.mesh, ctx.dt, ctx.nsteps, ctx.every = mesh, dt, nsteps, every
        ctx.last = last
        ctx.save_for_backward(theta, q, *checkpoints)
        return torch.tensor(J, dtype=torch.float64, device=theta.device)

    @staticmethod
    def backward(ctx, grad_out):
        mesh, dt, nsteps, every = ctx.mesh, ctx.dt, ctx.nsteps, ctx.every
        theta, qT, *checkpoints = ctx.saved_tensors
        lam = mesh.ke_grad(qT) * grad_out
        spare = torch.empty_like(lam)
        q = torch.empty_like(qT)
        for seg in reversed(range(len(checkpoints))):
            start = seg * every
            stop = min(start + every, nsteps)
            if seg == len(checkpoints) - 1 and ctx.last is not None:
                records = ctx.last          # kept by the forward pass
            else:
                # recompute the segment once, keeping every step's stage inputs
                records = []
                q.copy_(checkpoints[seg])
                for _ in range(start, stop):
                    rec = torch.empty(mesh.record_shape, dtype=torch.float64, device=qT.device)
                    mesh.step_record(q, q, rec, dt)
                    records.append(rec)
            for rec in reversed(records):
                mesh.step_vjp_record(rec, dt, lam, spare)
                lam, spare = spare, lam
        ctx.last = None
        grad_theta = mesh.theta_vjp(theta, lam)
        return grad_theta, None, None, None, None


def ke_gradient(mesh, theta, dt, nsteps, every=20):
    """(J, dJ/dtheta') for a device FP64 tensor theta of shape (elements, nodes per element)."""
    th = theta.detach().clone().requires_grad_(True)
    J = FinalKineticEnergy.apply(th, mesh, dt, nsteps, every)
    J.backward()
    return float(J.item()), th.grad
