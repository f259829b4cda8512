"""Discrete adjoint of the oracle's dGSEM operator (oracle; test infrastructure only).

The adjoint of a discrete map is the transpose of its Jacobian.  Here every Jacobian column is
obtained by complex-step differentiation of the oracle itself (Squire & Trapp 1998):
J e_j = Im(f(q + i h e_j)) / h with h = 1e-30, exact to rounding because no subtraction occurs.
So J^T lam is assembled entry by entry as (J^T lam)_j = lam . J e_j.  This is the plain definition
(no hand-derived transposes), usable on small meshes only.  The non-smooth parts of the Rusanov
flux (|u|, max) follow the derivative convention of physics.abs_cs / physics.max_cs: the active
branch, ties to the low side, sign(0) = 0.

Pinned by tests/test_oracle_adjoint.py: rhs_vjp and step_vjp by the adjoint identity
<lam, J v> = <J^T lam, v> with J v from central finite differences of dg.rhs and dg.step on
meshes with hanging faces (2D and 3D; planted mistakes in a copy of step_vjp -- half the time
step, lambda paired with the wrong variable, columns given to the wrong element -- fail it), the
local-support shortcut against full evaluation, and the final-KE gradient against central
differences.
"""
import numpy as np

from . import dg

H = 1e-30


def _support(mesh, e):
    """Elements whose tendency can depend on element e's state: e and its face neighbours
    (through a mortar the coarse element touches every fine one and vice versa)."""
    return np.array(sorted({e} | set(mesh.forest.face_neighbors(e))), dtype=np.int64)


def rhs_vjp(mesh, q, lam, local=True):
    """J(q)^T lam for J = d dg.rhs / dq, by complex-step columns."""
    out = np.zeros(q.size)
    nv, E, NP = q.shape
    for j in range(q.size):
        v, rem = divmod(j, E * NP)
        e, n = divmod(rem, NP)
        qc = q.astype(complex)
        qc[v, e, n] += 1j * H
        if local:
            sup = _support(mesh, e)
            r = dg.rhs(mesh, qc, elems=sup)
            out[j] = np.sum(lam[:, sup] * r[:, sup].imag) / H
        else:
            out[j] = np.sum(lam * dg.rhs(mesh, qc).imag) / H
    return out.reshape(q.shape)


def step_vjp(mesh, q, dt, lam):
    """(d ssprk3_step(q) / dq)^T lam, by complex-step columns over the whole mesh."""
    out = np.zeros(q.size)
    for j in range(q.size):
        qc = q.astype(complex)
        qc.flat[j] += 1j * H
        out[j] = np.sum(lam * dg.step(mesh, qc, dt, 1).imag) / H
    return out.reshape(q.shape)


def ke_functional(mesh, q):
    """KE = sum_nodes w J |U|^2 / (2 rho) (complex-safe; the KE entry of dg.integrals)."""
    rb, _, _ = mesh.bg
    rho = rb + q[0]
    ke = 0.5 * np.sum(q[1:1 + mesh.d] ** 2, axis=0) / rho
    W = mesh.wnode[None, :] * mesh.J[:, None]
    return np.sum(W * ke)


def final_ke(mesh, theta, dt, nsteps):
    """J(theta') = KE after nsteps SSP-RK3 steps from the hydrostatic-pressure state of theta'."""
    q = dg.state_from_theta(mesh, theta)
    q = dg.step(mesh, q, dt, nsteps)
    return ke_functional(mesh, q)


def final_ke_gradient(mesh, theta, dt, nsteps, nodes):
    """dJ/dtheta' at the flat node indices `nodes`, one complex-step run per node."""
    g = np.zeros(len(nodes))
    for k, j in enumerate(nodes):
        tc = theta.astype(complex)
        tc.flat[j] += 1j * H
        g[k] = final_ke(mesh, tc, dt, nsteps).imag / H
    return g
