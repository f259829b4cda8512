"""Passive tracer advected by a prescribed wind: the linear-advection test of Sec. 4.2 (swirling
deformational flow, after LeVeque) and the conservation comparison of its last figure, mortar
method vs point-to-point interpolation on hanging faces (Sec. 3.3, Sec. 4.2).

Test infrastructure, like the rest of ``oracle/``: plain FP64 numpy, no code shared with the
CUDA library.

Equation (Eq. 1, tracer row): dC/dt + div(C u) = 0 with the prescribed 2D wind of Sec. 4.2,

    u =  sin^2(pi x) sin(2 pi y) g(t),   v = -sin^2(pi y) sin(2 pi x) g(t),   g = cos(pi t / T),

which is divergence free and reverses at t = T/2, so the exact solution at t = T is the initial
cosine bell C = (h_max/2)(1 + cos(pi r / r_c)), r <= r_c.

Discretisation: the strong-form dGSEM of Sec. 2.2 on the oracle's Mesh (LGL nodes, D along each
axis, lift (2/h)/w0) with the upwind flux F* = u_n (C- + C+)/2 - |u_n| (C+ - C-)/2, which is the
Rusanov flux of Sec. 2.2 for a scalar with a continuous wind.  Walls carry no flux (mirror state:
the normal wind reverses, so F* = 0).  Hanging faces, ``mode``:

* "mortar": the coarse trace is projected onto each fine face with P = M^-1 S, F* is solved on
  the fine face nodes, the fine side lifts it directly and the coarse side receives
  sum_m s M^-1 S^T F*_m (the method of Sec. 3.3; conservative);
* "interp": the fine side is treated as above, but the coarse side solves its own F* at its own
  face nodes against the fine traces evaluated there (point-to-point interpolation, the
  non-conservative alternative the paper compares against).  A coarse node at the midpoint of
  the face, which lies on both fine faces, takes the mean of the two fine values.

Readings (the paper does not state them): h_max = 1, the bell at (0.25, 0.25) with r_c = 0.25
(Sec. 4.2), refinement where max |C| > 0.05, one extra level, buffer 2, 80 regrids over T = 5.

Pins: ``tests/test_oracle_tracer.py``.
"""
import math

import numpy as np

from . import basis as bmod


def leveque_wind(x, y, t, T):
    """Prescribed wind of Sec. 4.2 at points (x, y) and time t (period T)."""
    g = math.cos(math.pi * t / T)
    u = np.sin(math.pi * x) ** 2 * np.sin(2.0 * math.pi * y) * g
    v = -np.sin(math.pi * y) ** 2 * np.sin(2.0 * math.pi * x) * g
    return u, v


def bell(mesh, center, radius, amp):
    """C = amp (1 + cos(pi r)) for r <= 1, r = |x - center| / radius (Eq. "cosine-bell" with
    amp = h_max / 2)."""
    r2 = np.zeros((mesh.E, mesh.np_))
    for a in range(mesh.d):
        r2 = r2 + ((mesh.x[a] - center[a]) / radius) ** 2
    r = np.sqrt(r2)
    return np.where(r <= 1.0, amp * (1.0 + np.cos(np.pi * r)), 0.0)


def upwind(cm, cp, un):
    """F* = u_n (C- + C+)/2 - |u_n| (C+ - C-)/2 (Rusanov for a scalar with continuous wind)."""
    return 0.5 * un * (cm + cp) - 0.5 * np.abs(un) * (cp - cm)


def coarse_gather(nodes):
    """G[c][i, j]: value at coarse face node i of the fine face c's polynomial with nodal
    values j (c = 0 lower half, 1 upper half); 1/2 weights at a node on the face midpoint."""
    G = []
    for c in (0, 1):
        x = 2.0 * nodes - (2 * c - 1)              # child coordinate of the coarse node
        L = bmod.lagrange_matrix(nodes, x)
        w = np.where(np.isclose(nodes, 0.0, atol=1e-15), 0.5,
                     np.where((nodes < 0.0) == (c == 0), 1.0, 0.0))
        G.append(w[:, None] * L)
    return G


def rhs(mesh, C, t, T, mode="mortar"):
    """dC/dt of the tracer dGSEM at time t; C [E, NP]."""
    if mesh.d != 2:
        raise ValueError("the tracer test is two-dimensional")
    B = mesh.basis
    w0 = B.weights[0]
    ux, uy = leveque_wind(mesh.x[0], mesh.x[1], t, T)
    U = (ux, uy)
    out = np.zeros_like(C)
    for a in range(2):
        out = out - (2.0 / mesh.h[:, a])[:, None] * mesh.apply_1d(B.D, C * U[a], a)
    conf, mort, bnd = mesh.forest.face_lists()

    def lift(e, a, s, Fs, Fown):
        idx = mesh.trace_index(a, s)
        sign = -1.0 if s == 1 else 1.0
        out[e, idx] += sign * (2.0 / mesh.h[e, a]) / w0 * (Fs - Fown)

    for (m, p, a) in conf:
        im, ip = mesh.trace_index(a, 1), mesh.trace_index(a, 0)
        un = U[a][m, im]
        Fs = upwind(C[m, im], C[p, ip], un)
        lift(m, a, 1, Fs, C[m, im] * un)
        lift(p, a, 0, Fs, C[p, ip] * U[a][p, ip])
    for (e, a, s) in bnd:
        idx = mesh.trace_index(a, s)
        lift(e, a, s, 0.0 * C[e, idx], C[e, idx] * U[a][e, idx])
    G = coarse_gather(B.nodes)
    for (ec, a, s, fines) in mort:
        t_ax = 1 - a                                 # the one tangential axis in 2D
        ic, ifn = mesh.trace_index(a, s), mesh.trace_index(a, 1 - s)
        cc = C[ec, ic]
        back = np.zeros_like(cc)
        gathered = np.zeros_like(cc)
        for f in fines:
            cf = mesh.forest.leaves[f][1][t_ax] & 1
            proj = B.P[cf] @ cc                      # coarse trace on the fine face nodes
            unf = U[a][f, ifn]
            Fs = upwind(proj, C[f, ifn], unf) if s == 1 else upwind(C[f, ifn], proj, unf)
            lift(f, a, 1 - s, Fs, C[f, ifn] * unf)
            back = back + B.C[cf] @ Fs
            gathered = gathered + G[cf] @ C[f, ifn]
        unc = U[a][ec, ic]
        if mode == "mortar":
            Fc = back
        elif mode == "interp":
            Fc = upwind(cc, gathered, unc) if s == 1 else upwind(gathered, cc, unc)
        else:
            raise ValueError("mode must be 'mortar' or 'interp'")
        lift(ec, a, s, Fc, cc * unc)
    return out


def ssprk3_step(mesh, C, t, dt, T, mode="mortar"):
    """One Shu-Osher SSP-RK3 step; the stages see the wind at t, t + dt and t + dt/2."""
    c1 = C + dt * rhs(mesh, C, t, T, mode)
    c2 = 0.75 * C + 0.25 * (c1 + dt * rhs(mesh, c1, t + dt, T, mode))
    return C / 3.0 + 2.0 / 3.0 * (c2 + dt * rhs(mesh, c2, t + 0.5 * dt, T, mode))


def indicator(mesh, C):
    """Refinement indicator: max over the element's nodes of |C|."""
    return np.max(np.abs(C), axis=1)


def total(mesh, C):
    """Total tracer sum w_i w_j |J| C, exactly rounded."""
    W = mesh.wnode[None, :] * mesh.J[:, None]
    return math.fsum((W * C).ravel())
