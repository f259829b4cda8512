"""Strong-form nodal dGSEM on a 2:1-balanced forest (oracle; test infrastructure only).

Restates arXiv 2404.16648 in plain FP64 numpy:

* strong form (v, dq/dt) + <v n, F* - F> + (v, div F) = (v, S) with LGL collocation and the
  diagonal LGL mass matrix (Sec. 2.2, strong form); on an axis-aligned box the volume term is
  (2/h_a) sum_m D_im F_a(.., m, ..) per axis and the face term lifts (F* - F).n at each face node
  with weight 1 / (w_0 h_a / 2);
* Rusanov numerical flux (Sec. 2.2) -- see ``physics.rusanov``;
* mortar method on hanging faces (Sec. 3.3): the coarse trace is projected to each mortar with
  P = M^{-1} S, the fine side is the mortar itself (identity), the Riemann problem is solved on
  the mortar, and the mortar fluxes return to the coarse face as sum_i s M^{-1} S^T F*_i with
  s = 1/2 per tangential axis;
* explicit time stepping with one uniform dt (Sec. 3.1); SSP-RK3 in Shu-Osher form;
* conservative solution transfer: parent -> child by P_c per axis, children -> parent by
  sum_c C_c per axis (Sec. 3.3, "Solution transfer");
* mass / energy diagnostics (Sec. 4.3 and 4.4 report mass and energy loss).

Readings: the projected coarse state on a mortar is completed with the fine side's background
(the background is a function of z, and the mortar points are the fine face's points); the
initial bubble keeps the pressure hydrostatic (Theta' = 0, rho' = -rho_bar theta'/(theta0 +
theta')), the reading taken here of the balanced initial conditions of Sec. 4.3.

Node numbering inside an element: i_0 + (N+1) i_1 + (N+1)^2 i_2 (axis 0 fastest); the state is
an array [nv, E, (N+1)^d].  Pinned by tests/test_oracle_dg.py (rest state, free stream with
hanging faces, discrete conservation, convergence order, symmetry, RK3 stability polynomial,
refine/coarsen identity and conservation).
"""
import math

import numpy as np

from . import physics
from .basis import Basis
from .forest import Forest


class Mesh:
    """Forest + degree-N basis + box geometry [0, L_0] x ... x [0, L_{d-1}]."""

    def __init__(self, forest, N, lengths, K=None):
        self.forest = forest
        self.d = forest.d
        self.N = int(N)
        self.n1 = self.N + 1
        self.np_ = self.n1 ** self.d
        self.nv = self.d + 2
        self.L = tuple(float(x) for x in lengths)
        self.K = K if K is not None else physics.Constants()
        self.basis = Basis(self.N)
        self._geometry()

    @property
    def E(self):
        return len(self.forest)

    def _geometry(self):
        d, n1 = self.d, self.n1
        E = self.E
        lev = np.array([lf[0] for lf in self.forest.leaves], dtype=np.int64)
        crd = np.array([lf[1] for lf in self.forest.leaves], dtype=np.float64).reshape(E, d)
        root_h = np.array([self.L[a] / self.forest.base[a] for a in range(d)])
        # h = (L/base) / 2^level: power-of-two scaling is exact
        self.h = root_h[None, :] / (2.0 ** lev)[:, None]
        self.level = lev
        xi = self.basis.nodes
        # node coordinate x_a = (c_a + (xi+1)/2) h_a: faces shared by two elements get
        # bit-identical coordinates
        self.x = np.empty((d, E, self.np_))
        idx = np.arange(self.np_)
        for a in range(d):
            ia = (idx // (n1 ** a)) % n1
            self.x[a] = (crd[:, a:a + 1] + (xi[ia][None, :] + 1.0) / 2.0) * self.h[:, a:a + 1]
        z = self.x[d - 1]
        self.bg = physics.background(z, self.K)            # each [E, NP]
        self.J = np.prod(self.h / 2.0, axis=1)             # volume Jacobian per element
        w = self.basis.weights
        wn = np.ones(self.np_)
        for a in range(d):
            wn = wn * w[(idx // (n1 ** a)) % n1]
        self.wnode = wn

    # -- shaped views ------------------------------------------------------------------
    def shaped(self, arr):
        """[..., NP] -> [..., n1 (axis d-1), ..., n1 (axis 0)]."""
        return arr.reshape(arr.shape[:-1] + (self.n1,) * self.d)

    def dim_of_axis(self, arr_nd, axis):
        return arr_nd - 1 - axis

    def apply_1d(self, A, X, axis):
        """Apply the (n1 x n1) matrix A along element axis ``axis`` of X [..., NP]."""
        Xs = self.shaped(X)
        dim = Xs.ndim - 1 - axis
        Y = np.moveaxis(np.tensordot(A, Xs, axes=([1], [dim])), 0, dim)
        return Y.reshape(X.shape)

    def trace(self, X, axis, side):
        """Face trace of X [..., NP] on face (axis, side); remaining axes keep their order."""
        Xs = self.shaped(X)
        dim = Xs.ndim - 1 - axis
        sl = [slice(None)] * Xs.ndim
        sl[dim] = self.N if side == 1 else 0
        T = Xs[tuple(sl)]
        return T.reshape(X.shape[:-1] + (self.n1 ** (self.d - 1),))

    def trace_index(self, axis, side):
        """Element-node indices of face (axis, side), in trace order."""
        return self.trace(np.arange(self.np_), axis, side)

    def apply_face_1d(self, A, T, t):
        """Apply A along the t-th tangential axis of a face trace T [..., n1^(d-1)]."""
        shp = T.shape[:-1] + (self.n1,) * (self.d - 1)
        Ts = T.reshape(shp)
        dim = Ts.ndim - 1 - t
        Y = np.moveaxis(np.tensordot(A, Ts, axes=([1], [dim])), 0, dim)
        return Y.reshape(T.shape)


def _bg_at(mesh, elems, idx=None):
    rb, Tb, pb = mesh.bg
    if idx is None:
        return rb[elems], Tb[elems], pb[elems]
    return rb[elems][:, idx], Tb[elems][:, idx], pb[elems][:, idx]


def rhs(mesh, q, elems=None):
    """dq/dt of the strong-form dGSEM (Sec. 2.2) with mortars on hanging faces (Sec. 3.3).

    q: [nv, E, NP].  With ``elems`` (sorted array of element ids) only those elements'
    tendencies are computed (the others are returned as NaN); every face touching them is
    still evaluated in full.
    """
    K = mesh.K
    d, nv, E = mesh.d, mesh.nv, mesh.E
    w0 = mesh.basis.weights[0]
    out = np.full_like(q, np.nan)
    if elems is None:
        elems = np.arange(E)
    elems = np.asarray(elems, dtype=np.int64)
    want = np.zeros(E, dtype=bool)
    want[elems] = True

    # volume term: -(sum_a (2/h_a) D_a F_a) + S
    qe = q[:, elems]
    bge = _bg_at(mesh, elems)
    acc = physics.source(qe, K)
    for a in range(d):
        Fa = physics.flux(qe, bge, K, a)
        dF = mesh.apply_1d(mesh.basis.D, Fa, a)
        acc = acc - (2.0 / mesh.h[elems, a])[None, :, None] * dF
    out[:, elems] = acc

    conf, mort, bnd = mesh.forest.face_lists()

    def lift(e_list, axis, side, Fs, Fown):
        # outward normal +e_axis on side 1, -e_axis on side 0
        idx = mesh.trace_index(axis, side)
        coef = (2.0 / mesh.h[e_list, axis]) / w0
        sign = -1.0 if side == 1 else 1.0
        for k, e in enumerate(e_list):
            if want[e]:
                out[:, e, idx] += sign * coef[k] * (Fs[:, k] - Fown[:, k])

    # conforming faces, grouped by axis
    for a in range(d):
        faces = [(m, p) for (m, p, ax) in conf if ax == a and (want[m] or want[p])]
        if not faces:
            continue
        em = np.array([f[0] for f in faces])
        ep = np.array([f[1] for f in faces])
        im = mesh.trace_index(a, 1)
        ip = mesh.trace_index(a, 0)
        qm = q[:, em][:, :, im]
        qp = q[:, ep][:, :, ip]
        Fs, Fm, Fp = physics.rusanov(qm, qp, _bg_at(mesh, em, im), _bg_at(mesh, ep, ip), K, a)
        lift(em, a, 1, Fs, Fm)
        lift(ep, a, 0, Fs, Fp)

    # no-flux walls: mirror state on the outside
    for a in range(d):
        for s in (0, 1):
            es = np.array([e for (e, ax, sd) in bnd if ax == a and sd == s and want[e]])
            if len(es) == 0:
                continue
            idx = mesh.trace_index(a, s)
            qi = q[:, es][:, :, idx]
            bgi = _bg_at(mesh, es, idx)
            qg = physics.wall_mirror(qi, a)
            if s == 1:
                Fs, Fown, _ = physics.rusanov(qi, qg, bgi, bgi, K, a)
            else:
                Fs, _, Fown = physics.rusanov(qg, qi, bgi, bgi, K, a)
            lift(es, a, s, Fs, Fown)

    # hanging faces: mortar method (Sec. 3.3)
    B = mesh.basis
    for (ec, a, s, fines) in mort:
        if not (want[ec] or any(want[f] for f in fines)):
            continue
        tang = [t for t in range(d) if t != a]
        ic = mesh.trace_index(a, s)
        ifn = mesh.trace_index(a, 1 - s)
        qc = q[:, ec, ic]                                   # coarse trace [nv, n1^(d-1)]
        Fc_own = physics.flux(q[:, ec:ec + 1, ic], _bg_at(mesh, [ec], ic), K, a)[:, 0]
        Ftilde = np.zeros_like(qc)
        for f in fines:
            cf = mesh.forest.leaves[f][1]
            qproj = qc
            for t_i, t in enumerate(tang):
                qproj = mesh.apply_face_1d(B.P[cf[t] & 1], qproj, t_i)
            qf = q[:, f, ifn]
            bgf = _bg_at(mesh, [f], ifn)
            bgf = (bgf[0][0], bgf[1][0], bgf[2][0])
            if s == 1:   # coarse element is on the low side
                Fs, Fcm, Ffp = physics.rusanov(qproj, qf, bgf, bgf, K, a)
                Ff_own = Ffp
            else:
                Fs, Ffm, Fcp = physics.rusanov(qf, qproj, bgf, bgf, K, a)
                Ff_own = Ffm
            if want[f]:
                coef = (2.0 / mesh.h[f, a]) / w0
                sign = 1.0 if s == 1 else -1.0    # fine side's outward normal is opposite
                out[:, f, ifn] += sign * coef * (Fs - Ff_own)
            back = Fs
            for t_i, t in enumerate(tang):
                back = mesh.apply_face_1d(B.C[cf[t] & 1], back, t_i)
            Ftilde = Ftilde + back
        if want[ec]:
            coef = (2.0 / mesh.h[ec, a]) / w0
            sign = -1.0 if s == 1 else 1.0
            out[:, ec, ic] += sign * coef * (Ftilde - Fc_own)
    return out


def viscous_primitives(mesh, q):
    """phi = (u_0, .., u_{d-1}, theta') with theta' = (Theta' - theta0 rho') / rho, the exact
    rewriting of (Theta_bar + Theta')/(rho_bar + rho') - theta0 for Theta_bar = rho_bar theta0."""
    d = mesh.d
    rb, _, _ = mesh.bg
    rho = rb + q[0]
    phi = np.empty((d + 1,) + q.shape[1:], dtype=q.dtype)
    phi[:d] = q[1:1 + d] / rho
    phi[d] = (q[1 + d] - mesh.K.theta0 * q[0]) / rho
    return phi, rho


def _central_face_pass(mesh, X, conf, mort, bnd, out, scale_wall):
    """Adds the strong-form lift of central face values to out[..., a, :]:
    out_a += n_a (2/h_a)/w0 (X* - X_own) at face nodes, X* = (X- + X+)/2 on conforming faces and
    mortars (coarse values projected with P, results returned with sum_m C F*_m); on walls
    X* = X_own when scale_wall is None, else X* = 0 (no flux through the wall).
    X: [ncomp, d, E, NP] (the a-th component is the one used on faces of axis a)."""
    d = mesh.d
    w0 = mesh.basis.weights[0]
    B = mesh.basis

    def lift(e, a, s, Xs, Xo):
        idx = mesh.trace_index(a, s)
        n_a = 1.0 if s == 1 else -1.0
        out[:, a, e, idx] += n_a * (2.0 / mesh.h[e, a]) / w0 * (Xs - Xo)

    for (m, p, a) in conf:
        xm = X[:, a, m][:, mesh.trace_index(a, 1)]
        xp = X[:, a, p][:, mesh.trace_index(a, 0)]
        xs = 0.5 * (xm + xp)
        lift(m, a, 1, xs, xm)
        lift(p, a, 0, xs, xp)
    if scale_wall is not None:
        for (e, a, s) in bnd:
            xo = X[:, a, e][:, mesh.trace_index(a, s)]
            lift(e, a, s, 0.0 * xo, xo)
    for (ec, a, s, fines) in mort:
        tang = [t for t in range(d) if t != a]
        xc = X[:, a, ec][:, mesh.trace_index(a, s)]
        acc = np.zeros_like(xc)
        for f in fines:
            cf = mesh.forest.leaves[f][1]
            xproj = xc
            for t_i, t in enumerate(tang):
                xproj = mesh.apply_face_1d(B.P[cf[t] & 1], xproj, t_i)
            xf = X[:, a, f][:, mesh.trace_index(a, 1 - s)]
            xs = 0.5 * (xproj + xf)
            lift(f, a, 1 - s, xs, xf)
            back = xs
            for t_i, t in enumerate(tang):
                back = mesh.apply_face_1d(B.C[cf[t] & 1], back, t_i)
            acc = acc + back
        lift(ec, a, s, acc, xc)


def viscous_rhs(mesh, q, nu):
    """Viscous tendency nabla . (nu rho nabla phi) on momentum and Theta' by BR1 (Bassi & Rebay
    1997): pass 1 the DG gradient sigma of phi with central face values, pass 2 the strong-form
    divergence of G = nu rho sigma with central fluxes; no viscous flux through walls.  The paper
    names an artificial viscosity mu (Sec. 4.3) without its operator; this is the reading used."""
    d = mesh.d
    conf, mort, bnd = mesh.forest.face_lists()
    phi, rho = viscous_primitives(mesh, q)
    # pass 1: sigma[c, a] = d phi_c / d x_a
    sigma = np.empty((d + 1, d) + q.shape[1:], dtype=q.dtype)
    for a in range(d):
        sigma[:, a] = (2.0 / mesh.h[:, a])[None, :, None] * mesh.apply_1d(mesh.basis.D, phi, a)
    X = np.broadcast_to(phi[:, None], sigma.shape).copy()
    _central_face_pass(mesh, X, conf, mort, bnd, sigma, None)
    # pass 2: V_c = sum_a d/dx_a (nu rho sigma[c, a])
    G = nu * rho[None, None] * sigma
    div = np.zeros_like(G)
    for a in range(d):
        div[:, a] = (2.0 / mesh.h[:, a])[None, :, None] * mesh.apply_1d(mesh.basis.D, G[:, a], a)
    _central_face_pass(mesh, G, conf, mort, bnd, div, 0.0)
    V = np.zeros_like(q)
    V[1:2 + d] = div.sum(axis=1)
    return V


def ssprk3_step(q, dt, L):
    """One SSP-RK3 step (Shu-Osher form) of dq/dt = L(q)."""
    q1 = q + dt * L(q)
    q2 = 0.75 * q + 0.25 * (q1 + dt * L(q1))
    return (1.0 / 3.0) * q + (2.0 / 3.0) * (q2 + dt * L(q2))


def step(mesh, q, dt, nsteps=1, nu=0.0):
    L = (lambda s: rhs(mesh, s)) if nu == 0.0 else (lambda s: rhs(mesh, s) + viscous_rhs(mesh, s, nu))
    for _ in range(nsteps):
        q = ssprk3_step(q, dt, L)
    return q


def step_on(mesh, q, dt, elems):
    """One SSP-RK3 step (Shu-Osher form, as ssprk3_step) evaluated only where it is needed for
    the elements ``elems``: the tendency of stage s at an element reads its face neighbours'
    stage-s state, so stage 1 is taken on the elements within two face hops of ``elems``,
    stage 2 within one hop and stage 3 on ``elems`` alone.  Returns the new state there (other
    elements are NaN).  The same arithmetic as step(); for sampled checks on large meshes."""
    hop1 = set(int(e) for e in elems)
    for e in list(hop1):
        hop1 |= set(mesh.forest.face_neighbors(e))
    hop2 = set(hop1)
    for e in list(hop1):
        hop2 |= set(mesh.forest.face_neighbors(e))
    s0, s1, s2 = (np.array(sorted(x), dtype=np.int64) for x in (elems, hop1, hop2))
    q1 = q.copy()
    q1[:, s2] = q[:, s2] + dt * rhs(mesh, q, elems=s2)[:, s2]
    q2 = q.copy()
    q2[:, s1] = 0.75 * q[:, s1] + 0.25 * (q1[:, s1] + dt * rhs(mesh, q1, elems=s1)[:, s1])
    out = np.full_like(q, np.nan)
    out[:, s0] = (1.0 / 3.0) * q[:, s0] + (2.0 / 3.0) * (q2[:, s0] + dt * rhs(mesh, q2, elems=s0)[:, s0])
    return out


def transfer(q_old, mesh_old, mesh_new, tmap):
    """Conservative L2 solution transfer after a regrid (Sec. 3.3).

    child:  q_c = (P_{c_0} x P_{c_1} (x P_{c_2})) q_parent (exact interpolation);
    parent: q_p = sum_c (C_{c_0} x ...) q_c with C_c = (1/2) M^{-1} S_c^T per axis.
    """
    d = mesh_old.d
    B = mesh_old.basis
    q_new = np.empty((q_old.shape[0], mesh_new.E, q_old.shape[2]))
    for k, entry in enumerate(tmap):
        if entry[0] == "keep":
            q_new[:, k] = q_old[:, entry[1]]
        elif entry[0] == "child":
            _, e, ci = entry
            v = q_old[:, e]
            for a in range(d):
                v = mesh_old.apply_1d(B.P[(ci >> a) & 1], v, a)
            q_new[:, k] = v
        else:
            acc = np.zeros_like(q_old[:, 0])
            for ci, e in enumerate(entry[1]):
                v = q_old[:, e]
                for a in range(d):
                    v = mesh_old.apply_1d(B.C[(ci >> a) & 1], v, a)
                acc = acc + v
            q_new[:, k] = acc
    return q_new


def theta_prime(mesh, q):
    """theta' = (Theta_bar + Theta') / (rho_bar + rho') - theta0 at every node."""
    rb, Tb, _ = mesh.bg
    return (Tb + q[mesh.d + 1]) / (rb + q[0]) - mesh.K.theta0


def indicator(mesh, q):
    """Refinement indicator: max over element nodes of |theta'| (Sec. 4.3 tags by theta)."""
    return np.max(np.abs(theta_prime(mesh, q)), axis=1)


def integrals(mesh, q):
    """[mass, total energy, kinetic energy, volume, perturbation mass] (exactly rounded sums).

    Weights w_i w_j (w_k) |J|; E = p cv/R + |U|^2/(2 rho) + rho g z.
    """
    K = mesh.K
    d = mesh.d
    rb, Tb, pb = mesh.bg
    rho = rb + q[0]
    ke = 0.5 * np.sum(q[1:1 + d] ** 2, axis=0) / rho
    pp = physics.pressure_perturbation(q[1 + d], Tb, pb, K)
    p = pb + pp
    en = p * K.cv / K.R + ke + rho * K.g * mesh.x[d - 1]
    W = mesh.wnode[None, :] * mesh.J[:, None]
    return np.array([math.fsum((W * rho).ravel()), math.fsum((W * en).ravel()),
                     math.fsum((W * ke).ravel()), math.fsum(W.ravel()),
                     math.fsum((W * q[0]).ravel())])


def bubble_theta(mesh, center, radius, amp):
    """Cosine bell theta' = amp (1 + cos(pi r)) for r <= 1, r = |(x - c) / radius| (Sec. 4.2, 4.3)."""
    r2 = np.zeros((mesh.E, mesh.np_))
    for a in range(mesh.d):
        r2 = r2 + ((mesh.x[a] - center[a]) / radius[a]) ** 2
    r = np.sqrt(r2)
    return np.where(r <= 1.0, amp * (1.0 + np.cos(np.pi * r)), 0.0)


def rff_theta(mesh, sigma, kvec, phase):
    """Random Fourier-feature field sigma sqrt(2/K) sum_k cos(k.x + phi_k) (inputs drawn outside).

    With k ~ N(0, l^-2 I) and phi ~ U[0, 2 pi) its covariance over draws is
    sigma^2 exp(-r^2 / (2 l^2)) (Rahimi & Recht 2007); tests/test_oracle_rff.py pins the plane
    wave of one feature and that covariance at lags 0, l and 2 l."""
    kvec = np.asarray(kvec, dtype=np.float64)
    phase = np.asarray(phase, dtype=np.float64)
    nfeat = len(phase)
    acc = np.zeros((mesh.E, mesh.np_))
    for m in range(nfeat):
        arg = phase[m]
        for a in range(mesh.d):
            arg = arg + kvec[m, a] * mesh.x[a]
        acc = acc + np.cos(arg)
    return sigma * math.sqrt(2.0 / nfeat) * acc


def state_from_theta(mesh, th):
    """Hydrostatic-pressure initial state for a theta' field: Theta' = 0, U = 0,
    rho' = -rho_bar theta' / (theta0 + theta'): the pressure stays hydrostatic, which is how the
    paper's balanced initial conditions (Sec. 4.3) are read here."""
    rb, _, _ = mesh.bg
    q = np.zeros((mesh.nv, mesh.E, mesh.np_), dtype=np.result_type(th, np.float64))
    q[0] = -rb * th / (mesh.K.theta0 + th)
    return q


def adapt_initial(forest, N, lengths, theta_fn, thr, B, K=None):
    """Adapt a forest max_level times on the analytic initial condition, re-evaluated on each
    new mesh (not projected); returns the final Mesh."""
    mesh = Mesh(forest, N, lengths, K)
    for _ in range(forest.max_level):
        q = state_from_theta(mesh, theta_fn(mesh))
        tag = indicator(mesh, q) > thr
        forest, _ = mesh.forest.regrid(tag, B)
        mesh = Mesh(forest, N, lengths, K)
    return mesh
