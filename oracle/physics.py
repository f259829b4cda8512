"""Compressible Euler physics in perturbation form (oracle; test infrastructure only).

Restates arXiv 2404.16648:

* the flux vector F(q) = (U, U(x)U/rho + P I, Theta U/rho) and source S = (0, F, 0)
  (Sec. 2.1, Eq. 1 and Eq. "eulervector"), with the body force F reduced to buoyancy
  about the hydrostatic background (no Coriolis: none of the box tests uses it);
* the equation of state P = P0 (R Theta / P0)^gamma with R = cp - cv, gamma = cp/cv
  (Sec. 2.1, equation of state);
* the split rho = rho_bar(z) + rho', P = P_bar(z) + P' (Sec. 2.1);
* the hydrostatic neutral background p = p0 (1 - g z / (cp theta0))^(cp/R) (Sec. 4.3,
  rising thermal bubble);
* the Rusanov flux F* = {F} + n (|c|/2) [[q]] (Sec. 2.2).

Readings (the paper is silent on these):
* constants R = 287, cp = 1004.5, cv = 717.5, g = 9.81, p0 = 1e5, theta0 = 300;
* P_bar is defined nodewise as P(Theta_bar), so a fluid at rest has P' = 0 exactly;
* P' = P(Theta_bar + Theta') - P(Theta_bar) is evaluated through the exact identity
  P' = P_bar [(1 + Theta'/Theta_bar)^gamma - 1] = P_bar expm1(gamma log1p(Theta'/Theta_bar)),
  which avoids the cancellation of two ~1e5 Pa numbers;
* Rusanov wave speed lambda = max(|u_n^-| + c^-, |u_n^+| + c^+) with c = sqrt(gamma P / rho)
  of the total state; the jump acts on the perturbation variables (the background is
  continuous across faces);
* no-flux walls use a mirror state (normal momentum negated).

Variable order in a state vector: [rho', U_0, ..., U_{d-1}, Theta'] where axis d-1 is
vertical (z).  Pinned by tests/test_oracle_physics.py.
"""
import numpy as np


class Constants:
    """Physical constants (reading of the paper: it gives none)."""

    def __init__(self, theta0=300.0, p0=1.0e5, g=9.81, R=287.0, cp=1004.5):
        self.theta0 = float(theta0)
        self.p0 = float(p0)
        self.g = float(g)
        self.R = float(R)
        self.cp = float(cp)
        self.cv = self.cp - self.R
        self.gamma = self.cp / self.cv


def exner(z, K):
    """pi(z) = 1 - g z / (cp theta0) of the neutral atmosphere (Sec. 4.3)."""
    return 1.0 - K.g * np.asarray(z) / (K.cp * K.theta0)


def hydrostatic_pressure(z, K):
    """Closed form p = p0 pi^(cp/R) (Sec. 4.3)."""
    return K.p0 * exner(z, K) ** (K.cp / K.R)


def background_density(z, K):
    """rho_bar = p / (R T) with T = theta0 pi, i.e. p0 pi^(cv/R) / (R theta0)."""
    return K.p0 * exner(z, K) ** (K.cv / K.R) / (K.R * K.theta0)


def eos_pressure(Theta, K):
    """P = P0 (R Theta / P0)^gamma (Sec. 2.1)."""
    return K.p0 * (K.R * np.asarray(Theta) / K.p0) ** K.gamma


def background(z, K):
    """(rho_bar, Theta_bar, p_bar) at heights z; p_bar := P(Theta_bar), so that P' is exactly 0
    at rest (the discrete hydrostatic balance as read here; the paper does not define it)."""
    rb = background_density(z, K)
    Tb = rb * K.theta0
    pb = eos_pressure(Tb, K)
    return rb, Tb, pb


def pressure_perturbation(Theta_p, Theta_b, p_b, K):
    """P' = P(Theta_bar + Theta') - P(Theta_bar), via p_bar expm1(gamma log1p(Theta'/Theta_bar))."""
    return p_b * np.expm1(K.gamma * np.log1p(Theta_p / Theta_b))


def sound_speed(P, rho, K):
    """c = sqrt(gamma P / rho) (Sec. 4.4 quotes 347.3 m/s for the surface state)."""
    return np.sqrt(K.gamma * P / rho)


def primitives(q, bg, K):
    """Total density, velocity, total Theta, pressure perturbation, total pressure.

    q: array [nv, ...] of perturbation variables; bg: (rho_bar, Theta_bar, p_bar) broadcastable.
    """
    d = q.shape[0] - 2
    rb, Tb, pb = bg
    rho = rb + q[0]
    u = q[1:1 + d] / rho
    Theta = Tb + q[1 + d]
    pp = pressure_perturbation(q[1 + d], Tb, pb, K)
    return rho, u, Theta, pp, pb + pp


def flux(q, bg, K, axis):
    """Component ``axis`` of F(q) for every variable (Sec. 2.1, Eq. "eulervector").

    rho':  U_a;  U_b:  U_b u_a + P' delta_ab;  Theta':  Theta u_a (total Theta).
    """
    d = q.shape[0] - 2
    rho, u, Theta, pp, _ = primitives(q, bg, K)
    F = np.empty_like(q)
    F[0] = q[1 + axis]
    for b in range(d):
        F[1 + b] = q[1 + b] * u[axis]
        if b == axis:
            F[1 + b] = F[1 + b] + pp
    F[1 + d] = Theta * u[axis]
    return F


def source(q, K):
    """S = (0, F, 0) with F = -rho' g z_hat (buoyancy about the hydrostatic background)."""
    d = q.shape[0] - 2
    S = np.zeros_like(q)
    S[d] = -q[0] * K.g          # vertical momentum is U_{d-1}, stored at index d
    return S


def abs_cs(x):
    """|x|; on complex input (complex-step differentiation) sign(Re x) x with sign(0) = 0, the
    derivative a central finite difference sees at 0.  Same values as np.abs on real input."""
    x = np.asarray(x)
    if np.iscomplexobj(x):
        r = x.real
        return np.where(r > 0, x, np.where(r < 0, -x, r + 0j))
    return np.abs(x)


def max_cs(a, b):
    """max(a, b); on complex input chosen by the real part, ties to a (the low side)."""
    if np.iscomplexobj(a) or np.iscomplexobj(b):
        return np.where(np.real(a) >= np.real(b), a, b)
    return np.maximum(a, b)


def rusanov(qm, qp, bgm, bgp, K, axis):
    """Rusanov flux along +axis between the low-side state qm and high-side state qp.

    F* = (F(qm) + F(qp))/2 - lambda/2 (qp - qm), lambda = max(|u_a| + c) over both sides.
    Returns (F*, F(qm), F(qp)).
    """
    d = qm.shape[0] - 2
    Fm = flux(qm, bgm, K, axis)
    Fp = flux(qp, bgp, K, axis)
    rm, um, _, _, Pm = primitives(qm, bgm, K)
    rp, up, _, _, Pp = primitives(qp, bgp, K)
    lam = max_cs(abs_cs(um[axis]) + sound_speed(Pm, rm, K),
                 abs_cs(up[axis]) + sound_speed(Pp, rp, K))
    Fs = 0.5 * (Fm + Fp) - 0.5 * lam * (qp - qm)
    return Fs, Fm, Fp


def wall_mirror(q, axis):
    """Ghost state of a no-flux wall: normal momentum negated, everything else copied."""
    g = q.copy()
    g[1 + axis] = -q[1 + axis]
    return g
