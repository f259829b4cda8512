"""Isentropic vortex (Sec. 4.1): an exact solution of the Euler equations, a vortex carried
unchanged by a uniform stream.  Test infrastructure, like the rest of ``oracle/``.

Nondimensional free stream rho = 1, theta = 1, p = 1 (p0 = R = theta0 = 1, g = 0, cp = 3.5 R so
that gamma = 1.4, the ratio of the constants used everywhere else).  The initial state adds to
the stream (U_inf, V_inf)

    (u', v') = beta / (2 pi) exp((1 - r^2) / 2) (-(y - y_c), x - x_c),
    T = 1 - (gamma - 1) beta^2 / (8 gamma pi^2) exp(1 - r^2),   rho = T^(1 / (gamma - 1)),

with p = rho^gamma (isentropic), so theta = T p^(-(gamma-1)/gamma) = 1 and Theta = rho.  Reading:
the paper prints the temperature perturbation as a potential-temperature one and the isentropic
relation garbled; this is the standard vortex those lines describe.  At time t the solution is the
initial one moved by (U_inf, V_inf) t; on a periodic box the displacement wraps around (nearest
image; the vortex's tails at half a box, 6 units, are below 1e-7).

Coordinates are the box's [0, L]: the paper's [-6, 6]^2 box is [0, 12]^2 with the centre at
(6, 6).  The state is returned in the library's perturbation variables about the uniform
background (rho_bar = Theta_bar = p_bar = 1).
"""
import math

import numpy as np

from . import physics


def constants():
    """The nondimensional constants of the vortex (gamma = 1.4)."""
    return physics.Constants(theta0=1.0, p0=1.0, g=0.0, R=1.0, cp=3.5)


def vortex_state(mesh, center, beta, uinf, t=0.0):
    """Perturbation state [4, E, NP] of the vortex moved to time t (2D mesh with constants())."""
    K = mesh.K
    g = K.gamma
    d = []
    for a in range(2):
        dx = mesh.x[a] - (center[a] + uinf[a] * t)
        if mesh.forest.periodic[a]:
            L = mesh.L[a]
            dx = np.mod(dx + 0.5 * L, L) - 0.5 * L
        d.append(dx)
    r2 = d[0] ** 2 + d[1] ** 2
    T = 1.0 - (g - 1.0) * beta ** 2 / (8.0 * g * math.pi ** 2) * np.exp(1.0 - r2)
    rho = T ** (1.0 / (g - 1.0))
    amp = beta / (2.0 * math.pi) * np.exp(0.5 * (1.0 - r2))
    u = uinf[0] - amp * d[1]
    v = uinf[1] + amp * d[0]
    rb, Tb, _ = mesh.bg
    q = np.empty((4, mesh.E, mesh.np_))
    q[0] = rho - rb
    q[1] = rho * u
    q[2] = rho * v
    q[3] = rho - Tb                   # Theta = rho theta with theta = 1
    return q


def l2_paper(q, q_exact):
    """The error norm of Sec. 4.1: (1 / N_dof) sqrt(sum over all DOF of |q - q_exact|^2), with
    N_dof counting the nodes times the prognostic variables."""
    e = np.asarray(q) - np.asarray(q_exact)
    return math.sqrt(float(np.sum(e * e))) / e.size
