"""Solution transfer on a cubed sphere (oracle; test infrastructure only).

Restates Sec. 3.4 (spherical geometry) and Appendix B of arXiv 2404.16648
for the transfer of nodal fields between parent and child elements on a curved surface:

* the cubed sphere: six tiles, each an equiangular gnomonic map of the square
  [-pi/4, pi/4]^2 onto the sphere of radius r; every element is an isoparametric curvilinear
  quadrilateral (its surface is interpolated by the degree-N basis through its LGL nodes);
* per-node metrics of the 2D surface: J = |x_xi x x_eta| with the tangent vectors from the
  collocation derivative of the node positions (the columns of the 3 x 2 Jacobian of App. B;
  |x_xi x x_eta| = sqrt(det(J^T J)), the measure behind its pseudo-inverse), and nodal weights
  W = w_i w_j J;
* element areas by the spherical excess r^2 (theta_1 + theta_2 + theta_3 - pi) of the two
  spherical triangles of the element's corners (great-circle edges), so the total area does
  not change under refinement;
* the reference-element projections (one set for all elements) with the paper's corrections:
  refinement interpolates the parent onto the children and then scales each field uniformly
  over the children so that its integral equals the parent's; coarsening weighs each child's
  projected contribution by its volume, sum_c (2^d V_c / sum V) R_c q_c (R_c the reference
  restriction, whose own weight is 1/2^d), and applies the same integral-matching scale.

Readings (where the section is not explicit; the library follows the same, written separately):
* tiles laid side by side in one forest of 6n x n roots, tile t = root column // n; the 2:1
  rule then acts across the seams of that layout (the transfer itself needs no neighbours);
* "a single scale factor ... applied uniformly to all fields": one factor per field per family,
  s = (integral before) / (integral after) with the isoparametric weights W of the old and new
  elements; it is applied only when the new integral is not the residue of cancellation,
  |I_new| > 1e-8 sum W |q_new| (else s = 1);
* coarsening also takes that scale: volume weighting alone is exactly conservative only when
  every element's Jacobian is constant, which isoparametric elements on a sphere are not;
* element volume V = the spherical-excess area of its corner quadrilateral, split along the
  diagonal from corner 0 to corner 2.

Pinned by tests/test_oracle_sphere.py (octant area 4 pi r^2 / 8, the Van Oosterom-Strackee
form of the excess, total area 4 pi r^2 at any refinement, spectral convergence of the
isoparametric metrics to the analytic gnomonic area element, conservation and the closed-form
action on constants through refinement and coarsening, reduction to the reference transfer for
equal volumes).
"""
import math

import numpy as np

from .basis import Basis

# tile t: the unnormalised point of the gnomonic map at X = tan(alpha), Y = tan(beta)
_TILES = (
    lambda X, Y: (np.ones_like(X), X, Y),
    lambda X, Y: (-X, np.ones_like(X), Y),
    lambda X, Y: (-np.ones_like(X), -X, Y),
    lambda X, Y: (X, -np.ones_like(X), Y),
    lambda X, Y: (-Y, X, np.ones_like(X)),
    lambda X, Y: (Y, X, -np.ones_like(X)),
)


def tile_point(t, alpha, beta, r):
    """Point on the sphere of radius r at equiangular coordinates (alpha, beta) of tile t."""
    X, Y = np.tan(alpha), np.tan(beta)
    p = np.stack(_TILES[t](X, Y), axis=-1)
    return r * p / np.linalg.norm(p, axis=-1, keepdims=True)


def spherical_excess(a, b, c, r):
    """Area r^2 (A + B + C - pi) of the spherical triangle abc (points on the sphere), with the
    internal angle at each vertex between the great circles to the other two."""
    a, b, c = (np.asarray(x, dtype=np.float64) / np.linalg.norm(x) for x in (a, b, c))

    def angle(p, q1, q2):
        t1 = q1 - np.dot(p, q1) * p
        t2 = q2 - np.dot(p, q2) * p
        return math.atan2(np.linalg.norm(np.cross(t1, t2)), np.dot(t1, t2))

    return r * r * (angle(a, b, c) + angle(b, c, a) + angle(c, a, b) - math.pi)


class SphereMesh:
    """Isoparametric degree-N elements of a cubed-sphere forest (base (6n, n), 2D)."""

    def __init__(self, forest, N, n, radius):
        assert forest.d == 2 and forest.base == (6 * n, n)
        self.forest, self.N, self.n, self.r = forest, int(N), int(n), float(radius)
        self.n1 = self.N + 1
        self.np_ = self.n1 ** 2
        self.basis = Basis(self.N)
        E = len(forest)
        xi = self.basis.nodes
        self.tile = np.empty(E, dtype=np.int64)
        self.alpha = np.empty((E, self.np_))
        self.beta = np.empty((E, self.np_))
        self.x = np.empty((E, self.np_, 3))
        self.corners = np.empty((E, 4, 3))
        i = np.arange(self.np_) % self.n1
        j = np.arange(self.np_) // self.n1
        quarter = math.pi / 4
        for e, (lev, (cx, cy)) in enumerate(forest.leaves):
            t = (cx >> lev) // n
            self.tile[e] = t
            s = 2.0 ** lev
            # root units along the layout: u in [t n, (t+1) n), v in [0, n)
            u = lambda z: (cx + (z + 1.0) / 2.0) / s - t * n   # noqa: E731
            v = lambda z: (cy + (z + 1.0) / 2.0) / s            # noqa: E731
            a = -quarter + (math.pi / 2) * u(xi[i]) / n
            b = -quarter + (math.pi / 2) * v(xi[j]) / n
            self.alpha[e], self.beta[e] = a, b
            self.x[e] = tile_point(t, a, b, self.r)
            ca = -quarter + (math.pi / 2) * np.array([u(-1.0), u(1.0), u(1.0), u(-1.0)]) / n
            cb = -quarter + (math.pi / 2) * np.array([v(-1.0), v(-1.0), v(1.0), v(1.0)]) / n
            self.corners[e] = tile_point(t, ca, cb, self.r)
        self._metrics()

    def _metrics(self):
        """Per-node surface Jacobian J = |x_xi x x_eta| of the interpolated surface, the nodal
        weights W = w_i w_j J, and each element's spherical-excess area."""
        n1, D, w = self.n1, self.basis.D, self.basis.weights
        X = self.x.reshape(len(self.forest), n1, n1, 3)        # [e, j, i, :]
        x_xi = np.einsum("im,ejmk->ejik", D, X)
        x_eta = np.einsum("jm,emik->ejik", D, X)
        self.J = np.linalg.norm(np.cross(x_xi, x_eta), axis=-1).reshape(len(self.forest), self.np_)
        ww = np.outer(w, w).reshape(-1)                        # (j, i) order = node n = i + n1 j
        self.W = ww[None, :] * self.J
        self.area = np.array([spherical_excess(c[0], c[1], c[2], self.r) + spherical_excess(c[0], c[2], c[3], self.r)
                              for c in self.corners])

    def apply_1d(self, A, X, axis):
        """(n1 x n1) matrix A along element axis `axis` of X [..., NP] (node n = i + n1 j)."""
        n1 = self.n1
        Xs = X.reshape(X.shape[:-1] + (n1, n1))
        dim = Xs.ndim - 1 - axis
        Y = np.moveaxis(np.tensordot(A, Xs, axes=([1], [dim])), 0, dim)
        return Y.reshape(X.shape)

    def integrals(self, q):
        """sum over nodes of W q per field (q: [nv, E, NP])."""
        return np.einsum("en,ven->v", self.W, q)


def _scale(q_new, W_new, I_old):
    """The integral-matching factor of each field over a set of new elements."""
    I_new = np.einsum("en,ven->v", W_new, q_new)
    mag = np.einsum("en,ven->v", W_new, np.abs(q_new))
    s = np.ones_like(I_new)
    ok = np.abs(I_new) > 1e-8 * mag
    s[ok] = I_old[ok] / I_new[ok]
    return s


def transfer(q_old, m_old, m_new, tmap, volume_weights=True):
    """Cubed-sphere transfer after a regrid (tmap entries as Forest.regrid returns them).

    keep: copy.  Children of an old parent: reference interpolation P_c, then one scale factor
    per field over the family.  New parent of old children: sum_c (4 V_c / sum V) R_c q_c
    (volume_weights=False: the reference weights), then one scale factor per field."""
    B = m_old.basis
    nv = q_old.shape[0]
    q_new = np.empty((nv, len(m_new.forest), m_new.np_))
    families = {}
    for k, entry in enumerate(tmap):
        if entry[0] == "child":
            families.setdefault(entry[1], []).append((k, entry[2]))
    for k, entry in enumerate(tmap):
        if entry[0] == "keep":
            q_new[:, k] = q_old[:, entry[1]]
        elif entry[0] == "parent":
            olds = list(entry[1])
            V = m_old.area[olds]
            acc = np.zeros((nv, m_new.np_))
            for ci, e in enumerate(olds):
                v = q_old[:, e]
                for a in range(2):
                    v = m_old.apply_1d(B.C[(ci >> a) & 1], v, a)
                wgt = 4.0 * V[ci] / V.sum() if volume_weights else 1.0
                acc = acc + wgt * v
            I_old = np.einsum("en,ven->v", m_old.W[olds], q_old[:, olds])
            s = _scale(acc[:, None, :], m_new.W[[k]], I_old)
            q_new[:, k] = acc * s[:, None]
    for e, kids in families.items():
        ks = [k for k, _ in kids]
        for k, ci in kids:
            v = q_old[:, e]
            for a in range(2):
                v = m_old.apply_1d(B.P[(ci >> a) & 1], v, a)
            q_new[:, k] = v
        I_old = np.einsum("n,vn->v", m_old.W[e], q_old[:, e])
        s = _scale(q_new[:, ks], m_new.W[ks], I_old)
        q_new[:, ks] *= s[:, None, None]
    return q_new
