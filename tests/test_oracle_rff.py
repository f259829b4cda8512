"""Pins of the oracle's random Fourier-feature field (dg.rff_theta), the Gaussian random theta'
of the adjoint workload: sigma sqrt(2/K) sum_m cos(k_m . x + phi_m) with k ~ N(0, l^-2 I) and
phi ~ U[0, 2 pi) (Rahimi & Recht 2007).

What the mathematics fixes, independent of how the sum is written:
- one feature is a plane wave of amplitude sigma sqrt(2): its value at the origin, its period
  along k and its invariance across k;
- over independent draws the field has mean 0 and covariance E[f(x) f(y)] = sigma^2
  exp(-|x - y|^2 / (2 l^2)) at every x (Bochner: the Gaussian spectrum of k gives the Gaussian
  kernel, the uniform phase makes the field stationary).  The draws come from workloads.rff_draws,
  so the pin covers the pair the adjoint workload uses.
"""
import math

import numpy as np

import workloads
from oracle import dg


class _Points:
    """The attributes rff_theta reads from a mesh, for an arbitrary list of points."""

    def __init__(self, pts):
        pts = np.asarray(pts, dtype=np.float64)
        self.d = pts.shape[1]
        self.E, self.np_ = 1, pts.shape[0]
        self.x = [pts[:, a].reshape(1, -1) for a in range(self.d)]


def test_single_feature_is_a_plane_wave():
    sigma, lam = 0.05, 700.0
    n = np.array([3.0, 4.0, 12.0]) / 13.0
    k = (2 * math.pi / lam) * n
    phase = math.pi / 3
    rng = np.random.default_rng(0)
    base = rng.uniform(0.0, 5000.0, (20, 3))
    t = np.cross(n, [1.0, 0.0, 0.0])
    t /= np.linalg.norm(t)
    pts = np.concatenate([[[0.0, 0.0, 0.0]], base, base + lam * n, base + 900.0 * t])
    f = dg.rff_theta(_Points(pts), sigma, k[None, :], [phase]).ravel()
    assert abs(f[0] - sigma * math.sqrt(2.0) * 0.5) <= 1e-15
    b = f[1:21]
    np.testing.assert_allclose(f[21:41], b, rtol=0, atol=1e-12)   # one wavelength along k
    np.testing.assert_allclose(f[41:61], b, rtol=0, atol=1e-12)   # across k
    assert np.abs(f).max() <= sigma * math.sqrt(2.0) * (1 + 1e-15)


def test_gaussian_covariance_over_draws():
    sigma, ell, K = 0.05, 300.0, 512
    rng = np.random.default_rng(1)
    P = 48
    far = rng.uniform(2000.0, 8000.0, (P, 3))
    near = rng.uniform(-0.2 * ell, 0.2 * ell, (16, 3))    # near the origin: catches a lost phase
    u = rng.standard_normal((P, 3))
    u /= np.linalg.norm(u, axis=1, keepdims=True)
    lags = (0.0, ell, 2.0 * ell)
    pts = np.concatenate([far] + [far + r * u for r in lags[1:]] + [near])
    M = 300
    F = np.empty((M, pts.shape[0]))
    for s in range(M):
        sg, k, ph = workloads.rff_draws(3, sigma, ell, K, seed=100 + s)
        F[s] = dg.rff_theta(_Points(pts), sg, k, ph).ravel()
    f0 = F[:, :P]
    # mean zero (standard error about sigma / sqrt(M P))
    assert abs(F[:, :P].mean()) <= 5 * sigma / math.sqrt(M * P) * 3
    for i, r in enumerate(lags):
        fr = F[:, i * P:(i + 1) * P]
        cov = np.mean(f0 * fr) / sigma ** 2
        want = math.exp(-r * r / (2 * ell * ell))
        assert abs(cov - want) <= 0.06, (r, cov, want)
    # variance sigma^2 at every point, including next to the origin
    var_near = np.mean(F[:, 3 * P:] ** 2) / sigma ** 2
    assert abs(var_near - 1.0) <= 0.3, var_near


def test_covariance_pin_rejects_planted_mistakes():
    """The same statistics with a mistake planted in a copy of the field: no sqrt(2/K) factor,
    k drawn with l instead of 1/l, the phase left out."""
    sigma, ell, K = 0.05, 300.0, 512
    rng = np.random.default_rng(2)
    near = rng.uniform(-0.2 * ell, 0.2 * ell, (8, 3))
    far = rng.uniform(2000.0, 8000.0, (24, 3))
    u = np.array([1.0, 0.0, 0.0])
    pts = np.concatenate([far, far + ell * u, near])
    mesh = _Points(pts)

    def field(mistake, k, ph):
        acc = np.zeros(pts.shape[0])
        for m in range(K):
            arg = (0.0 if mistake == "no_phase" else ph[m]) + pts @ k[m]
            acc += np.cos(arg)
        scale = sigma if mistake == "no_norm" else sigma * math.sqrt(2.0 / K)
        return scale * acc

    def stats(fn):
        F = np.array([fn(*workloads.rff_draws(3, sigma, ell, K, seed=500 + s)[1:]) for s in range(120)])
        var_far = np.mean(F[:, :24] ** 2) / sigma ** 2
        cov_l = np.mean(F[:, :24] * F[:, 24:48]) / sigma ** 2
        var_near = np.mean(F[:, 48:] ** 2) / sigma ** 2
        return var_far, cov_l, var_near

    good = stats(lambda k, ph: dg.rff_theta(mesh, sigma, k, ph).ravel())
    assert abs(good[0] - 1) <= 0.15 and abs(good[1] - math.exp(-0.5)) <= 0.1 and abs(good[2] - 1) <= 0.35
    bad_norm = stats(lambda k, ph: field("no_norm", k, ph))
    assert abs(bad_norm[0] - 1) > 0.15
    bad_len = stats(lambda k, ph: field("ok", k * ell * ell, ph))   # k ~ N(0, l^2 I)
    assert abs(bad_len[1] - math.exp(-0.5)) > 0.1
    bad_phase = stats(lambda k, ph: field("no_phase", k, ph))
    assert abs(bad_phase[2] - 1) > 0.35
