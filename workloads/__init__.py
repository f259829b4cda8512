"""Seeded synthetic inputs shared by the tests, the benchmark and the oracle comparisons.

This module holds no arithmetic of the method: it only names the workloads (sizes, bubble
parameters, time steps) and draws random numbers.  Both the CUDA library and the oracle take
what it produces as inputs.

Workloads restate the five benchmark configurations of the tree-based dGSEM study
(2D rising bubble on a uniform grid, 2D cold bubble with AMR, 3D octree bubble, a batch of
small 2D instances, and a 3D adjoint case); values the source leaves open are the readings
listed beside them.
"""
import numpy as np

SEED_BASE = 0x2404166480000000


def rng(config_id, stream=0):
    """Seeded generator for a workload (PCG64 seeded from the base seed + ids)."""
    return np.random.Generator(np.random.PCG64([SEED_BASE + int(config_id), int(stream)]))


# 2D x-z, uniform 10 x 10, N = 4: rising thermal bubble (theta_c = 0.5 K, r = 250 m)
RTB_2D = dict(name="rtb2d_10x10_N4", dim=2, N=4, base=(10, 10), length=(1000.0, 1000.0),
              max_level=0, bubble=dict(center=(500.0, 350.0), radius=(250.0, 250.0), amp=0.25),
              dt=0.02, steps=100, threshold=None, buffer=2, regrid_every=None)

# 2D x-z, 32 x 8 base, N = 5, up to 3 levels: cold bubble (theta' = -7.5 (1 + cos(pi r)))
# dt reading: 0.01 s (0.05 s is above the explicit limit at 100 m); viscosity 75 m^2/s (BR1)
COLD_2D = dict(name="cold2d_32x8_N5_L3", dim=2, N=5, base=(32, 8), length=(25600.0, 6400.0),
               max_level=3, bubble=dict(center=(0.0, 3000.0), radius=(4000.0, 2000.0), amp=-7.5),
               dt=0.01, steps=2000, threshold=0.1, buffer=2, regrid_every=10, nu=75.0)

# 3D octree, 16^3 base, N = 7, 2 extra levels where |theta'| > 0.05 K: warm bubble
# theta' = 2 (1 + cos(pi r / 2 km)) at (5, 5, 2) km; dt reading 0.005 s; buffer reading B = 2
BUBBLE_3D = dict(name="bubble3d_16cube_N7_L2", dim=3, N=7, base=(16, 16, 16),
                 length=(10000.0, 10000.0, 10000.0), max_level=2,
                 bubble=dict(center=(5000.0, 5000.0, 2000.0), radius=(2000.0, 2000.0, 2000.0), amp=2.0),
                 dt=0.005, steps=1000, threshold=0.05, buffer=2, regrid_every=20)

# 3D 12^3, N = 5, warm bubble + Gaussian random theta' (sigma 0.05 K, length 300 m)
ADJOINT_3D = dict(name="adjoint3d_12cube_N5", dim=3, N=5, base=(12, 12, 12),
                  length=(5000.0, 5000.0, 5000.0), max_level=0,
                  bubble=dict(center=(2500.0, 2500.0, 2000.0), radius=(1000.0, 1000.0, 1000.0), amp=1.0),
                  dt=0.02, steps=200, rff=dict(sigma=0.05, length=300.0, features=512))

CONFIGS = {c["name"]: c for c in (RTB_2D, COLD_2D, BUBBLE_3D, ADJOINT_3D)}

# Swirling deformational flow (Sec. 4.2, after LeVeque): tracer cosine bell (h_max = 1) at
# (0.25, 0.25) with r_c = 0.25 on [0, 1]^2, 16 x 16 roots, N = 4, one extra level where |C| > 0.05
# (reading), buffer 2, period T = 5 with 80 regrids; dt reading 2.5e-3 (2000 steps).
LEVEQUE_2D = dict(name="leveque2d_16x16_N4_L1", dim=2, N=4, base=(16, 16), length=(1.0, 1.0),
                  max_level=1, bubble=dict(center=(0.25, 0.25), radius=(0.25, 0.25), amp=0.5),
                  period=5.0, dt=2.5e-3, steps=2000, threshold=0.05, buffer=2, regrid_every=25)

# Batched 2D bubbles: 256 instances on [0, 1000]^2 with seeded radius U[150, 400] m, amplitude
# U[0.1, 2] K, centre (500, 350) m, mesh 10x10 ... 64x32, N in {3..7}, precision 50/50, 500 steps.
BATCH_MESHES = ((10, 10), (16, 16), (20, 16), (32, 16), (32, 32), (48, 24), (64, 32))
BATCH_2D = dict(name="batch2d_256_bubbles", count=256, steps=500, length=(1000.0, 1000.0))


def batch_instances(count=256, seed=4, meshes=BATCH_MESHES):
    """Seeded instance descriptions of the batched workload.  dt is half of the explicit limit
    estimate h_min / ((2N + 1) c) with c = 360 m/s."""
    g = rng(seed, 7)
    out = []
    for i in range(count):
        base = meshes[int(g.integers(len(meshes)))]
        N = int(g.integers(3, 8))
        prec = "fp32" if g.random() < 0.5 else "fp64"
        radius = float(g.uniform(150.0, 400.0))
        amp = float(g.uniform(0.1, 2.0))
        hmin = min(1000.0 / base[0], 1000.0 / base[1])
        out.append(dict(base=base, N=N, precision=prec, dt=0.5 * hmin / ((2 * N + 1) * 360.0),
                        bubble=dict(center=(500.0, 350.0), radius=(radius, radius), amp=amp / 2.0)))
    return out


def scaled(cfg, base_div=1, N=None):
    """A smaller copy of a workload (same physics, fewer root cells and/or lower degree)."""
    c = dict(cfg)
    c["base"] = tuple(max(1, b // base_div) for b in cfg["base"])
    if N is not None:
        c["N"] = N
    c["name"] = cfg["name"] + "_div%d" % base_div + ("_N%d" % N if N else "")
    return c


def rff_draws(dim, sigma, length, features, seed=5):
    """Random Fourier features of a Gaussian covariance sigma^2 exp(-r^2 / (2 l^2)):
    wave vectors k ~ N(0, l^-2 I), phases ~ U[0, 2 pi)."""
    g = rng(seed, 1)
    k = g.standard_normal((features, dim)) / length
    phase = g.uniform(0.0, 2.0 * np.pi, features)
    return sigma, k, phase


def random_state(nv, E, NP, seed, rho_scale=1e-3, u_scale=2.0, theta_scale=0.3, dtype=np.float64):
    """White-noise perturbation state [nv, E, NP] (discontinuous across elements, so every
    face term is exercised)."""
    g = rng(1000 + int(seed))
    q = np.empty((nv, E, NP))
    q[0] = rho_scale * g.standard_normal((E, NP))
    q[1:nv - 1] = u_scale * g.standard_normal((nv - 2, E, NP))
    q[nv - 1] = theta_scale * g.standard_normal((E, NP))
    return q.astype(dtype)


def random_scalar(E, NP, seed, scale=1.0, offset=0.0):
    """White-noise scalar field [E, NP] (a tracer), offset + scale * N(0, 1)."""
    g = rng(4000 + int(seed))
    return offset + scale * g.standard_normal((E, NP))


def random_flags(n, p, seed):
    return (rng(2000 + int(seed)).random(n) < p).astype(np.uint8)


def sample_elements(E, count, seed):
    """Sorted sample of element ids (for full-size parity on sampled outputs)."""
    g = rng(3000 + int(seed))
    return np.sort(g.choice(E, size=min(count, E), replace=False))
