"""The FP64 reciprocal and square root of the flux kernels (Newton-Raphson from the hardware
approximations) against the correctly rounded values: within one ulp everywhere on a range that
covers the densities, pressures and sound speeds of the workloads and every binade position."""
import ctypes

import numpy as np
import pytest

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def pkg():
    import torch
    assert torch.cuda.is_available()
    from paper_2404_16648_gb300 import build as b
    b.build()
    import paper_2404_16648_gb300 as p
    return p


def _ulps(got, want):
    return np.abs(got - want) / np.spacing(np.abs(want))


def test_recip_and_sqrt_within_one_ulp(pkg):
    import torch
    rng = np.random.default_rng(1)
    x = np.concatenate([10.0 ** rng.uniform(-6, 8, 200000),
                        np.ldexp(1.0, np.arange(-30, 40)),                       # powers of two
                        np.nextafter(np.ldexp(1.0, np.arange(-30, 40)), 0.0),   # just below them
                        1.0 + rng.uniform(-1e-3, 1e-3, 20000)])                  # densities near 1
    xd = torch.from_numpy(x).cuda()
    r = torch.empty_like(xd)
    s = torch.empty_like(xd)
    lib = pkg.load_library()
    assert lib.dg_probe_recip_sqrt(x.size, ctypes.c_void_p(xd.data_ptr()), ctypes.c_void_p(r.data_ptr()),
                                   ctypes.c_void_p(s.data_ptr()), None) == 0
    torch.cuda.synchronize()
    assert _ulps(r.cpu().numpy(), 1.0 / x).max() <= 1.0
    assert _ulps(s.cpu().numpy(), np.sqrt(x)).max() <= 1.0
