"""P' of the FP32 path (FP64 is kept for the pressure perturbation, read as: P' carried to FP64
accuracy before its FP32 rounding).  The line stage kernel (layout 4) forms P' of its output by a
split-FP32 product, the half-column layout and the P' kernel in FP64 arithmetic.  On the same FP32
state the P' planes must agree bit for bit for layout 3 and within one ulp, on a small fraction of
the nodes, for layout 4; nodes with |Theta'/Theta_bar| > 2^-5 take the FP64 form in both.  The
FP64 line-pass stage (layout 5) sums the FP64 series with a number of terms matched to |x|: its
P' plane agrees with the P' kernel's within a few ulps."""
import numpy as np
import pytest

import workloads

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def pkg():
    import torch
    assert torch.cuda.is_available()
    from paper_2404_16648_gb300 import build as b
    b.build()
    import paper_2404_16648_gb300 as p
    return p


def _mesh(pkg):
    lm = pkg.Mesh(3, 7, (3, 3, 2), (3000.0, 3000.0, 2000.0), max_level=1, precision="fp32")
    lm.adapt(flags=workloads.random_flags(lm.num_elements, 0.3, seed=77), buffer=1)
    return lm


def _state(lm, seed):
    q = workloads.random_state(5, lm.num_elements, 512, seed=seed, theta_scale=2.0)
    q[4, ::7, 5] = 20.0        # |x| above 2^-5: the full FP64 form on both sides
    q[4, 3::11, 9] = -15.0
    return q.astype(np.float32)


@pytest.mark.parametrize("layout", [3, 4])
def test_stage_pprime_against_fp64_form(pkg, layout):
    lm = _mesh(pkg)
    lm.set_stage_kernel(layout)
    for seed in (1, 2):
        lm.set_state(_state(lm, seed))
        lm.step(0.02, 1)
        p_stage = lm.pprime()          # written by the stage epilogue
        q = lm.get_state()
        lm.set_state(q)                # P' of the same state from the FP64-form kernel
        p_ref = lm.pprime()
        assert np.all(np.isfinite(p_ref)) and np.abs(p_ref).max() > 100.0
        ulps = np.abs(p_stage.astype(np.float64) - p_ref) / np.spacing(np.abs(p_ref))
        if layout == 3:
            np.testing.assert_array_equal(p_stage, p_ref)
        else:
            assert ulps.max() <= 1.0
            assert (ulps > 0).mean() <= 0.05, (ulps > 0).mean()
            # the large-|x| nodes take the same FP64 form
            sel = np.abs(q[4]) >= 15.0
            np.testing.assert_array_equal(p_stage[sel], p_ref[sel])


def test_fp64_line_pass_pprime_tiers(pkg):
    """The FP64 line-pass stage (layout 5) sums the binomial series of P' with as many terms as
    |x| = |Theta' / Theta_bar| needs (2 terms below 2^-27, up to 7 below 2^-7; the general form
    above), the tier picked from the bits of x.  On a state whose Theta' spans all tiers
    (log-uniform |x| from 1e-11 to 0.06, both signs, some elements at rest) and a step short
    enough to leave it in place, the P' plane the stage writes matches the P' kernel's general
    form on the same state within 4 ulps, and both are exactly 0 where Theta' is."""
    lm = pkg.Mesh(3, 7, (3, 3, 2), (3000.0, 3000.0, 2000.0), max_level=1, precision="fp64")
    lm.adapt(flags=workloads.random_flags(lm.num_elements, 0.3, seed=77), buffer=1)
    lm.set_stage_kernel(5)
    E = lm.num_elements
    q = workloads.random_state(5, E, 512, seed=6, rho_scale=1e-6, u_scale=0.2)
    g = np.random.default_rng(11)
    sign = np.where(g.random((E, 512)) < 0.5, -1.0, 1.0)
    x = sign * 10.0 ** g.uniform(-11.0, np.log10(0.06), size=(E, 512))
    q[4] = 350.0 * x                   # Theta_bar is about 290-350 kg K/m^3 below 2 km
    q[:, : E // 3] = 0.0               # elements at rest: P' stays 0 where nothing reaches them
    lm.set_state(q)
    lm.step(1e-30, 1)                  # leaves Theta' where it was: every tier stays visited
    p_stage = lm.pprime()              # written by the layout-5 stage epilogue
    q1 = lm.get_state()
    lm.set_state(q1)                   # P' of the same state from the general FP64 form
    p_ref = lm.pprime()
    th = np.abs(q1[4])
    assert th[th > 0].min() < 1e-6 and th.max() > 15.0      # every tier is visited
    zero = p_ref == 0.0
    np.testing.assert_array_equal(p_stage[zero], 0.0)
    ulps = np.abs(p_stage[~zero] - p_ref[~zero]) / np.spacing(np.abs(p_ref[~zero]))
    print("P' tiers: max %.1f ulp, %.3f of the nodes differ" % (ulps.max(), (ulps > 0).mean()))
    assert ulps.max() <= 4.0
