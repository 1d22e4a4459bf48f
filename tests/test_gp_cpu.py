"""Host-side parts of the GP visibility model in the library (no GPU): the record layout and
the maximum-marginal-likelihood length scale, checked against the FP64 oracle's likelihood."""
import math

import numpy as np
import pytest

import oracle as O
from paper_2008_03324_gb300 import synth


@pytest.fixture(scope="module")
def F():
    from paper_2008_03324_gb300 import build as B
    B.build()
    from paper_2008_03324_gb300 import fif
    return fif


def test_record_layout(F):
    """rs is the smallest count >= N_s with rs = 2 (mod 4); the node record is 21 rs floats
    rounded up to 16 bytes; bad counts give 0."""
    for ns in range(1, F.GP_MAX_SAMPLES + 1):
        rs = F.gp_row_stride(ns)
        assert rs >= ns and rs % 4 == 2 and rs - ns < 4
        st = F.gp_stride(ns)
        assert st >= 21 * rs and st % 4 == 0 and st - 21 * rs < 4
        assert F.gp_aux_bytes(ns) >= 8 * ns * rs
    for bad in (0, -3, F.GP_MAX_SAMPLES + 1):
        assert F.gp_row_stride(bad) == 0 and F.gp_stride(bad) == 0 and F.gp_aux_bytes(bad) == 0
    g = F.make_grid((0, 0, 0), 0.5, (4, 5, 6))
    assert F.gp_field_bytes(g, 70) == 4 * 5 * 6 * F.gp_stride(70) * 4


@pytest.mark.parametrize("ns", [30, 50, 70])
def test_length_scale_fit_maximises_the_oracle_likelihood(F, ns):
    """Sec. V-B-2: the length scale maximises the marginal likelihood of the sigmoid training
    vectors.  The library's fit (Cholesky, golden section) lands on the maximiser of the
    oracle's likelihood (Gauss-Jordan inverse, LU determinant): nearby scales score lower."""
    axes = synth.fibonacci_sphere(ns)
    P = synth.sphere_points(7, 2000)
    l = F.gp_fit_length_scale(axes, P, half_fov=math.pi / 4, k_s=15.0, noise_var=1e-10)
    Y = O.gp_training(axes, 15.0, math.pi / 4, P)
    f0 = O.gp_log_marginal(axes, l, 1e-10, Y)
    for d in (1e-3, -1e-3, 1e-2, -1e-2):
        assert O.gp_log_marginal(axes, l * (1 + d), 1e-10, Y) < f0
    from tests.test_oracle_gp import FITTED
    assert l == pytest.approx(FITTED[ns], rel=2e-4)


def test_fit_rejects_bad_arguments(F):
    axes = synth.fibonacci_sphere(10)
    P = synth.sphere_points(1, 20)
    with pytest.raises(F.FifError):
        F.gp_fit_length_scale(axes, P, l_lo=1.0, l_hi=0.5)
    with pytest.raises(F.FifError):
        F.gp_fit_length_scale(np.zeros((3, 3)), P)
