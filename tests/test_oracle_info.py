"""Pins of the FP64 oracle's information threshold and potential cost (Sec. VI-B, Eq.
info_pot_cost) against what the paper and the mathematics fix: each set's FIM against the
point-cloud routines (a different code path), the trace's closed form sum_i v_i (2 + 2/n_i^2)
and its expectation over the sampling distribution, the exclusion of degenerate sets, and
the continuity and shape of the potential cost.  No GPU."""
import math

import numpy as np
import pytest

import oracle as O
from paper_2008_03324_gb300 import synth
from tests.test_oracle_gp import FITTED


def _as_world(sets):
    """Each camera-frame set as a world map seen from the identity pose at the origin."""
    return [np.ascontiguousarray(s, np.float32) for s in sets]


POSE0 = np.array([[0, 0, 0, 1, 0, 0, 0]], np.float32)


@pytest.mark.parametrize("model", [O.MODEL_POINTCLOUD, O.MODEL_QUAD, O.MODEL_GP])
def test_set_fim_matches_point_cloud_routines(model):
    """The FIM of a set equals the point-cloud FIM at the camera with v = 1, the quadratic
    visibility weight, or the GP visibility weight (the routines the field pins use)."""
    sets = synth.threshold_sets(3, 6, 40)
    prm = O.make_params(r_max=8.0)
    gp = O.GP(synth.fibonacci_sphere(30), FITTED[30]) if model == O.MODEL_GP else None
    met, _ = O.info_threshold(sets, prm, model, gp, exclude_degenerate=False)
    for s, lm in enumerate(_as_world(sets)):
        if model == O.MODEL_POINTCLOUD:
            I = O.pc_fim(lm, POSE0, prm, vis=O.VIS_ONE)[0]
        elif model == O.MODEL_QUAD:
            I = O.pc_fim(lm, POSE0, prm, vis=O.VIS_QUAD)[0]
        else:
            I = O.pc_fim_gp(lm, POSE0, prm, gp)[0]
        ref = O.metrics(I[None])[0]
        np.testing.assert_allclose(met[s], ref, rtol=1e-10, atol=1e-10)


@pytest.mark.parametrize("model", [O.MODEL_POINTCLOUD, O.MODEL_QUAD])
def test_trace_closed_form(model):
    """tr I_i = (2 + 2/n^2) / sigma^2 for any bearing (P = I - u u^T has trace 2), so
    tr I_s = sum_i v_i (2 + 2/n_i^2) / sigma^2."""
    sets = synth.threshold_sets(4, 20, 30)
    prm = O.make_params(sigma=0.5, v_alpha=0.7)
    met, thr = O.info_threshold(sets, prm, model, exclude_degenerate=False)
    k = O.quad_coeffs(math.pi / 4, 0.7)
    S = sets.astype(np.float64)
    n = np.linalg.norm(S, axis=-1)
    c = S[..., 2] / n
    v = np.ones_like(n) if model == O.MODEL_POINTCLOUD else k[2] * c * c + k[1] * c + k[0]
    ref = (v * (2 + 2 / n ** 2)).sum(1) / 0.25
    np.testing.assert_allclose(met[:, 0], ref, rtol=1e-12)
    assert thr[0] == pytest.approx(ref.mean(), rel=1e-12)


def test_trace_threshold_matches_expectation():
    """For r^3 uniform on [a, b], E[1/r^2] = 3 (b - a) / (b^3 - a^3): the point-cloud trace
    threshold of M landmarks converges to M (2 + 6 (b - a) / (b^3 - a^3))."""
    a, b, M = 0.3, 1.0, 200
    sets = synth.threshold_sets(5, 3000, M, a, b)
    _, thr = O.info_threshold(sets, O.make_params(), O.MODEL_POINTCLOUD)
    expect = M * (2 + 6 * (b - a) / (b ** 3 - a ** 3))
    assert thr[0] == pytest.approx(expect, rel=3e-3)


def test_degenerate_sets_are_excluded():
    """Two bearings give a rank-4 FIM (each bearing adds rank 2): its lambda_min is rounding
    noise, so the condition test (lambda_min > 1e-6 trace) excludes it; with only degenerate
    sets the thresholds are NaN; the mean runs over the rest."""
    deg = synth.threshold_sets(6, 5, 2)
    _, thr = O.info_threshold(deg, O.make_params(), O.MODEL_POINTCLOUD, exclude_degenerate=True)
    assert np.all(np.isnan(thr))
    good = synth.threshold_sets(7, 5, 50)
    mix = np.concatenate([good, np.concatenate([deg, np.zeros((5, 48, 3), np.float32) + good[:, :48]], 1)])
    met, thr = O.info_threshold(mix, O.make_params(), O.MODEL_POINTCLOUD, exclude_degenerate=True)
    ok = (met[:, 2] > 0) & (met[:, 3] > 1e-6 * met[:, 0])
    assert ok.sum() == 10
    np.testing.assert_allclose(thr, [met[ok, 0].mean(), met[ok, 1].mean(), met[ok, 3].mean()], rtol=1e-12)
    _, thr_all = O.info_threshold(deg, O.make_params(), O.MODEL_POINTCLOUD, exclude_degenerate=False)
    assert np.all(np.isfinite(thr_all[[0]]))


@pytest.mark.parametrize("eps,kq", [(1.0, 3.0), (26.5, 0.01), (13.4, 2.0)])
def test_potential_cost_shape(eps, kq):
    """Eq. info_pot_cost: zero above the threshold, a parabola with its vertex at eps on
    [0, eps], and a line below 0 that continues the parabola's value and slope (the reading of
    the garbled continuity condition); c >= 0 and non-increasing, dc/dv the derivative."""
    v = np.linspace(-2 * eps, 2 * eps, 4001)
    c, dc = O.info_cost(v, eps, kq)
    assert np.all(c >= 0) and np.all(np.diff(c) <= 1e-12 * max(1.0, c.max()))
    assert np.all(c[v > eps] == 0) and np.all(dc[v > eps] == 0)
    h = 1e-6 * eps
    for x in (-0.7 * eps, 0.3 * eps, 0.9 * eps):
        cp, _ = O.info_cost([x + h], eps, kq)
        cm, _ = O.info_cost([x - h], eps, kq)
        _, d0 = O.info_cost([x], eps, kq)
        assert (cp[0] - cm[0]) / (2 * h) == pytest.approx(d0[0], rel=1e-6)
    for x0 in (0.0, eps):
        lo, dlo = O.info_cost([x0 - 1e-9 * eps], eps, kq)
        hi, dhi = O.info_cost([x0 + 1e-9 * eps], eps, kq)
        assert lo[0] == pytest.approx(hi[0], abs=1e-6 * kq * eps * eps)
        assert dlo[0] == pytest.approx(dhi[0], abs=1e-6 * kq * eps)
    c0, d0 = O.info_cost([0.0], eps, kq)
    assert c0[0] == pytest.approx(kq * eps * eps) and d0[0] == pytest.approx(-2 * kq * eps)
    cn, dn = O.info_cost([np.nan], eps, kq)
    assert np.isnan(cn[0]) and np.isnan(dn[0])
