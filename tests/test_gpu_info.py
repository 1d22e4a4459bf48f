"""Information threshold and potential cost on the GPU (Sec. VI-B, Eq. info_pot_cost) against the
FP64 oracle: per-set metrics and thresholds for the point cloud, the quadratic field and the GP
field (2,000 sets of 200 landmarks at 0.3-1.0 m, the paper's specification), degenerate sets,
the empty batch, the cost and its derivative elementwise (a strided metric column, NaN), and a
trajectory objective built on the cost whose gradient goes through the query adjoint.

Tolerances: each set's FIM is summed in single precision (relative Frobenius <= 1e-5, as for
the field); for a positive semidefinite FIM ||I||_F <= trace, so the metric bounds of the query
tests become |d trace| <= sqrt(6) tau tr, |d lambda_min| <= tau tr and
|d log|det|| <= 2 sqrt(6) tau tr / lambda_min, and a threshold (a mean) is within the mean of
its sets' bounds."""
import math

import numpy as np
import pytest
import torch

import oracle as O
from paper_2008_03324_gb300 import synth
from tests import _fixtures as X
from tests.test_oracle_gp import FITTED

pytestmark = pytest.mark.gpu
TAU = X.TAU_F32


@pytest.fixture(scope="module")
def F():
    from paper_2008_03324_gb300 import build as B
    B.build()
    from paper_2008_03324_gb300 import fif
    return fif


def bounds(m_ref):
    tr, lm = m_ref[:, 0], m_ref[:, 3]
    return math.sqrt(6) * TAU * tr, 2 * math.sqrt(6) * TAU * tr / np.maximum(lm, 1e-300), TAU * tr


@pytest.mark.parametrize("model", ["pointcloud", "quad", "gp"])
def test_threshold_vs_oracle(F, model):
    sets = synth.threshold_sets(11, 2000, 200, 0.3, 1.0)
    fmodel = {"pointcloud": F.MODEL_POINTCLOUD, "quad": F.MODEL_QUAD, "gp": F.MODEL_GP}[model]
    omodel = {"pointcloud": O.MODEL_POINTCLOUD, "quad": O.MODEL_QUAD, "gp": O.MODEL_GP}[model]
    axes = synth.fibonacci_sphere(30)
    gpc = F.gp_struct(axes, FITTED[30]) if model == "gp" else None
    ogp = O.GP(axes, FITTED[30]) if model == "gp" else None
    prm = F.make_params(v_alpha=0.6, sigma=0.8)
    met, thr = F.info_threshold(prm, torch.from_numpy(sets).cuda(), fmodel, gpc)
    torch.cuda.synchronize()
    met, thr = met.cpu().numpy(), thr.cpu().numpy()
    m_ref, t_ref = O.info_threshold(sets, O.make_params(v_alpha=0.6, sigma=0.8), omodel, ogp)
    t_tr, t_ld, t_lm = bounds(m_ref)
    assert np.all(np.abs(met[:, 0] - m_ref[:, 0]) <= t_tr)
    assert np.all(np.abs(met[:, 1] - m_ref[:, 1]) <= t_ld)
    assert np.all(np.abs(met[:, 2] - m_ref[:, 3]) <= t_lm)
    assert np.all(m_ref[:, 3] > 1e-3 * m_ref[:, 0])          # no set near the exclusion test
    for c, tol in enumerate((t_tr, t_ld, t_lm)):
        assert abs(thr[c] - t_ref[c]) <= tol.mean()
    # bitwise reproducible
    _, thr2 = F.info_threshold(prm, torch.from_numpy(sets).cuda(), fmodel, gpc)
    assert np.array_equal(thr, thr2.cpu().numpy())


def test_degenerate_and_empty(F):
    prm = F.make_params()
    deg = torch.from_numpy(synth.threshold_sets(6, 70, 2)).cuda()
    _, thr = F.info_threshold(prm, deg, F.MODEL_POINTCLOUD, exclude_degenerate=True)
    assert torch.all(torch.isnan(thr))
    _, thr = F.info_threshold(prm, deg, F.MODEL_POINTCLOUD, exclude_degenerate=False)
    assert torch.isfinite(thr[0])
    empty = torch.empty(0, 5, 3, device="cuda")
    _, thr = F.info_threshold(prm, empty, F.MODEL_QUAD)
    torch.cuda.synchronize()
    assert torch.all(torch.isnan(thr))
    with pytest.raises(F.FifError):
        F.info_threshold(prm, deg, F.MODEL_GP, None)


def test_cost_vs_oracle(F):
    rng = np.random.default_rng(8)
    v = rng.uniform(-40, 60, size=(5000, 3))
    v[::97, 1] = np.nan
    eps, kq = 26.5, 0.02
    c, dc = F.info_cost(torch.from_numpy(v).cuda(), eps, kq, column=1)
    torch.cuda.synchronize()
    c_ref, dc_ref = O.info_cost(v[:, 1], eps, kq)
    np.testing.assert_allclose(c.cpu().numpy(), c_ref, rtol=1e-14, atol=1e-12)
    np.testing.assert_allclose(dc.cpu().numpy(), dc_ref, rtol=1e-14, atol=1e-12)
    c1, _ = F.info_cost(torch.from_numpy(np.ascontiguousarray(v[:, 1])).cuda(), eps, kq)
    assert torch.equal(c1.nan_to_num(-1.0), c.nan_to_num(-1.0))
    with pytest.raises(F.FifError):
        F.info_cost(torch.from_numpy(v).cuda(), -1.0, kq, column=0)


def test_potential_cost_trajectory_gradient(F):
    """loss = sum_s c(log|det| I_s) over a trajectory batch on the room field: value against the
    oracle objective, gradient against the oracle's analytic gradient with d c/d v as the
    metric weight (chain rule through Eq. info_pot_cost and the query adjoint)."""
    from paper_2008_03324_gb300 import traj
    from tests.test_gpu_traj import setup_batch
    spec = X.ROOM["grid"]
    field = F.Field(spec.origin, spec.res, spec.dims, F.make_params(r_max=8.0, v_alpha=0.8))
    field.coeffs.copy_(torch.from_numpy(X.pack_field(X.room_field_oracle(True))))
    ctrl, yaw, basis = setup_batch()
    t = np.einsum("sc,tcd->tsd", basis.astype(np.float64), ctrl.astype(np.float64)).reshape(-1, 3)
    psi = (yaw.astype(np.float64) @ basis.T.astype(np.float64)).reshape(-1)
    poses = np.concatenate([t, synth.horizontal_quats(psi)], axis=1)
    grid = X.oracle_grid(spec)
    nodes, w, dw, _ = O.query_cells(grid, poses)
    k = O.quad_coeffs(math.pi / 4, 0.8)
    Fw = X.room_field_oracle(False)
    m_ref = O.metrics(O.query(Fw[nodes], w, poses, k))
    eps, kq = float(np.percentile(m_ref[:, 1], 70)), 0.05     # samples on both sides of eps
    c_ref, dc_ref = O.info_cost(m_ref[:, 1], eps, kq)
    gm = np.zeros((len(poses), 3))
    gm[:, 1] = dc_ref
    g_ref = O.query_grad(Fw[nodes], w, dw, poses, k, gm)
    c = torch.from_numpy(ctrl).cuda().requires_grad_(True)
    loss, phi, met = traj.potential_cost_objective(c, torch.from_numpy(yaw).cuda(), torch.from_numpy(basis).cuda(),
                                                   field, eps, kq, column=1)
    loss.backward()
    torch.cuda.synchronize()
    assert 0 < (c_ref > 0).sum() < len(c_ref)
    assert float(loss) == pytest.approx(c_ref.sum(), rel=1e-3)
    T, C, _ = ctrl.shape
    gc_ref = np.einsum("sc,tsd->tcd", basis.astype(np.float64), g_ref[:, :3].reshape(T, basis.shape[0], 3))
    gc = c.grad.cpu().numpy().astype(np.float64)
    assert np.linalg.norm(gc - gc_ref) <= 1e-3 * np.linalg.norm(gc_ref)
    gphi = phi.grad.cpu().numpy().astype(np.float64)
    assert np.linalg.norm(gphi - g_ref[:, 3:]) <= 1e-3 * np.linalg.norm(g_ref[:, 3:])
