"""Differentiable trajectory batch (B-spline positions, per-sample yaw, objective sum -log det):
the library's forward and hand-written backward, chained through the B-spline map, against the
FP64 oracle objective, the oracle's analytic gradient and central differences (step 1e-4) of the
oracle objective, at <= 1e-3 relative."""
import math

import numpy as np
import pytest
import torch

import oracle as O
from paper_2008_03324_gb300 import synth
from tests import _fixtures as X

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def F():
    from paper_2008_03324_gb300 import build as B
    B.build()
    from paper_2008_03324_gb300 import fif
    return fif


def setup_batch(n_traj=6, n_ctrl=8, n_samples=16, seed=61):
    rng = np.random.default_rng(seed)
    ctrl = np.stack([rng.uniform(1.0, 9.0, (n_traj, n_ctrl)), rng.uniform(1.0, 9.0, (n_traj, n_ctrl)),
                     rng.uniform(0.6, 2.4, (n_traj, n_ctrl))], axis=-1)
    yaw = np.cumsum(rng.uniform(-0.5, 0.5, (n_traj, n_ctrl)), axis=1) + rng.uniform(-3, 3, (n_traj, 1))
    return ctrl.astype(np.float32), yaw.astype(np.float32), synth.bspline_basis(n_ctrl, n_samples).astype(np.float32)


def oracle_objective(ctrl, yaw, basis):
    t = np.einsum("sc,tcd->tsd", basis.astype(np.float64), ctrl.astype(np.float64)).reshape(-1, 3)
    psi = (yaw.astype(np.float64) @ basis.T.astype(np.float64)).reshape(-1)
    q = synth.horizontal_quats(psi)
    poses = np.concatenate([t, q], axis=1)
    grid = X.oracle_grid(X.ROOM["grid"])
    nodes, w, dw, _ = O.query_cells(grid, poses)
    k = O.quad_coeffs(math.pi / 4, 0.8)
    Fw = X.room_field_oracle(False)
    I = O.query(Fw[nodes], w, poses, k)
    m = O.metrics(I)
    mask = m[:, 2] > 0
    gm = np.zeros((len(poses), 3))
    gm[mask, 1] = -1.0
    g = O.query_grad(Fw[nodes], w, dw, poses, k, gm)
    return -(m[mask, 1]).sum(), g, mask


def test_trajectory_objective_and_gradients(F):
    from paper_2008_03324_gb300 import traj
    spec = X.ROOM["grid"]
    field = F.Field(spec.origin, spec.res, spec.dims, F.make_params(r_max=8.0, v_alpha=0.8))
    field.coeffs.copy_(torch.from_numpy(X.pack_field(X.room_field_oracle(True))))
    ctrl, yaw, basis = setup_batch()
    c = torch.from_numpy(ctrl).cuda().requires_grad_(True)
    y = torch.from_numpy(yaw).cuda()
    B = torch.from_numpy(basis).cuda()
    loss, phi, met, sg = traj.neg_logdet_objective(c, y, B, field)
    loss.backward()
    torch.cuda.synchronize()
    L_ref, g_ref, mask = oracle_objective(ctrl, yaw, basis)
    assert (sg.cpu().numpy() > 0).sum() == mask.sum()
    assert float(loss) == pytest.approx(L_ref, rel=1e-5)
    # d loss / d ctrl = sum over samples B[s, c] d loss / d t
    T, C, _ = ctrl.shape
    S = basis.shape[0]
    gt = g_ref[:, :3].reshape(T, S, 3)
    gc_ref = np.einsum("sc,tsd->tcd", basis.astype(np.float64), gt)
    gc = c.grad.cpu().numpy().astype(np.float64)
    assert np.linalg.norm(gc - gc_ref) <= 1e-3 * np.linalg.norm(gc_ref)
    gphi = phi.grad.cpu().numpy().astype(np.float64)
    assert np.linalg.norm(gphi - g_ref[:, 3:]) <= 1e-3 * np.linalg.norm(g_ref[:, 3:])
    # central differences of the FP64 oracle objective on a few control-point coordinates
    h = 1e-4
    rng = np.random.default_rng(3)
    for _ in range(6):
        tt, cc, dd = rng.integers(T), rng.integers(C), rng.integers(3)
        cp, cm = ctrl.astype(np.float64).copy(), ctrl.astype(np.float64).copy()
        cp[tt, cc, dd] += h
        cm[tt, cc, dd] -= h
        fd = (oracle_objective(cp, yaw, basis)[0] - oracle_objective(cm, yaw, basis)[0]) / (2 * h)
        assert abs(gc[tt, cc, dd] - fd) <= 1e-3 * max(abs(fd), 1e-3 * np.abs(gc_ref).max())


def test_graphed_objective_replays_the_eager_result(F):
    """traj.GraphedObjective (the objective and its backward captured in one CUDA graph): for two
    different sets of control points, a replay gives bitwise the loss and the control-point and
    so(3) gradients of the eager evaluation, and the first set's again after the second."""
    from paper_2008_03324_gb300 import traj
    spec = X.ROOM["grid"]
    field = F.Field(spec.origin, spec.res, spec.dims, F.make_params(r_max=8.0, v_alpha=0.8))
    field.coeffs.copy_(torch.from_numpy(X.pack_field(X.room_field_oracle(True))))
    ctrl, yaw, basis = setup_batch(n_traj=16, n_ctrl=8, n_samples=32)
    B = torch.from_numpy(basis).cuda()
    sets = [(torch.from_numpy(ctrl).cuda(), torch.from_numpy(yaw).cuda()),
            (torch.from_numpy(ctrl + np.float32(0.05)).cuda(), torch.from_numpy(yaw - np.float32(0.1)).cuda())]

    def eager(c0, y0):
        c = c0.clone().requires_grad_(True)
        loss, phi, _, _ = traj.neg_logdet_objective(c, y0, B, field)
        loss.backward()
        return float(loss), c.grad.clone(), phi.grad.clone()

    ref = [eager(c, y) for c, y in sets]
    g = traj.GraphedObjective(sets[0][0], sets[0][1], B, field)
    for k in (0, 1, 0):
        loss, gc = g.step(*sets[k])
        torch.cuda.synchronize()
        assert F.device_error() == 0
        assert float(loss) == ref[k][0]
        assert torch.equal(gc, ref[k][1]) and torch.equal(g.phi_grad, ref[k][2])
