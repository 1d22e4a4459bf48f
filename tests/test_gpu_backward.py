"""GPU adjoint (fif_query_backward, FifQuery) against the FP64 oracle gradient and central
finite differences of the FP64 oracle (step 1e-4), at <= 1e-3 relative."""
import math

import numpy as np
import pytest
import torch

import oracle as O
from paper_2008_03324_gb300 import synth
from tests import _fixtures as X
from tests import _np_geom as G

pytestmark = pytest.mark.gpu

TOL = 1e-3


@pytest.fixture(scope="module")
def F():
    from paper_2008_03324_gb300 import build as B
    B.build()
    from paper_2008_03324_gb300 import fif
    return fif


def uploaded(F, v_alpha):
    spec = X.ROOM["grid"]
    field = F.Field(spec.origin, spec.res, spec.dims, F.make_params(r_max=8.0, v_alpha=v_alpha))
    field.coeffs.copy_(torch.from_numpy(X.pack_field(X.room_field_oracle(True))))
    return field


def well_posed(I, which):
    """lambda_min's derivative needs a simple smallest eigenvalue: keep poses whose two
    smallest eigenvalues are separated by more than 1e-3 of the second one."""
    if which != 2:
        return np.ones(len(I), bool)
    ev = np.linalg.eigvalsh(I)
    return (ev[:, 1] - ev[:, 0]) > 1e-3 * np.abs(ev[:, 1])


@pytest.mark.parametrize("which", [0, 1, 2])
@pytest.mark.parametrize("world", [False, True])
def test_adjoint_matches_oracle_gradient(F, which, world):
    field = uploaded(F, 0.8)
    poses = synth.random_poses(51, 300, (0.3, 0.3, 0.3), (9.7, 9.7, 2.7))
    p = torch.from_numpy(poses).cuda()
    flags = F.Q_METRICS | (F.Q_WORLD if world else 0)
    fim, met, sg, st = field.query(p, flags)
    gm = np.zeros((300, 3))
    gm[:, which] = 1.0
    out = torch.empty(300, 6, device="cuda")
    F.query_backward(field.c, p, fim, torch.from_numpy(gm).cuda(), out, flags)
    torch.cuda.synchronize()
    g = out.cpu().numpy().astype(np.float64)
    grid = X.oracle_grid(X.ROOM["grid"])
    nodes, w, dw, _ = O.query_cells(grid, poses)
    k = O.quad_coeffs(math.pi / 4, 0.8)
    Fw = X.room_field_oracle(False)
    if world:
        # world-frame metrics: differentiate the oracle's world-frame query by central differences
        ref = np.array([fd_grad(p_, which, O.FRAME_WORLD, k) for p_ in poses[:40]])
        g, poses_c = g[:40], poses[:40]
    else:
        ref = O.query_grad(Fw[nodes], w, dw, poses, k, gm)
        poses_c = poses
    I_ref = O.query(Fw[nodes], w, poses, k, O.FRAME_WORLD if world else O.FRAME_CAMERA)[: len(ref)]
    ok = well_posed(I_ref, which)
    err = np.linalg.norm(g - ref, axis=1) / np.linalg.norm(ref, axis=1)
    assert ok.sum() >= 0.5 * len(ok)
    assert err[ok].max() <= TOL, (err[ok].max(), np.argmax(np.where(ok, err, 0)))
    assert np.all(g[:, 5] == 0.0)


def fd_grad(pose, which, frame, k, h=1e-4):
    grid = X.oracle_grid(X.ROOM["grid"])
    Fw = X.room_field_oracle(False)

    def metric(p):
        nodes, w, dw, _ = O.query_cells(grid, p[None])
        I = O.query(Fw[nodes], w, p[None], k, frame)
        m = O.metrics(I)[0]
        return [m[0], m[1], m[3]][which]

    pose = pose.astype(np.float64)
    g = np.zeros(6)
    for a in range(3):
        pp, pm = pose.copy(), pose.copy()
        pp[a] += h
        pm[a] -= h
        g[a] = (metric(pp) - metric(pm)) / (2 * h)
    R = G.R_from_quat(pose[3:])
    for a in range(3):
        e = np.zeros(3)
        e[a] = h
        pp, pm = pose.copy(), pose.copy()
        pp[3:] = G.quat_from_R(R @ G.so3_exp(e))
        pm[3:] = G.quat_from_R(R @ G.so3_exp(-e))
        g[3 + a] = (metric(pp) - metric(pm)) / (2 * h)
    return g


def test_adjoint_matches_central_differences(F):
    """Central differences with step 1e-4 on the FP64 oracle forward (camera frame, -log det
    as in the trajectory objective)."""
    field = uploaded(F, 0.8)
    poses = synth.random_poses(52, 24, (0.3, 0.3, 0.3), (9.7, 9.7, 2.7))
    p = torch.from_numpy(poses).cuda()
    fim, met, sg, st = field.query(p)
    gm = np.zeros((24, 3))
    gm[:, 1] = -1.0
    out = torch.empty(24, 6, device="cuda")
    F.query_backward(field.c, p, fim, torch.from_numpy(gm).cuda(), out, F.Q_METRICS)
    torch.cuda.synchronize()
    g = out.cpu().numpy()
    k = O.quad_coeffs(math.pi / 4, 0.8)
    for pose, gg in zip(poses, g):
        fd = -fd_grad(pose, 1, O.FRAME_CAMERA, k)
        assert np.linalg.norm(gg - fd) <= TOL * np.linalg.norm(fd)


def test_autograd_function(F):
    field = uploaded(F, 0.8)
    poses = torch.from_numpy(synth.random_poses(53, 100, (0.3, 0.3, 0.3), (9.7, 9.7, 2.7))).cuda()
    t = poses[:, :3].clone().requires_grad_(True)
    phi = torch.zeros(100, 3, device="cuda", requires_grad=True)
    met, sg, st = F.FifQuery.apply(t, phi, poses[:, 3:], field, F.Q_METRICS)
    loss = -(met[:, 1]).sum()
    loss.backward()
    fim, _, _, _ = field.query(poses)
    gm = torch.zeros(100, 3, dtype=torch.float64, device="cuda")
    gm[:, 1] = -1.0
    out = torch.empty(100, 6, device="cuda")
    F.query_backward(field.c, poses, fim, gm, out, F.Q_METRICS)
    torch.cuda.synchronize()
    assert torch.allclose(t.grad, out[:, :3]) and torch.allclose(phi.grad, out[:, 3:])
