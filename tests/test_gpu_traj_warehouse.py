"""The differentiable trajectory batch at its full size on the warehouse field, and the query
adjoint on the warehouse lattice (lever arms up to 50 m from the world origin).

Batch: 256 cubic B-spline trajectories x 32 control positions x 128 samples (32,768 poses,
per-sample yaw, cameras looking horizontally) on the GPU-built 200 x 200 x 40 field of the
200,000-landmark warehouse at v_alpha = 0.8 -- the batch the benchmark times.  Objective:
sum of -log det I over the samples.  Checked against the FP64 oracle (Sec. VII-B uses the
metrics of sampled poses as the planner's cost; the derivative is the paper's differentiability
claim of Sec. I) at <= 1e-3 relative:
  * the adjoint's own arithmetic: the oracle's analytic gradient evaluated on the same stored
    (GPU-built) coefficients, for 512 sampled poses and for every pose of four trajectories;
  * end to end: the oracle gradient on oracle-built corner nodes, and central differences
    (step 1e-4) of the oracle objective, for control-point coordinates of those trajectories.
"""
import math

import numpy as np
import pytest
import torch

import oracle as O
from paper_2008_03324_gb300 import synth
from tests import _fixtures as X

pytestmark = pytest.mark.gpu
TOL = 1e-3
V_ALPHA = 0.8
R_MAX = 10.0


@pytest.fixture(scope="module")
def F():
    from paper_2008_03324_gb300 import build as B
    B.build()
    from paper_2008_03324_gb300 import fif
    return fif


@pytest.fixture(scope="module")
def wh(F):
    sc = X.warehouse_scene()
    spec = X.WAREHOUSE["grid"]
    field = F.Field(spec.origin, spec.res, spec.dims, F.make_params(r_max=R_MAX, v_alpha=V_ALPHA))
    field.build(torch.from_numpy(sc.landmarks).cuda())
    torch.cuda.synchronize()
    assert F.device_error() == 0
    nodes = X.OracleNodes(sc.landmarks, spec, O.make_params(r_max=R_MAX, v_alpha=V_ALPHA))
    return field, sc, spec, nodes


def stored_world(field, spec, nodes):
    """World-frame FP64 copy of the GPU-built coefficients of `nodes` [..., 8]."""
    nodes = np.asarray(nodes, dtype=np.int64)
    loc = X.unpack_field(field.coeffs[torch.from_numpy(nodes.reshape(-1)).cuda()].cpu().numpy())
    return X.local_to_world(loc, spec, nodes.reshape(-1)).reshape(nodes.shape + (10, 6, 6))


def rel_rows(a, b):
    return np.linalg.norm(a - b, axis=-1) / np.maximum(np.linalg.norm(b, axis=-1), 1e-300)


def test_trajectory_batch_full_size_on_warehouse_field(F, wh):
    from paper_2008_03324_gb300 import traj
    field, sc, spec, onodes = wh
    ctrl_np, yaw_np, basis_np = synth.bspline_batch(6, sc, 256, 32, 128)
    Bt = torch.from_numpy(basis_np.astype(np.float32)).cuda()
    yt = torch.from_numpy(yaw_np.astype(np.float32)).cuda()
    ct = torch.from_numpy(ctrl_np.astype(np.float32)).cuda().requires_grad_(True)
    loss, phi, met, sg = traj.neg_logdet_objective(ct, yt, Bt, field)
    loss.backward()
    torch.cuda.synchronize()
    assert F.device_error() == 0
    T, C, S = 256, 32, 128
    # the poses the library saw (the B-spline map runs in PyTorch, single precision)
    with torch.no_grad():
        t = torch.einsum("sc,tcd->tsd", Bt, ct).reshape(-1, 3)
        quat = traj.horizontal_quats((yt @ Bt.T).reshape(-1))
        poses_t = torch.cat([t, quat], 1).contiguous()
    poses = poses_t.cpu().numpy()
    mask_gpu = (sg > 0).cpu().numpy()
    # per-pose gradient of the objective from the adjoint kernel (what FifQuery's backward ran)
    fim, _, _, _ = field.query(poses_t)
    gm = np.zeros((T * S, 3))
    gm[mask_gpu, 1] = -1.0
    g_pose = torch.empty(T * S, 6, device="cuda")
    F.query_backward(field.c, poses_t, fim, torch.from_numpy(gm).cuda(), g_pose)
    torch.cuda.synchronize()
    g_pose = g_pose.cpu().numpy().astype(np.float64)
    assert np.array_equal(phi.grad.cpu().numpy(), g_pose[:, 3:].astype(np.float32))
    k = O.quad_coeffs(math.pi / 4, V_ALPHA)
    grid = X.oracle_grid(spec)

    # (1) the adjoint's arithmetic at full size: 512 sampled poses, oracle gradient on the stored field
    rng = np.random.default_rng(41)
    pick = np.sort(rng.choice(T * S, 512, replace=False))
    nodes, w, dw, _ = O.query_cells(grid, poses[pick])
    g_st = O.query_grad(stored_world(field, spec, nodes), w, dw, poses[pick], k, gm[pick])
    live = np.linalg.norm(g_st, axis=1) > 0
    assert live.sum() >= 400
    err = rel_rows(g_pose[pick][live], g_st[live])
    assert err.max() <= TOL, (err.max(), np.percentile(err, 99))

    # (2) end to end for four whole trajectories: the field at their corner nodes, the objective,
    # the per-pose and the control-point gradients against the oracle-built nodes
    trajs = np.array([3, 77, 150, 241])
    sel = (trajs[:, None] * S + np.arange(S)[None, :]).reshape(-1)
    corners, w, dw, nodes = onodes.corners(poses[sel])
    uniq = np.unique(nodes)
    got = X.unpack_field(field.coeffs[torch.from_numpy(uniq).cuda()].cpu().numpy())
    ref = onodes.local(uniq)
    assert X.rel_fro(got.reshape(-1, 60, 6), ref.reshape(-1, 60, 6)).max() <= X.TAU_F32
    I_ref = O.query(corners, w, poses[sel], k)
    m_ref = O.metrics(I_ref)
    mask_ref = m_ref[:, 2] > 0
    # the positive-definite decisions agree wherever the FIM is not numerically singular
    clear = np.abs(m_ref[:, 3]) > 1e-6 * np.abs(m_ref[:, 0])
    assert np.array_equal(mask_ref[clear], mask_gpu[sel][clear])
    met_sel = met.detach().cpu().numpy()[sel]
    _, _, t_ld = X.metric_tolerances(I_ref, X.TAU_F32)
    both = mask_ref & mask_gpu[sel]
    assert np.all(np.abs(met_sel[both, 1] - m_ref[both, 1]) <= t_ld[both])
    g_ref = O.query_grad(corners, w, dw, poses[sel], k, gm[sel])
    g_st4 = O.query_grad(stored_world(field, spec, nodes), w, dw, poses[sel], k, gm[sel])
    live = np.linalg.norm(g_ref, axis=1) > 0
    e_adj = rel_rows(g_pose[sel][live], g_st4[live])
    e_end = rel_rows(g_pose[sel][live], g_ref[live])
    assert e_adj.max() <= TOL, e_adj.max()
    # d loss / d ctrl = sum_s B[s, c] d loss / d t_s, per trajectory
    Bd = basis_np.astype(np.float64)
    gc = ct.grad.cpu().numpy().astype(np.float64)[trajs]
    gc_ref = np.einsum("sc,tsd->tcd", Bd, g_ref[:, :3].reshape(len(trajs), S, 3))
    e_ctrl = np.linalg.norm((gc - gc_ref).reshape(len(trajs), -1), axis=1) / np.linalg.norm(
        gc_ref.reshape(len(trajs), -1), axis=1)
    summary = (f"adjoint vs stored field: 512 sampled poses max {err.max():.2e}, four trajectories max "
               f"{e_adj.max():.2e}; vs oracle-built nodes: per pose max {e_end.max():.2e} (p99 "
               f"{np.percentile(e_end, 99):.2e}), control points {e_ctrl.max():.2e}")
    print(summary)
    assert e_ctrl.max() <= TOL, summary
    assert e_end.max() <= TOL, summary

    # (3) central differences (step 1e-4) of the FP64 oracle objective of one trajectory
    def objective(tr, ctrl_tr):
        tt = Bd @ ctrl_tr
        psi = Bd @ yaw_np[tr].astype(np.float32).astype(np.float64)
        ps = np.concatenate([tt, synth.horizontal_quats(psi)], axis=1)
        cn, ww, _, _ = onodes.corners(ps)
        mm = O.metrics(O.query(cn, ww, ps, k))
        ok = mm[:, 2] > 0
        return -mm[ok, 1].sum()

    h = 1e-4
    rng = np.random.default_rng(5)
    for i in range(6):
        ti = int(rng.integers(len(trajs)))
        tr, cc, dd = int(trajs[ti]), int(rng.integers(C)), int(rng.integers(3))
        base = ctrl_np[tr].astype(np.float32).astype(np.float64)
        cp, cm = base.copy(), base.copy()
        cp[cc, dd] += h
        cm[cc, dd] -= h
        fd = (objective(tr, cp) - objective(tr, cm)) / (2 * h)
        scale = np.abs(gc_ref[ti]).max()
        assert abs(gc[ti, cc, dd] - fd) <= TOL * max(abs(fd), 1e-2 * scale), (tr, cc, dd, gc[ti, cc, dd], fd)


@pytest.mark.parametrize("which", [0, 1, 2])
def test_adjoint_on_warehouse_poses(F, wh, which):
    """300 uniform warehouse poses, one metric at a time, camera frame: the adjoint against the
    oracle's analytic gradient.  The library's field holds the oracle-built coefficients of every
    node these poses touch (stored in single precision), so the comparison is the adjoint's own
    arithmetic at 50 m lever arms."""
    _, sc, spec, onodes = wh
    poses = synth.random_poses(88, 300, spec.lo, spec.hi)
    corners, w, dw, nodes = onodes.corners(poses)
    uniq = np.unique(nodes)
    field = F.Field(spec.origin, spec.res, spec.dims, F.make_params(r_max=R_MAX, v_alpha=V_ALPHA))
    field.coeffs[torch.from_numpy(uniq).cuda()] = torch.from_numpy(X.pack_field(onodes.local(uniq))).cuda()
    p = torch.from_numpy(poses).cuda()
    fim, met, sg, st = field.query(p)
    gm = np.zeros((300, 3))
    gm[:, which] = 1.0
    out = torch.empty(300, 6, device="cuda")
    F.query_backward(field.c, p, fim, torch.from_numpy(gm).cuda(), out)
    torch.cuda.synchronize()
    assert F.device_error() == 0
    g = out.cpu().numpy().astype(np.float64)
    k = O.quad_coeffs(math.pi / 4, V_ALPHA)
    # the oracle on the same single-precision coefficients
    stored = X.local_to_world(X.unpack_field(X.pack_field(onodes.local(nodes.reshape(-1)))), spec,
                              nodes.reshape(-1)).reshape(nodes.shape + (10, 6, 6))
    ref = O.query_grad(stored, w, dw, poses, k, gm)
    I_ref = O.query(stored, w, poses, k)
    ok = np.linalg.norm(ref, axis=1) > 0
    if which == 2:   # lambda_min's derivative needs a simple smallest eigenvalue
        ev = np.linalg.eigvalsh(I_ref)
        ok &= (ev[:, 1] - ev[:, 0]) > 1e-3 * np.abs(ev[:, 1])
    assert ok.sum() >= 150
    err = rel_rows(g[ok], ref[ok])
    assert err.max() <= TOL, (err.max(), np.percentile(err, 99))
    assert np.all(g[:, 5] == 0.0)
