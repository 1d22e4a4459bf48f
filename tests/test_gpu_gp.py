"""GPU GP-visibility field (Sec. V-B-2) against the FP64 oracle: the build of the sigmoid-value
basis D_g on every node of the room and on sampled warehouse nodes, the query (kriging weights
in double precision, contraction, frame change, metrics) on an uploaded oracle field and end to
end, ragged batches, edge poses, the update path and determinism.

Tolerances.  The build stores D_g = sum_i v^s_g I_i, sums of positive weights: relative
Frobenius error <= 1e-5 per node, as for the quadratic field.  The query forms
I = sum_j w_j sum_g a_g(z) D_g(c_j) moved to the camera; storage rounding of D (unit roundoff
u = 2^-24) reaches I amplified by the contraction's condition number
    kappa = sum_j w_j (1 + |c_j - t|)^2 sum_g |a_g| ||D_g(c_j)||_F / ||I||_F
(the weights a_g change sign; (1 + |d|)^2 bounds the norm of the move by d).  Storage rounds
every entry of D by at most u/2 (u kappa / 2), the single-precision a_g by at most u/2 (another
u kappa / 2); the moves and the rotation that follow act on the contracted, already cancelled
matrices (errors of order u ||I||, inside the 1e-5 floor).  The default single-precision
contraction adds a summation error of a few u kappa: a pose passes within max(1e-5, 16 u kappa).
With FIF_Q_GP_COMPENSATED the contraction is a compensated dot product whose own error is of
order u ||I||: within max(1e-5, 2 u kappa).  End to end the per-node build error (<= 1e-5) is
amplified the same way: max(1e-5, 2e-5 kappa)."""
import functools
import math

import numpy as np
import pytest
import torch

import oracle as O
from paper_2008_03324_gb300 import synth
from tests import _fixtures as X
from tests.test_oracle_gp import FITTED

pytestmark = pytest.mark.gpu

U32 = 2.0 ** -24


@pytest.fixture(scope="module")
def F():
    from paper_2008_03324_gb300 import build as B
    B.build()
    from paper_2008_03324_gb300 import fif
    return fif


@functools.lru_cache(maxsize=None)
def ogp(ns):
    return O.GP(synth.fibonacci_sphere(ns), FITTED[ns])


def room_params(F=None):
    return (F.make_params if F else O.make_params)(r_max=X.ROOM["r_max"])


@functools.lru_cache(maxsize=None)
def room_D(ns):
    """Oracle sigmoid basis about each node, every node of the room: [N, ns, 6, 6]."""
    sc = X.room_scene()
    spec = X.ROOM["grid"]
    return O.field_nodes_gp(sc.landmarks, X.oracle_grid(spec), room_params(), ogp(ns), np.arange(spec.n_nodes),
                            about_node=True, basis="sigmoid")


def gp_model(F, ns):
    return F.GPModel(synth.fibonacci_sphere(ns), FITTED[ns])


def pack_gp(D, rs, stride):
    N, ns = D.shape[:2]
    out = np.zeros((N, stride), np.float32)
    vals = D[:, :, X.SYM_R, X.SYM_C]
    for e in range(21):
        out[:, e * rs:e * rs + ns] = vals[:, :, e]
    return out


def unpack_gp(buf, ns, rs):
    buf = np.asarray(buf, np.float64)
    vals = np.stack([buf[:, e * rs:e * rs + ns] for e in range(21)], axis=-1)    # [N, ns, 21]
    return X.unpack21(vals)


def node_rel_err(got, ref):
    d = np.sqrt(((got - ref) ** 2).sum(axis=(1, 2, 3)))
    return d / np.maximum(np.sqrt((ref ** 2).sum(axis=(1, 2, 3))), 1e-300)


def gp_field(F, ns, spec=None, r_max=None):
    spec = spec or X.ROOM["grid"]
    gp = gp_model(F, ns)
    prm = F.make_params(r_max=r_max or X.ROOM["r_max"])
    return F.Field(spec.origin, spec.res, spec.dims, prm, storage=F.STORAGE_GP, gp=gp)


def run(F, field, poses, flags=None):
    p = torch.from_numpy(np.ascontiguousarray(poses, np.float32)).cuda()
    fim, met, sg, st = field.query(p, F.Q_METRICS if flags is None else flags)
    torch.cuda.synchronize()
    assert F.device_error() == 0
    return fim.cpu().numpy(), met.cpu().numpy(), sg.cpu().numpy(), st.cpu().numpy()


def kappa(ns, poses, I_ref, interp=O.INTERP_TRILINEAR, world=False):
    """Condition number of the contraction for each pose (see the module docstring); in the
    world frame the corner matrices move to the origin instead of the camera position."""
    gp = ogp(ns)
    spec = X.ROOM["grid"]
    nodes, w, _, _ = O.query_cells(X.oracle_grid(spec), poses, interp)
    Dn = np.sqrt((room_D(ns) ** 2).sum(axis=(2, 3)))                       # [N, ns]
    nx, ny = spec.dims[0], spec.dims[1]
    out = np.zeros(len(poses))
    for i, p in enumerate(np.asarray(poses, np.float64)):
        R = O.quat_to_rot(p[3:])
        a = gp.W @ gp.vr(R[:, 2])
        s = 0.0
        for j in range(8):
            n = nodes[i, j]
            c = np.array([spec.origin[0] + spec.res * (n % nx), spec.origin[1] + spec.res * ((n // nx) % ny),
                          spec.origin[2] + spec.res * (n // (nx * ny))])
            d = c if world else c - p[:3]
            s += w[i, j] * (1 + np.linalg.norm(d)) ** 2 * (np.abs(a) @ Dn[n])
        out[i] = s / max(X.fro(I_ref[i]), 1e-300)
    return out


def check_metrics(I_ref, met, sg, tau):
    mo = O.metrics(I_ref)
    t_tr, t_lm, t_ld = X.metric_tolerances(I_ref, tau)
    assert np.all(np.abs(met[:, 0] - mo[:, 0]) <= t_tr)
    assert np.all(np.abs(met[:, 2] - mo[:, 3]) <= t_lm)
    ok = t_ld < 1.0
    assert np.all(np.abs(met[ok, 1] - mo[ok, 1]) <= t_ld[ok])
    np.testing.assert_array_equal(sg[ok], mo[ok, 2].astype(np.int8))


# ---------------------------------------------------------------------------
# build
# ---------------------------------------------------------------------------

@pytest.mark.parametrize("ns", [30, 50, 70])
def test_gp_build_room_all_nodes(F, ns):
    sc = X.room_scene()
    field = gp_field(F, ns)
    ws = field.build(torch.from_numpy(sc.landmarks).cuda())
    torch.cuda.synchronize()
    assert F.device_error() == 0
    rs, stride = F.gp_row_stride(ns), F.gp_stride(ns)
    buf = field.coeffs.cpu().numpy()
    err = node_rel_err(unpack_gp(buf, ns, rs), room_D(ns))
    assert err.max() <= X.TAU_F32, err.max()
    # pads are zero
    mask = np.ones(stride, bool)
    for e in range(21):
        mask[e * rs:e * rs + ns] = False
    assert np.all(buf[:, mask] == 0)
    spec = X.ROOM["grid"]
    pairs = O.field_pairs(sc.landmarks, X.oracle_grid(spec), room_params(), np.arange(spec.n_nodes))
    assert F.build_stats(ws, field, len(sc.landmarks))[0] == pairs


@pytest.mark.parametrize("ns", [12, 40, 65])
def test_gp_build_last_slot_packing(F, ns):
    """Sample counts whose last slot of 32 axes holds r <= 16 samples, so that slot takes
    32 // r landmarks per pass (12: two per pass in the only slot; 40: r = 8, four per pass;
    65: r = 1, 32 per pass): every node of the room against the oracle, pads zero, and the
    in-shell pair count exact.  The stored basis does not depend on the length scale."""
    sc = X.room_scene()
    spec = X.ROOM["grid"]
    axes = synth.fibonacci_sphere(ns)
    field = F.Field(spec.origin, spec.res, spec.dims, room_params(F), storage=F.STORAGE_GP, gp=F.GPModel(axes, 0.7))
    ws = field.build(torch.from_numpy(sc.landmarks).cuda())
    torch.cuda.synchronize()
    assert F.device_error() == 0
    rs, stride = F.gp_row_stride(ns), F.gp_stride(ns)
    buf = field.coeffs.cpu().numpy()
    ref = O.field_nodes_gp(sc.landmarks, X.oracle_grid(spec), room_params(), O.GP(axes, 0.7), np.arange(spec.n_nodes),
                           about_node=True, basis="sigmoid")
    err = node_rel_err(unpack_gp(buf, ns, rs), ref)
    assert err.max() <= X.TAU_F32, err.max()
    mask = np.ones(stride, bool)
    for e in range(21):
        mask[e * rs:e * rs + ns] = False
    assert np.all(buf[:, mask] == 0)
    pairs = O.field_pairs(sc.landmarks, X.oracle_grid(spec), room_params(), np.arange(spec.n_nodes))
    assert F.build_stats(ws, field, len(sc.landmarks))[0] == pairs


def test_gp_build_warehouse_sampled_nodes(F):
    ns = 30
    sc = X.warehouse_scene()
    spec = X.WAREHOUSE["grid"]
    field = gp_field(F, ns, spec, X.WAREHOUSE["r_max"])
    field.build(torch.from_numpy(sc.landmarks).cuda())
    torch.cuda.synchronize()
    assert F.device_error() == 0
    nodes = np.sort(np.random.default_rng(5).choice(spec.n_nodes, 300, replace=False))
    ref = O.field_nodes_gp(sc.landmarks, X.oracle_grid(spec), O.make_params(r_max=X.WAREHOUSE["r_max"]), ogp(ns),
                           nodes, about_node=True, basis="sigmoid")
    got = unpack_gp(field.coeffs[torch.from_numpy(nodes).cuda()].cpu().numpy(), ns, F.gp_row_stride(ns))
    err = node_rel_err(got, ref)
    assert err.max() <= X.TAU_F32, err.max()


@pytest.mark.parametrize("dims", [(5, 3, 6), (2, 2, 2)])
def test_gp_build_ragged_lattice_max_samples(F, dims):
    ns = 96
    rng = np.random.default_rng(sum(dims))
    lm = rng.uniform(-3, 6, size=(1500, 3)).astype(np.float32)
    spec = synth.GridSpec((0.25, -0.5, 0.0), 0.37, dims)
    gp = F.GPModel(synth.fibonacci_sphere(ns), 0.55)
    field = F.Field(spec.origin, spec.res, spec.dims, F.make_params(r_max=4.0), storage=F.STORAGE_GP, gp=gp)
    field.build(torch.from_numpy(lm).cuda())
    torch.cuda.synchronize()
    assert F.device_error() == 0
    ref = O.field_nodes_gp(lm, X.oracle_grid(spec), O.make_params(r_max=4.0), O.GP(synth.fibonacci_sphere(ns), 0.55),
                           np.arange(spec.n_nodes), about_node=True, basis="sigmoid")
    err = node_rel_err(unpack_gp(field.coeffs.cpu().numpy(), ns, F.gp_row_stride(ns)), ref)
    assert err.max() <= X.TAU_F32, err.max()


def test_gp_build_deterministic_and_update(F):
    """Equal inputs give bitwise equal fields; build(A) + update(+B) is the field of A u B and
    update(-B) returns to the field of A (Sec. VI-A-1)."""
    ns = 30
    sc = X.room_scene()
    a = gp_field(F, ns)
    b = gp_field(F, ns)
    a.build(torch.from_numpy(sc.landmarks).cuda())
    b.build(torch.from_numpy(sc.landmarks).cuda())
    torch.cuda.synchronize()
    assert torch.equal(a.coeffs, b.coeffs)
    A, Bm = sc.landmarks[:1400], sc.landmarks[1400:]
    f = gp_field(F, ns)
    ws = f.build(torch.from_numpy(np.ascontiguousarray(A)).cuda())
    lmB = torch.from_numpy(np.ascontiguousarray(Bm)).cuda()
    wsb = torch.empty(F.build_workspace_bytes(f.c, lmB.shape[0]), dtype=torch.uint8, device="cuda")
    F.build_update(f.c, lmB, +1, wsb)
    torch.cuda.synchronize()
    rs = F.gp_row_stride(ns)
    err = node_rel_err(unpack_gp(f.coeffs.cpu().numpy(), ns, rs), room_D(ns))
    assert err.max() <= X.TAU_F32
    F.build_update(f.c, lmB, -1, wsb)
    torch.cuda.synchronize()
    spec = X.ROOM["grid"]
    ref_A = O.field_nodes_gp(A, X.oracle_grid(spec), room_params(), ogp(ns), np.arange(spec.n_nodes),
                             about_node=True, basis="sigmoid")
    err = node_rel_err(unpack_gp(f.coeffs.cpu().numpy(), ns, rs), ref_A)
    assert err.max() <= 2 * X.TAU_F32
    assert F.device_error() == 0


# ---------------------------------------------------------------------------
# query
# ---------------------------------------------------------------------------

def uploaded(F, ns):
    field = gp_field(F, ns)
    buf = pack_gp(room_D(ns), F.gp_row_stride(ns), F.gp_stride(ns))
    field.coeffs.copy_(torch.from_numpy(buf))
    return field


def oracle_gp_query(ns, poses, frame=O.FRAME_CAMERA, interp=O.INTERP_TRILINEAR):
    sc = X.room_scene()
    I, st, _, _ = O.query_gp_from_landmarks(sc.landmarks, X.oracle_grid(X.ROOM["grid"]), room_params(), ogp(ns),
                                            poses, interp=interp, frame=frame)
    return I


@pytest.mark.parametrize("comp", [False, True])
@pytest.mark.parametrize("ns", [30, 70])
def test_gp_query_uploaded_room(F, ns, comp):
    """1000 random room poses (31 full groups of 32 and a ragged tail of 8) on the oracle's own
    D, camera frame: the query's arithmetic alone against the oracle's paper-basis query, with
    the single-precision and the compensated contraction."""
    field = uploaded(F, ns)
    poses = X.room_poses(1000)
    fim, met, sg, st = run(F, field, poses, F.Q_METRICS | (F.Q_GP_COMPENSATED if comp else 0))
    I_ref = oracle_gp_query(ns, poses)
    kap = kappa(ns, poses, I_ref)
    tau = np.maximum(X.TAU_F32, (2 if comp else 16) * U32 * kap)
    err = X.rel_fro(X.unpack21(fim), I_ref)
    big = kap > X.TAU_F32 / U32 / 16        # poses whose kappa term exceeds the 1e-5 floor at 16 u
    print(f"GP query N_s = {ns}, oracle D uploaded, {'compensated' if comp else 'single-precision'} "
          f"contraction: error max {err.max():.2e} p99 {np.percentile(err, 99):.2e}; kappa median "
          f"{np.median(kap):.1f} p99 {np.percentile(kap, 99):.1f} max {kap.max():.1f}; error / (u kappa) max "
          f"{(err / (U32 * kap)).max():.2f}, over the {int(big.sum())} poses with kappa > {X.TAU_F32 / U32 / 16:.0f}: "
          f"{(err[big] / (U32 * kap[big])).max() if big.any() else 0:.2f}")
    assert np.all(err <= tau), (err.max(), (err / tau).max())
    assert np.median(err) <= X.TAU_F32
    check_metrics(I_ref, met, sg, tau)


def test_gp_query_world_frame_and_nearest(F):
    ns = 50
    field = uploaded(F, ns)
    poses = X.room_poses(1000)[:300]
    fim, *_ = run(F, field, poses, F.Q_METRICS | F.Q_WORLD)
    I_ref = oracle_gp_query(ns, poses, frame=O.FRAME_WORLD)
    tau = np.maximum(X.TAU_F32, 16 * U32 * kappa(ns, poses, I_ref, world=True))
    assert np.all(X.rel_fro(X.unpack21(fim), I_ref) <= tau)
    fim, met, sg, _ = run(F, field, poses, F.Q_METRICS | F.Q_NEAREST)
    I_ref = oracle_gp_query(ns, poses, interp=O.INTERP_NEAREST)
    tau = np.maximum(X.TAU_F32, 16 * U32 * kappa(ns, poses, I_ref, O.INTERP_NEAREST))
    assert np.all(X.rel_fro(X.unpack21(fim), I_ref) <= tau)


@pytest.mark.parametrize("m", [1, 31, 33, 97])
def test_gp_query_ragged_batches(F, m):
    ns = 30
    field = uploaded(F, ns)
    poses = X.room_poses(1000)[-m:]
    fim, *_ = run(F, field, poses)
    I_ref = oracle_gp_query(ns, poses)
    tau = np.maximum(X.TAU_F32, 16 * U32 * kappa(ns, poses, I_ref))
    assert np.all(X.rel_fro(X.unpack21(fim), I_ref) <= tau)


def test_gp_query_edge_poses_and_empty_batch(F):
    ns = 30
    field = uploaded(F, ns)
    poses = np.array([
        [-1.0, 5.0, 1.0, 1, 0, 0, 0],
        [10.0, 10.0, 3.0, 0.3, 0.5, -0.2, 0.7],
        [4.2, 3.3, 1.1, 2.0, 0.0, 0.0, 0.0],
        [np.nan, 1.0, 1.0, 1, 0, 0, 0],
        [12.0, -3.0, 7.0, 0.1, 0.9, 0.3, -0.2],
    ], np.float32)
    fim, met, sg, st = run(F, field, poses)
    good = [0, 1, 2, 4]
    I_ref = oracle_gp_query(ns, poses[good])
    tau = np.maximum(X.TAU_F32, 16 * U32 * kappa(ns, poses[good], I_ref))
    assert np.all(X.rel_fro(X.unpack21(fim[good]), I_ref) <= tau)
    assert st[0] & F.POSE_OUTSIDE and st[4] & F.POSE_OUTSIDE and not (st[1] & F.POSE_OUTSIDE)
    assert st[2] & F.POSE_QUAT
    assert st[3] & F.POSE_NAN and np.all(np.isnan(fim[3])) and np.all(np.isnan(met[3]))
    empty = torch.empty(0, 7, device="cuda")
    F.query(field.c, empty, F.Q_METRICS, None, torch.empty(0, 3, dtype=torch.float64, device="cuda"), None, None)
    torch.cuda.synchronize()


def test_gp_query_deterministic_and_backward_rejected(F):
    field = uploaded(F, 30)
    p = torch.from_numpy(X.room_poses(1000)).cuda()
    a = field.query(p)
    b = field.query(p)
    for x, y in zip(a, b):
        assert torch.equal(x.nan_to_num(), y.nan_to_num())
    fim, *_ = a
    g = torch.ones(p.shape[0], 3, dtype=torch.float64, device="cuda")
    out = torch.empty(p.shape[0], 6, device="cuda")
    with pytest.raises(F.FifError):
        F.query_backward(field.c, p, fim, g, out)


@pytest.mark.parametrize("ns", [30, 70])
def test_gp_build_and_query_end_to_end(F, ns):
    """GPU build + GPU query against the oracle field + oracle query, and at node positions
    against the GP-weighted point-cloud sum (Eq. fim_separation)."""
    sc = X.room_scene()
    field = gp_field(F, ns)
    field.build(torch.from_numpy(sc.landmarks).cuda())
    poses = X.room_poses(1000)[:400]
    fim, met, sg, st = run(F, field, poses)
    I_ref = oracle_gp_query(ns, poses)
    tau = np.maximum(X.TAU_F32, 2 * X.TAU_F32 * kappa(ns, poses, I_ref))
    err = X.rel_fro(X.unpack21(fim), I_ref)
    assert np.all(err <= tau), (err.max(), (err / tau).max())
    rng = np.random.default_rng(9)
    spec = X.ROOM["grid"]
    idx = rng.integers(0, [21, 21, 7], size=(20, 3))
    q = rng.standard_normal((20, 4))
    q /= np.linalg.norm(q, axis=1, keepdims=True)
    at_nodes = np.concatenate([spec.res * idx + np.array(spec.origin), q], axis=1).astype(np.float32)
    fim, *_ = run(F, field, at_nodes)
    ref = O.pc_fim_gp(sc.landmarks, at_nodes, room_params(), ogp(ns))
    tau = np.maximum(X.TAU_F32, 2 * X.TAU_F32 * kappa(ns, at_nodes, ref))
    assert np.all(X.rel_fro(X.unpack21(fim), ref) <= tau)


def test_gp_query_host_matches_device(F):
    """fif_query_host on a GP field (N_s = 30): page-locked buffers queried in place, and pageable
    ones in chunks through device staging, give every pose the device results bitwise."""
    field = uploaded(F, 30)
    poses = X.room_poses(300)
    fim, met, sg, st = run(F, field, poses)
    staging = torch.empty(F.query_host_staging_bytes(128), dtype=torch.uint8, device="cuda")
    for pinned in (True, False):
        pin = (lambda t: t.pin_memory()) if pinned else (lambda t: t)
        h = pin(torch.from_numpy(np.ascontiguousarray(poses, np.float32)))
        h_fim = pin(torch.empty(len(poses), 21, dtype=torch.float32))
        h_met = pin(torch.empty(len(poses), 3, dtype=torch.float64))
        h_sg = pin(torch.empty(len(poses), dtype=torch.int8))
        h_st = pin(torch.empty(len(poses), dtype=torch.int32))
        F.query_host(field.c, h, F.Q_METRICS, h_fim, h_met, h_sg, h_st, chunk=128, staging=staging,
                     copy_stream=torch.cuda.Stream())
        torch.cuda.current_stream().synchronize()
        np.testing.assert_array_equal(h_fim.numpy(), fim)
        np.testing.assert_array_equal(h_met.numpy(), met)
        np.testing.assert_array_equal(h_sg.numpy(), sg)
        np.testing.assert_array_equal(h_st.numpy(), st)
