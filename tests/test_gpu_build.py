"""GPU field build (fif_build) against the FP64 oracle: every node of the room, 10,000
sampled nodes of the 200,000-landmark warehouse at the full 200 x 200 x 40 lattice (the
launch the benchmark times), a ragged lattice, the empty map, determinism, bfloat16 storage,
and an end-to-end build + query."""
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


def gpu_build(F, landmarks, spec, r_max, storage=0, bin_size=0.0):
    field = F.Field(spec.origin, spec.res, spec.dims, F.make_params(r_max=r_max, bin_size=bin_size), storage=storage)
    lm = torch.from_numpy(np.ascontiguousarray(landmarks, np.float32)).cuda()
    ws = field.build(lm)
    torch.cuda.synchronize()
    assert F.device_error() == 0
    return field, ws


def test_room_build_all_nodes(F):
    sc = X.room_scene()
    field, ws = gpu_build(F, sc.landmarks, X.ROOM["grid"], X.ROOM["r_max"])
    got = X.unpack_field(field.coeffs.cpu().numpy())
    ref = X.room_field_oracle(True)
    err = X.rel_fro(got.reshape(-1, 10 * 6, 6), ref.reshape(-1, 10 * 6, 6))
    assert err.max() <= X.TAU_F32, err.max()
    blk = X.block_ratio(got, ref, X.TAU_F32)
    assert blk.max() <= 1.0, (blk.max(), np.unravel_index(blk.argmax(), blk.shape))
    assert np.all(field.coeffs.cpu().numpy()[:, 210:] == 0)
    # the in-shell pair count is an integer decision taken identically on both sides
    grid = X.oracle_grid(X.ROOM["grid"])
    pairs = O.field_pairs(sc.landmarks, grid, O.make_params(r_max=X.ROOM["r_max"]), np.arange(field.n_nodes))
    assert F.build_stats(ws, field, len(sc.landmarks))[0] == pairs


def test_warehouse_build_sampled_nodes(F):
    sc = X.warehouse_scene()
    spec = X.WAREHOUSE["grid"]
    field, ws = gpu_build(F, sc.landmarks, spec, X.WAREHOUSE["r_max"])
    rng = np.random.default_rng(77)
    nodes = np.sort(rng.choice(spec.n_nodes, 10_000, replace=False))
    ref = O.field_nodes(sc.landmarks, X.oracle_grid(spec), O.make_params(r_max=X.WAREHOUSE["r_max"]), nodes,
                        about_node=True)
    got = X.unpack_field(field.coeffs[torch.from_numpy(nodes).cuda()].cpu().numpy())
    err = X.rel_fro(got.reshape(-1, 60, 6), ref.reshape(-1, 60, 6))
    assert err.max() <= X.TAU_F32, (err.max(), nodes[err.argmax()])
    blk = X.block_ratio(got, ref, X.TAU_F32)
    assert blk.max() <= 1.0, (blk.max(), np.unravel_index(blk.argmax(), blk.shape))
    inshell, cand, dropped = F.build_stats(ws, field, len(sc.landmarks))
    assert 0 < inshell <= cand and dropped == 0


@pytest.mark.parametrize("dims", [(5, 3, 6), (2, 2, 2), (9, 17, 5)])
def test_ragged_lattice(F, dims):
    rng = np.random.default_rng(sum(dims))
    lm = rng.uniform(-3, 6, size=(3000, 3)).astype(np.float32)
    spec = synth.GridSpec((0.25, -0.5, 0.0), 0.37, dims)
    field, _ = gpu_build(F, lm, spec, 4.0)
    ref = O.full_field(lm, X.oracle_grid(spec), O.make_params(r_max=4.0), about_node=True)
    got = X.unpack_field(field.coeffs.cpu().numpy())
    assert X.rel_fro(got.reshape(-1, 60, 6), ref.reshape(-1, 60, 6)).max() <= X.TAU_F32
    assert X.block_ratio(got, ref, X.TAU_F32).max() <= 1.0


def test_empty_map_and_far_landmarks(F):
    spec = X.ROOM["grid"]
    field, _ = gpu_build(F, np.zeros((0, 3), np.float32), spec, 8.0)
    assert torch.count_nonzero(field.coeffs) == 0
    far = np.array([[500.0, 0, 0], [0, -400.0, 0], [np.nan, 1, 1]], np.float32)
    field, ws = gpu_build(F, far, spec, 8.0)
    assert torch.count_nonzero(field.coeffs) == 0
    assert F.build_stats(ws, field, 3)[2] == 3


def test_build_is_deterministic_and_bin_size_independent(F):
    sc = X.room_scene()
    a, _ = gpu_build(F, sc.landmarks, X.ROOM["grid"], 8.0)
    b, _ = gpu_build(F, sc.landmarks, X.ROOM["grid"], 8.0)
    assert torch.equal(a.coeffs, b.coeffs)
    c, _ = gpu_build(F, sc.landmarks, X.ROOM["grid"], 8.0, bin_size=2.5)
    ref = X.room_field_oracle(True)
    got = X.unpack_field(c.coeffs.cpu().numpy())
    assert X.rel_fro(got.reshape(-1, 60, 6), ref.reshape(-1, 60, 6)).max() <= X.TAU_F32


def test_bf16_storage(F):
    sc = X.room_scene()
    field, _ = gpu_build(F, sc.landmarks, X.ROOM["grid"], 8.0, storage=F.STORAGE_BF16)
    got = X.unpack_field(field.coeffs.float().cpu().numpy())
    ref = X.room_field_oracle(True)
    assert X.rel_fro(got.reshape(-1, 60, 6), ref.reshape(-1, 60, 6)).max() <= X.TAU_BF16
    # each entry is rounded to bfloat16 on its own, so every block keeps the relative bound
    assert X.block_ratio(got, ref, X.TAU_BF16).max() <= 1.0


def test_end_to_end_warehouse_build_and_query(F):
    """GPU build + GPU query vs oracle build + oracle query on 400 random warehouse poses."""
    sc = X.warehouse_scene()
    spec = X.WAREHOUSE["grid"]
    field, _ = gpu_build(F, sc.landmarks, spec, X.WAREHOUSE["r_max"])
    poses = synth.random_poses(31, 400, spec.lo, spec.hi)
    p = torch.from_numpy(poses).cuda()
    fim, met, sg, st = field.query(p)
    torch.cuda.synchronize()
    prm = O.make_params(r_max=X.WAREHOUSE["r_max"])
    I_ref, st_ref, *_ = O.query_from_landmarks(sc.landmarks, X.oracle_grid(spec), prm, poses)
    err = X.rel_fro(X.unpack21(fim.cpu().numpy()), I_ref)
    assert err.max() <= X.TAU_F32, err.max()


def test_incremental_update_add_and_remove(F):
    """Sec. VI-A-1: adding or deleting landmarks adds or subtracts their terms.  build(A) then
    +B equals the oracle field of A u B; then -B returns to the oracle field of A."""
    sc = X.room_scene()
    A, Bm = sc.landmarks[:1400], sc.landmarks[1400:]
    spec = X.ROOM["grid"]
    field, ws = gpu_build(F, A, spec, 8.0)
    lmB = torch.from_numpy(np.ascontiguousarray(Bm)).cuda()
    ws_b = torch.empty(F.build_workspace_bytes(field.c, lmB.shape[0]), dtype=torch.uint8, device="cuda")
    F.build_update(field.c, lmB, +1, ws_b)
    torch.cuda.synchronize()
    ref_all = X.room_field_oracle(True)
    got = X.unpack_field(field.coeffs.cpu().numpy())
    assert X.rel_fro(got.reshape(-1, 60, 6), ref_all.reshape(-1, 60, 6)).max() <= X.TAU_F32
    F.build_update(field.c, lmB, -1, ws_b)
    torch.cuda.synchronize()
    ref_A = O.full_field(A, X.oracle_grid(spec), O.make_params(r_max=8.0), about_node=True)
    got = X.unpack_field(field.coeffs.cpu().numpy())
    assert X.rel_fro(got.reshape(-1, 60, 6), ref_A.reshape(-1, 60, 6)).max() <= 2 * X.TAU_F32
    assert F.device_error() == 0


def test_update_touches_only_nodes_in_reach(F):
    """A landmark far outside the lattice reaches no node: the update leaves the field bitwise
    unchanged; removing a landmark inside changes only nodes within r_max of it."""
    sc = X.room_scene()
    spec = X.ROOM["grid"]
    field, ws = gpu_build(F, sc.landmarks, spec, 3.0)
    before = field.coeffs.clone()
    far = torch.tensor([[60.0, 60.0, 60.0]], device="cuda")
    F.build_update(field.c, far, +1, ws)
    torch.cuda.synchronize()
    assert torch.equal(before, field.coeffs)
    one = torch.from_numpy(sc.landmarks[5:6].copy()).cuda()
    F.build_update(field.c, one, -1, ws)
    torch.cuda.synchronize()
    changed = (before != field.coeffs).any(dim=1).cpu().numpy()
    n = np.arange(spec.n_nodes)
    c = np.stack([spec.origin[0] + spec.res * (n % 21), spec.origin[1] + spec.res * ((n // 21) % 21),
                  spec.origin[2] + spec.res * (n // 441)], axis=1)
    d = np.linalg.norm(c - sc.landmarks[5].astype(np.float64), axis=1)
    assert not np.any(changed & (d > 3.0 + 1e-3))
    assert np.all(changed[(d < 2.9) & (d > 0.2)])


def test_trace_factor_field(F):
    """Sec. VI-A-2: the positional trace factor stores tr(C_k) of the world-frame coefficients
    (Eq. general_trace_pif), and the query v_r^T C_Tr (Eq. general_trace_query) is the trace of
    the world-frame FIM."""
    sc = X.room_scene()
    spec = X.ROOM["grid"]
    tf, _ = gpu_build(F, sc.landmarks, spec, 8.0, storage=F.STORAGE_TRACE)
    got = tf.coeffs.cpu().numpy()
    assert np.all(got[:, 10:] == 0)
    Fw = X.room_field_oracle(False)
    ref = np.trace(Fw, axis1=2, axis2=3)                        # [N, 10]
    err = np.linalg.norm(got[:, :10] - ref, axis=1) / np.linalg.norm(ref, axis=1)
    assert err.max() <= X.TAU_F32, err.max()
    poses = X.room_poses(1000)
    _, met, _, st = tf.query(torch.from_numpy(poses).cuda())
    torch.cuda.synchronize()
    grid = X.oracle_grid(spec)
    nodes, w, dw, _ = O.query_cells(grid, poses)
    I_w = O.query(Fw[nodes], w, poses, O.quad_coeffs(math.pi / 4, 0.5), O.FRAME_WORLD)
    t_tr, _, _ = X.metric_tolerances(I_w, X.TAU_F32)
    assert np.all(np.abs(met[:, 0].cpu().numpy() - np.trace(I_w, axis1=1, axis2=2)) <= t_tr)
    # same as the trace of the full field's world-frame query
    full, _ = gpu_build(F, sc.landmarks, spec, 8.0)
    _, met_full, _, _ = full.query(torch.from_numpy(poses).cuda(), F.Q_TRACE | F.Q_WORLD)
    torch.cuda.synchronize()
    assert np.all(np.abs(met[:, 0].cpu().numpy() - met_full[:, 0].cpu().numpy()) <= t_tr)
    # a batch of 40,000 poses (many groups of 32 and a ragged last one) with a non-finite pose,
    # one outside the lattice and one with an unnormalised quaternion: status bits and the
    # non-finite flag as the full query gives them, traces within the same bound
    many = X.room_poses(40_000)
    many[7, 0] = np.nan
    many[100, :3] = (-3.0, 50.0, 1.0)
    many[39_999, 3:] *= 1.5
    _, mt, _, stt = tf.query(torch.from_numpy(many).cuda())
    ff, mf, _, stf = full.query(torch.from_numpy(many).cuda(), F.Q_TRACE | F.Q_WORLD)
    torch.cuda.synchronize()
    mask = F.POSE_OUTSIDE | F.POSE_QUAT | F.POSE_NAN
    np.testing.assert_array_equal(stt.cpu().numpy() & mask, stf.cpu().numpy() & mask)
    assert stt[7].item() & F.POSE_NAN and stt[100].item() & F.POSE_OUTSIDE and stt[39_999].item() & F.POSE_QUAT
    a, b = mt[:, 0].cpu().numpy(), mf[:, 0].cpu().numpy()
    assert np.isnan(a[7]) and np.isnan(b[7])
    ok = np.isfinite(b)
    # both are within the FP32 metric bound of the exact trace, so within twice it of each other
    t_many, _, _ = X.metric_tolerances(X.unpack21(ff.cpu().numpy()[ok].astype(np.float64)), X.TAU_F32)
    assert np.all(np.abs(a[ok] - b[ok]) <= 2 * t_many)


@pytest.mark.parametrize("case", ["tall_room", "warehouse"])
def test_slab_builds_reproduce_the_whole_field_bitwise(F, case):
    """fif_build_slab (Sec. VI-A-1, nodes independent): z-slabs built apart, each from only the
    landmarks in its band, reproduce the whole-lattice build bitwise; nodes outside a slab keep
    their contents.  The bands cut the maps (range shells of 2.5 m and 3 m)."""
    from paper_2008_03324_gb300 import dist
    if case == "tall_room":
        spec = synth.GridSpec((0.0, 0.0, 0.0), 0.5, (9, 9, 25))
        lm_np = synth.room_landmarks(seed=4, n=4000, size=(4.0, 4.0, 12.0)).landmarks
        r_max, cuts = 2.5, [(0, 8), (8, 13), (13, 25)]
    else:
        spec = X.WAREHOUSE["grid"]
        lm_np = X.warehouse_scene().landmarks
        r_max, cuts = 3.0, dist.slab_ranges(spec.dims[2], 2)
    lm = torch.from_numpy(lm_np).cuda()
    whole, _ = gpu_build(F, lm_np, spec, r_max)
    slabbed = F.Field(spec.origin, spec.res, spec.dims, F.make_params(r_max=r_max))
    slabbed.coeffs.fill_(float("nan"))
    nxy = spec.dims[0] * spec.dims[1]
    for k0, k1 in cuts:
        band = F.slab_landmark_band(slabbed.c, k0, k1)
        sub = torch.from_numpy(np.ascontiguousarray(dist.slab_landmarks(lm_np, band))).cuda()
        assert sub.shape[0] < lm.shape[0]
        ws = torch.empty(F.build_workspace_bytes(slabbed.c, sub.shape[0]), dtype=torch.uint8, device="cuda")
        before = slabbed.coeffs.clone()
        F.build_slab(slabbed.c, k0, k1, sub, ws)
        torch.cuda.synchronize()
        assert F.device_error() == 0
        rows = slice(k0 * nxy, k1 * nxy)
        assert torch.equal(slabbed.coeffs[rows], whole.coeffs[rows])
        outside = torch.ones(spec.n_nodes, dtype=torch.bool, device="cuda")
        outside[rows] = False
        assert torch.equal(slabbed.coeffs[outside].isnan(), before[outside].isnan())
    assert torch.equal(slabbed.coeffs, whole.coeffs)
    with pytest.raises(F.FifError):
        F.build_slab(slabbed.c, 3, 3, lm, ws)
