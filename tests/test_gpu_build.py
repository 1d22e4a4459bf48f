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
