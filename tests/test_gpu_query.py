"""GPU query (fif_query) against the FP64 oracle, element by element on the same seeded
inputs: the 10 x 10 x 3 m room (21 x 21 x 7 nodes at 0.5 m, 2000 landmarks, 1000 poses --
a ragged tail of 8 past 31 full groups of 32), plus edge cases."""
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


def uploaded_room_field(F, v_alpha=0.5, storage=0):
    spec = X.ROOM["grid"]
    field = F.Field(spec.origin, spec.res, spec.dims, F.make_params(r_max=X.ROOM["r_max"], v_alpha=v_alpha),
                    storage=storage)
    buf = X.pack_field(X.room_field_oracle(True), stride=field.coeffs.shape[1])
    field.coeffs.copy_(torch.from_numpy(buf).to(field.coeffs.dtype))
    return field


def oracle_query(poses, v_alpha=0.5, frame=O.FRAME_CAMERA, interp=O.INTERP_TRILINEAR):
    grid = X.oracle_grid(X.ROOM["grid"])
    nodes, w, dw, st = O.query_cells(grid, poses, interp)
    k = O.quad_coeffs(math.pi / 4, v_alpha)
    I = O.query(X.room_field_oracle(False)[nodes], w, poses, k, frame)
    return I, st


def run(F, field, poses, flags=None):
    p = torch.from_numpy(np.ascontiguousarray(poses, np.float32)).cuda()
    fim, met, sg, st = field.query(p, F.Q_METRICS if flags is None else flags)
    torch.cuda.synchronize()
    return fim.cpu().numpy(), met.cpu().numpy(), sg.cpu().numpy(), st.cpu().numpy()


def check_metrics(I_ref, met, sg, tau, check_sign=True):
    mo = O.metrics(I_ref)
    t_tr, t_lm, t_ld = X.metric_tolerances(I_ref, tau)
    assert np.all(np.abs(met[:, 0] - mo[:, 0]) <= t_tr)
    assert np.all(np.abs(met[:, 2] - mo[:, 3]) <= t_lm)
    ok = t_ld < 1.0   # log|det| is meaningful where the FIM is not near-singular
    assert np.all(np.abs(met[ok, 1] - mo[ok, 1]) <= t_ld[ok])
    if check_sign:
        np.testing.assert_array_equal(sg[ok], mo[ok, 2].astype(np.int8))


@pytest.mark.parametrize("v_alpha", [0.5, 0.8])
def test_room_query_matches_oracle(F, v_alpha):
    field = uploaded_room_field(F, v_alpha)
    poses = X.room_poses(1000)
    fim, met, sg, st = run(F, field, poses)
    I_ref, st_ref = oracle_query(poses, v_alpha)
    err = X.rel_fro(X.unpack21(fim), I_ref)
    assert err.max() <= X.TAU_F32, err.max()
    check_metrics(I_ref, met, sg, X.TAU_F32)
    np.testing.assert_array_equal(st & F.POSE_OUTSIDE, st_ref)


def test_world_frame_and_nearest(F):
    field = uploaded_room_field(F)
    poses = X.room_poses(1000)[:300]
    fim, met, sg, st = run(F, field, poses, F.Q_METRICS | F.Q_WORLD)
    I_ref, _ = oracle_query(poses, frame=O.FRAME_WORLD)
    assert X.rel_fro(X.unpack21(fim), I_ref).max() <= X.TAU_F32
    fim, met, sg, st = run(F, field, poses, F.Q_METRICS | F.Q_NEAREST)
    I_ref, _ = oracle_query(poses, interp=O.INTERP_NEAREST)
    assert X.rel_fro(X.unpack21(fim), I_ref).max() <= X.TAU_F32
    check_metrics(I_ref, met, sg, X.TAU_F32)


@pytest.mark.parametrize("m", [1, 31, 32, 33, 65])
def test_ragged_batch_sizes(F, m):
    field = uploaded_room_field(F)
    poses = X.room_poses(1000)[:m]
    fim, met, sg, st = run(F, field, poses)
    I_ref, _ = oracle_query(poses)
    assert X.rel_fro(X.unpack21(fim), I_ref).max() <= X.TAU_F32


def test_edge_poses(F):
    """Outside the lattice (clamped, status bit), exactly on the last node, a non-unit
    quaternion (renormalised, status bit) and a NaN pose (NaN outputs, status bit)."""
    field = uploaded_room_field(F)
    poses = np.array([
        [-1.0, 5.0, 1.0, 1, 0, 0, 0],
        [10.0, 10.0, 3.0, 0.3, 0.5, -0.2, 0.7],
        [4.2, 3.3, 1.1, 2.0, 0.0, 0.0, 0.0],
        [np.nan, 1.0, 1.0, 1, 0, 0, 0],
        [12.0, -3.0, 7.0, 0.1, 0.9, 0.3, -0.2],
    ], np.float32)
    fim, met, sg, st = run(F, field, poses)
    I_ref, st_ref = oracle_query(poses[[0, 1, 2, 4]])
    good = [0, 1, 2, 4]
    assert X.rel_fro(X.unpack21(fim[good]), I_ref).max() <= X.TAU_F32
    assert st[0] & F.POSE_OUTSIDE and st[4] & F.POSE_OUTSIDE
    assert not (st[1] & F.POSE_OUTSIDE)
    assert st[2] & F.POSE_QUAT
    assert st[3] & F.POSE_NAN and np.all(np.isnan(fim[3])) and np.all(np.isnan(met[3]))


def test_metric_subsets_and_optional_outputs(F):
    field = uploaded_room_field(F)
    poses = torch.from_numpy(X.room_poses(1000)[:100]).cuda()
    fim_all, met_all, _, _ = field.query(poses, F.Q_METRICS)
    met = torch.full((100, 3), -7.0, dtype=torch.float64, device="cuda")
    F.query(field.c, poses, F.Q_TRACE, None, met, None, None)
    torch.cuda.synchronize()
    assert torch.equal(met[:, 0], met_all[:, 0])
    assert torch.all(met[:, 1:] == -7.0)
    fim = torch.empty(100, 21, device="cuda")
    F.query(field.c, poses, 0, fim, None, None, None)
    torch.cuda.synchronize()
    assert torch.equal(fim, fim_all)


def test_query_is_deterministic(F):
    field = uploaded_room_field(F)
    poses = torch.from_numpy(X.room_poses(1000)).cuda()
    a = field.query(poses)
    b = field.query(poses)
    for x, y in zip(a, b):
        assert torch.equal(x.nan_to_num(), y.nan_to_num())


def test_bf16_storage_query_exact_arithmetic(F):
    """BF16 storage: upload the oracle field rounded to bfloat16, then the GPU query must match the
    FP64 oracle query of that same rounded field at the FP32 bound (only the storage rounds)."""
    spec = X.ROOM["grid"]
    F_loc = X.round_bf16(X.room_field_oracle(True))
    field = F.Field(spec.origin, spec.res, spec.dims, F.make_params(r_max=8.0), storage=F.STORAGE_BF16)
    buf = X.pack_field(F_loc, 224)
    field.coeffs.copy_(torch.from_numpy(buf).to(torch.bfloat16))
    poses = X.room_poses(1000)
    fim, met, sg, st = run(F, field, poses)
    Fw = X.local_to_world(F_loc, spec)
    grid = X.oracle_grid(spec)
    nodes, w, dw, _ = O.query_cells(grid, poses)
    I_ref = O.query(Fw[nodes], w, poses, O.quad_coeffs(math.pi / 4, 0.5))
    assert X.rel_fro(X.unpack21(fim), I_ref).max() <= X.TAU_F32


def test_bf16_build_and_query_vs_fp64_oracle(F):
    """BF16 end to end (GPU build into bfloat16 storage, GPU query) vs the FP64 oracle: <= 1e-2."""
    sc = X.room_scene()
    spec = X.ROOM["grid"]
    field = F.Field(spec.origin, spec.res, spec.dims, F.make_params(r_max=8.0), storage=F.STORAGE_BF16)
    field.build(torch.from_numpy(sc.landmarks).cuda())
    poses = X.room_poses(1000)
    fim, met, sg, st = run(F, field, poses)
    I_ref, _ = oracle_query(poses)
    assert X.rel_fro(X.unpack21(fim), I_ref).max() <= X.TAU_BF16


@pytest.mark.parametrize("storage", [0, 1])
def test_metrics_of_the_returned_fim(F, storage):
    """The metric arithmetic alone: log|det|, its sign and lambda_min of the FIM the kernel
    returned (read back as float32 and evaluated in FP64 by the oracle) agree to double
    precision -- log|det| within 1e-12 ||I|| ||I^-1|| + 5e-7, lambda_min within 1e-9 ||I||
    (single-precision inverse iteration for the eigenvector, double-precision Rayleigh quotient)."""
    field = uploaded_room_field(F, storage=storage)
    fim, met, sg, st = run(F, field, X.room_poses(1000))
    I = X.unpack21(fim)
    mo = O.metrics(I)
    n = X.fro(I)
    inv = np.array([X.fro(np.linalg.pinv(M)) for M in I])
    ok = mo[:, 2] != 0
    assert np.all(np.abs(met[ok, 1] - mo[ok, 1]) <= 1e-12 * n[ok] * inv[ok] + 5e-7)
    np.testing.assert_array_equal(sg[ok], mo[ok, 2].astype(np.int8))
    assert np.all(np.abs(met[:, 2] - mo[:, 3]) <= 1e-9 * n)
    assert np.all(np.abs(met[:, 0] - np.trace(I, axis1=1, axis2=2)) <= 1e-6 * n)


@pytest.mark.parametrize("storage", [0, 1])
def test_query_host_matches_device(F, storage):
    """fif_query_host (page-locked host buffers queried in place; pageable ones in chunks
    double-buffered through device staging, copies on a second stream) gives every pose exactly
    the results fif_query gives it on the device:
    a ragged last chunk, a chunk larger than the batch, a subset of the outputs, the empty
    batch and the argument checks."""
    field = uploaded_room_field(F, storage=storage)
    poses = X.room_poses(3000)[:2517]
    fim, met, sg, st = run(F, field, poses)
    h_poses = torch.from_numpy(np.ascontiguousarray(poses, np.float32)).pin_memory()
    cs = torch.cuda.Stream()
    # page-locked buffers are queried in place; pageable ones go through the staged chunks
    for pinned, chunk in ((True, 700), (False, 64), (False, 700), (False, 4096)):
        pin = (lambda t: t.pin_memory()) if pinned else (lambda t: t)
        hp = h_poses if pinned else h_poses.clone()
        staging = torch.empty(F.query_host_staging_bytes(chunk), dtype=torch.uint8, device="cuda")
        h_fim = pin(torch.full((len(poses), 21), np.nan, dtype=torch.float32))
        h_met = pin(torch.full((len(poses), 3), np.nan, dtype=torch.float64))
        h_sg = pin(torch.zeros(len(poses), dtype=torch.int8))
        h_st = pin(torch.full((len(poses),), -1, dtype=torch.int32))
        F.query_host(field.c, hp, F.Q_METRICS, h_fim, h_met, h_sg, h_st, chunk=chunk, staging=staging,
                     copy_stream=cs)
        torch.cuda.current_stream().synchronize()
        assert F.device_error() == 0
        np.testing.assert_array_equal(h_fim.numpy(), fim)
        np.testing.assert_array_equal(h_met.numpy(), met)
        np.testing.assert_array_equal(h_sg.numpy(), sg)
        np.testing.assert_array_equal(h_st.numpy(), st)
    # metrics only (no FIM buffer), chunk of 512
    staging = torch.empty(F.query_host_staging_bytes(512), dtype=torch.uint8, device="cuda")
    h_met = torch.full((len(poses), 3), np.nan, dtype=torch.float64).pin_memory()
    F.query_host(field.c, h_poses, F.Q_METRICS, None, h_met, None, None, chunk=512, staging=staging, copy_stream=cs)
    torch.cuda.current_stream().synchronize()
    np.testing.assert_array_equal(h_met.numpy(), met)
    # empty batch, undersized staging, the same stream twice
    F.query_host(field.c, h_poses[:0], F.Q_METRICS, None, h_met[:0], None, None, chunk=512, staging=staging,
                 copy_stream=cs)
    with pytest.raises(F.FifError):
        F.query_host(field.c, h_poses, F.Q_METRICS, None, h_met, None, None, chunk=4096, staging=staging,
                     copy_stream=cs)
    with pytest.raises(F.FifError):
        F.query_host(field.c, h_poses, F.Q_METRICS, None, h_met, None, None, chunk=512, staging=staging,
                     copy_stream=torch.cuda.current_stream())


def test_fma_probe_runs(F):
    """The benchmark's FP32 FMA throughput probe (measurement infrastructure, its own library)
    runs in both forms and leaves finite values; bad arguments are rejected."""
    import bench
    sink = torch.full((4 * 256,), float("nan"), device="cuda")
    stream = torch.cuda.current_stream()
    for packed in (False, True):
        bench.fma_probe(sink, 4, 1000, packed, stream)
        torch.cuda.synchronize()
        assert bool(torch.isfinite(sink).all())
    P = bench.probe_lib()
    assert P.fif_fma_probe(None, 4, 10, 0, None) == F.EINVAL
    assert P.fif_fma_probe(sink.data_ptr(), 4, 0, 0, None) == F.EINVAL


def test_c_client_runs(F, tmp_path):
    """A plain C client of the library (tests/abi_client.c) builds a field, queries it through
    host and device buffers, and finds the two bitwise equal."""
    import subprocess
    exe = X.build_c_client(tmp_path)
    r = subprocess.run([exe], capture_output=True, text=True, timeout=120)
    assert r.returncode == 0, r.stderr
    assert "abi client ok" in r.stdout


@pytest.mark.parametrize("storage", [0, 1])
def test_field_save_load_round_trip(F, tmp_path, storage):
    """fif_field_save / fif_field_load (the field as a file: header + coefficient blob + checksum):
    the loaded field has the same coefficients and answers queries bitwise alike; a corrupted
    payload is refused."""
    field = uploaded_room_field(F, storage=storage)
    path = str(tmp_path / "room.fif")
    F.field_save(field.c, path)
    coeffs = torch.empty_like(field.coeffs)
    fc = F.field_load(path, coeffs)
    torch.cuda.synchronize()
    assert torch.equal(coeffs, field.coeffs)
    assert fc.storage == field.c.storage and fc.stride == field.c.stride
    p = torch.from_numpy(np.ascontiguousarray(X.room_poses(200), np.float32)).cuda()
    outs = []
    for fcs in (field.c, fc):
        met = torch.empty(200, 3, dtype=torch.float64, device="cuda")
        fim = torch.empty(200, 21, device="cuda")
        F.query(fcs, p, F.Q_METRICS, fim, met, None, None)
        outs.append((fim.cpu(), met.cpu()))
    torch.cuda.synchronize()
    assert torch.equal(outs[0][0], outs[1][0]) and torch.equal(outs[0][1], outs[1][1])
    data = bytearray(open(path, "rb").read())
    data[-1] ^= 0xFF
    bad = str(tmp_path / "bad.fif")
    open(bad, "wb").write(bytes(data))
    with pytest.raises(F.FifError):
        F.field_load(bad, coeffs)
