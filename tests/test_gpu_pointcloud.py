"""GPU point-cloud FIM (fif_pointcloud_fim) against the FP64 oracle (Eq. cost_info with the
exact pinhole visibility of Eq. exact_vis_func; the visibility decision is taken in single
precision on both sides, so the visible sets agree exactly)."""
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


def gpu_pc(F, landmarks, poses, r_max, flags):
    lm = torch.from_numpy(np.ascontiguousarray(landmarks, np.float32)).cuda()
    p = torch.from_numpy(np.ascontiguousarray(poses, np.float32)).cuda()
    m = p.shape[0]
    fim = torch.empty(m, 21, device="cuda")
    met = torch.empty(m, 3, dtype=torch.float64, device="cuda")
    sg = torch.empty(m, dtype=torch.int8, device="cuda")
    st = torch.empty(m, dtype=torch.int32, device="cuda")
    F.pointcloud_fim(lm, F.make_params(r_max=r_max), F.make_pinhole(), p, flags, fim, met, sg, st)
    torch.cuda.synchronize()
    return fim.cpu().numpy(), met.cpu().numpy(), sg.cpu().numpy(), st.cpu().numpy()


@pytest.mark.parametrize("world", [False, True])
def test_room_pointcloud_matches_oracle(F, world):
    sc = X.room_scene()
    poses = X.room_poses(1000)
    flags = F.Q_METRICS | (F.Q_WORLD if world else 0)
    fim, met, sg, st = gpu_pc(F, sc.landmarks, poses, 8.0, flags)
    I_ref = O.pc_fim(sc.landmarks, poses, O.make_params(r_max=8.0), vis=O.VIS_PINHOLE,
                     frame=O.FRAME_WORLD if world else O.FRAME_CAMERA)
    nz = X.fro(I_ref) > 0
    err = X.rel_fro(X.unpack21(fim[nz]), I_ref[nz])
    assert err.max() <= X.TAU_F32, err.max()
    assert np.all(X.unpack21(fim[~nz]) == 0)
    mo = O.metrics(I_ref[nz])
    t_tr, t_lm, _ = X.metric_tolerances(I_ref[nz], X.TAU_F32)
    assert np.all(np.abs(met[nz, 0] - mo[:, 0]) <= t_tr)
    assert np.all(np.abs(met[nz, 2] - mo[:, 3]) <= t_lm)


def test_warehouse_pointcloud_full_map(F):
    sc = X.warehouse_scene()
    spec = X.WAREHOUSE["grid"]
    poses = synth.random_poses(41, 96, spec.lo, spec.hi)
    fim, met, sg, st = gpu_pc(F, sc.landmarks, poses, 10.0, F.Q_METRICS)
    I_ref = O.pc_fim(sc.landmarks, poses, O.make_params(r_max=10.0), vis=O.VIS_PINHOLE)
    nz = X.fro(I_ref) > 0
    assert X.rel_fro(X.unpack21(fim[nz]), I_ref[nz]).max() <= X.TAU_F32
    assert not np.any(st & F.POSE_OUTSIDE)


def test_pointcloud_ragged_landmark_count(F):
    """Landmark counts that are not a multiple of the tile (and the empty map)."""
    sc = X.room_scene()
    poses = X.room_poses(1000)[:40]
    for n in (0, 1, 511, 513, 1031):
        lm = sc.landmarks[:n]
        fim, met, sg, st = gpu_pc(F, lm if n else np.zeros((0, 3), np.float32), poses, 8.0, 0)
        I_ref = O.pc_fim(lm, poses, O.make_params(r_max=8.0), vis=O.VIS_PINHOLE) if n else np.zeros((40, 6, 6))
        nz = X.fro(I_ref) > 0
        if nz.any():
            assert X.rel_fro(X.unpack21(fim[nz]), I_ref[nz]).max() <= X.TAU_F32
        assert np.all(X.unpack21(fim[~nz]) == 0)
