"""Large map: 2,000,000 landmarks on a 100 x 100 x 20 m multi-room building, 400 x 400 x 80
nodes at 0.25 m (12.8M nodes, 11 GB in float32), r_max 12 m.  Sampled nodes of the GPU build
against the FP64 oracle (FP32 and BF16 storage), and an end-to-end query."""
import numpy as np
import pytest
import torch

import oracle as O
from paper_2008_03324_gb300 import synth
from tests import _fixtures as X

pytestmark = pytest.mark.gpu
R_MAX = 12.0


@pytest.fixture(scope="module")
def F():
    from paper_2008_03324_gb300 import build as B
    B.build()
    from paper_2008_03324_gb300 import fif
    return fif


@pytest.fixture(scope="module")
def scene():
    return synth.building(seed=5, n=2_000_000)


def test_large_map_build_and_query(F, scene):
    spec = synth.BUILDING_GRID
    lm = torch.from_numpy(scene.landmarks).cuda()
    field = F.Field(spec.origin, spec.res, spec.dims, F.make_params(r_max=R_MAX))
    ws = field.build(lm)
    torch.cuda.synchronize()
    assert F.device_error() == 0
    rng = np.random.default_rng(5)
    nodes = np.sort(rng.choice(spec.n_nodes, 1000, replace=False))
    grid = X.oracle_grid(spec)
    prm = O.make_params(r_max=R_MAX)
    ref = O.field_nodes(scene.landmarks, grid, prm, nodes, about_node=True)
    got = X.unpack_field(field.coeffs[torch.from_numpy(nodes).cuda()].cpu().numpy())
    nz = X.fro(ref.reshape(-1, 60, 6)) > 0
    assert X.rel_fro(got.reshape(-1, 60, 6)[nz], ref.reshape(-1, 60, 6)[nz]).max() <= X.TAU_F32
    assert X.block_ratio(got[nz], ref[nz], X.TAU_F32).max() <= 1.0
    inshell, cand, dropped = F.build_stats(ws, field, lm.shape[0])
    assert dropped == 0 and inshell > 1e11
    # end to end query of 150 poses in the building
    poses = synth.random_poses(71, 150, (0.2, 0.2, 0.2), (99.8, 99.8, 19.8))
    fim, met, sg, st = field.query(torch.from_numpy(poses).cuda())
    torch.cuda.synchronize()
    I_ref, *_ = O.query_from_landmarks(scene.landmarks, grid, prm, poses)
    assert X.rel_fro(X.unpack21(fim.cpu().numpy()), I_ref).max() <= X.TAU_F32
    del field, ws
    torch.cuda.empty_cache()
    # bfloat16 storage of the same map
    f16 = F.Field(spec.origin, spec.res, spec.dims, F.make_params(r_max=R_MAX), storage=F.STORAGE_BF16)
    f16.build(lm)
    got16 = X.unpack_field(f16.coeffs[torch.from_numpy(nodes[:200]).cuda()].float().cpu().numpy())
    nz16 = nz[:200]
    assert X.rel_fro(got16.reshape(-1, 60, 6)[nz16], ref[:200].reshape(-1, 60, 6)[nz16]).max() <= X.TAU_BF16
    assert X.block_ratio(got16[nz16], ref[:200][nz16], X.TAU_BF16).max() <= 1.0
