"""Failure handling on the GPU without a fault: every device wait of the query and build kernels
is bounded, and a wait that runs out makes its block record FIF_ETIMEOUT, wait for the bulk copies
it has issued and return.  fif_set_wait_limit lowers the bound far below the time one hand-over
between warps takes, which forces that path in a real launch; the test then checks that the
device error word reads FIF_ETIMEOUT and that the same context still gives the oracle's results.
Nothing here traps, faults or waits without a bound."""
import numpy as np
import pytest
import torch

import oracle as O
from tests import _fixtures as X

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def F():
    from paper_2008_03324_gb300 import build as B
    B.build()
    from paper_2008_03324_gb300 import fif
    return fif


def _forced_timeout(F, fn):
    """Run fn with a 1 ns wait limit; return the device error word it left (then cleared)."""
    torch.cuda.synchronize()
    assert F.device_error() == 0
    F.set_wait_limit(1)
    try:
        fn()
        torch.cuda.synchronize()
    finally:
        F.set_wait_limit(0)
    return F.device_error()


@pytest.mark.parametrize("storage", [0, 1])
def test_query_wait_timeout_is_reported_and_the_context_recovers(F, storage):
    spec = X.ROOM["grid"]
    field = F.Field(spec.origin, spec.res, spec.dims, F.make_params(r_max=X.ROOM["r_max"]), storage=storage)
    field.build(torch.from_numpy(X.room_scene().landmarks).cuda())
    poses = X.room_poses(1000)
    p = torch.from_numpy(poses).cuda()
    # a metric warp waits tens of microseconds for its first group of 32 gathered poses
    assert _forced_timeout(F, lambda: field.query(p)) == F.ETIMEOUT
    fim, met, sg, st = field.query(p)
    torch.cuda.synchronize()
    assert F.device_error() == 0
    I_ref, *_ = O.query_from_landmarks(X.room_scene().landmarks, X.oracle_grid(spec),
                                       O.make_params(r_max=X.ROOM["r_max"]), poses)
    tau = X.TAU_F32 if storage == 0 else X.TAU_BF16
    assert X.rel_fro(X.unpack21(fim.cpu().numpy()), I_ref).max() <= tau


def test_build_wait_timeout_is_reported_and_the_context_recovers(F):
    spec = X.ROOM["grid"]
    lm = torch.from_numpy(X.room_scene().landmarks).cuda()
    field = F.Field(spec.origin, spec.res, spec.dims, F.make_params(r_max=X.ROOM["r_max"]))
    ws = torch.empty(F.build_workspace_bytes(field.c, lm.shape[0]), dtype=torch.uint8, device="cuda")
    # the landmark producer waits for the node warps to release a tile (microseconds of work)
    assert _forced_timeout(F, lambda: F.build(field.c, lm, ws)) == F.ETIMEOUT
    F.build(field.c, lm, ws)
    torch.cuda.synchronize()
    assert F.device_error() == 0
    got = X.unpack_field(field.coeffs.cpu().numpy())
    ref = X.room_field_oracle(True)
    assert X.rel_fro(got.reshape(-1, 60, 6), ref.reshape(-1, 60, 6)).max() <= X.TAU_F32
    # and bitwise the field of a build that never saw the short limit
    again = F.Field(spec.origin, spec.res, spec.dims, F.make_params(r_max=X.ROOM["r_max"]))
    again.build(lm)
    torch.cuda.synchronize()
    assert torch.equal(again.coeffs, field.coeffs)
