"""fif_build_static: the field build for callers that cannot allocate device memory while they
run (a planner plug-in inside an application that owns the GPU memory, a real-time loop that
forbids cudaMalloc after start-up).  Its scratch is a fixed array inside the library, so the
test checks, through the C ABI, that two calls in a row reproduce fif_build with a
caller-allocated workspace, and that an oversized request is refused without a launch.
This file is collected last so that a failure here leaves every other test already run."""
import ctypes

import numpy as np
import pytest
import torch

from tests import _fixtures as X

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def F():
    from paper_2008_03324_gb300 import build as B
    B.build()
    from paper_2008_03324_gb300 import fif
    return fif


def test_static_scratch_build_matches_workspace_build_twice(F):
    sc = X.room_scene()
    spec = X.ROOM["grid"]
    prm = F.make_params(r_max=X.ROOM["r_max"])
    lm = torch.from_numpy(sc.landmarks).cuda()
    ref = F.Field(spec.origin, spec.res, spec.dims, prm)
    ref.build(lm)                         # existing entry point, caller-owned workspace
    torch.cuda.synchronize()
    lib = F.lib()
    for _ in range(2):                    # the shared scratch keeps the previous call's contents
        out = F.Field(spec.origin, spec.res, spec.dims, prm)
        out.coeffs.fill_(7.0)
        stream = ctypes.c_void_p(torch.cuda.current_stream().cuda_stream)
        rc = lib.fif_build_static(ctypes.byref(out.c), ctypes.c_void_p(lm.data_ptr()), lm.shape[0], stream)
        assert rc == F.OK, F.status_str(rc)
        torch.cuda.synchronize()
        # the same kernels in the same order: bitwise the field of the workspace build, so no
        # contents of the previous call's scratch can leak into this one
        assert torch.equal(out.coeffs, ref.coeffs)
        got = X.unpack_field(out.coeffs.cpu().numpy()).reshape(-1, 60, 6)
        assert X.rel_fro(got, X.room_field_oracle(True).reshape(-1, 60, 6)).max() <= X.TAU_F32
        assert np.all(out.coeffs.cpu().numpy()[:, 210:] == 0)
    assert F.device_error() == 0


def test_static_scratch_refuses_oversized_request(F):
    spec = X.WAREHOUSE["grid"]
    fld = F.Field(spec.origin, spec.res, spec.dims, F.make_params(r_max=10.0))
    n = 2_000_000
    assert F.build_workspace_bytes(fld.c, n) > F.BUILD_STATIC_SCRATCH_BYTES
    lm = torch.zeros(n, 3, device="cuda")
    fld.coeffs.fill_(3.0)
    rc = F.lib().fif_build_static(ctypes.byref(fld.c), ctypes.c_void_p(lm.data_ptr()), n,
                                  ctypes.c_void_p(torch.cuda.current_stream().cuda_stream))
    assert rc == F.ERANGE
    torch.cuda.synchronize()
    assert torch.all(fld.coeffs == 3.0)   # nothing was launched


def test_static_scratch_refuses_gp_field(F):
    """A GP-visibility field is refused with FIF_EINVAL before anything runs."""
    from paper_2008_03324_gb300 import synth
    spec = X.ROOM["grid"]
    gp = F.GPModel(synth.fibonacci_sphere(30), 0.89754)
    fld = F.Field(spec.origin, spec.res, spec.dims, F.make_params(r_max=8.0), storage=F.STORAGE_GP, gp=gp)
    fld.coeffs.fill_(5.0)
    lm = torch.from_numpy(X.room_scene().landmarks).cuda()
    rc = F.lib().fif_build_static(ctypes.byref(fld.c), ctypes.c_void_p(lm.data_ptr()), lm.shape[0],
                                  ctypes.c_void_p(torch.cuda.current_stream().cuda_stream))
    assert rc == F.EINVAL
    torch.cuda.synchronize()
    assert torch.all(fld.coeffs == 5.0)
