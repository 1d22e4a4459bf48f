"""Full-size parity in the launch configuration bench.py times: the 200,000-landmark warehouse,
its 200 x 200 x 40 field built on the GPU, and one fif_query of 2^22 uniform-random poses (the
bench's pose stream); sampled poses spread over the whole batch (first and last groups
included) against the FP64 oracle, which builds their corner nodes from the landmarks.  FP32
and BF16 storage, and the GP-visibility field with N_s = 70 (the bench's GP block)."""
import numpy as np
import pytest
import torch

import oracle as O
from paper_2008_03324_gb300 import synth
from tests import _fixtures as X

pytestmark = pytest.mark.gpu
M = 1 << 22


@pytest.fixture(scope="module")
def F():
    from paper_2008_03324_gb300 import build as B
    B.build()
    from paper_2008_03324_gb300 import fif
    return fif


@pytest.fixture(scope="module")
def setup():
    sc = X.warehouse_scene()
    spec = X.WAREHOUSE["grid"]
    poses = synth.random_poses(1000, M, spec.lo, spec.hi)      # bench.py's timed pose stream
    rng = np.random.default_rng(17)
    sample = np.unique(np.concatenate([np.arange(40), M - 40 + np.arange(40), rng.choice(M, 176, replace=False)]))
    return sc, spec, poses, sample


def run_query(F, field, poses, flags):
    p = torch.from_numpy(poses).cuda()
    fim = torch.empty(M, 21, device="cuda")
    met = torch.empty(M, 3, dtype=torch.float64, device="cuda")
    sg = torch.empty(M, dtype=torch.int8, device="cuda")
    st = torch.empty(M, dtype=torch.int32, device="cuda")
    F.query(field.c, p, flags, fim, met, sg, st)
    torch.cuda.synchronize()
    assert F.device_error() == 0
    return fim, met, st


@pytest.mark.parametrize("storage", ["f32", "bf16"])
def test_warehouse_query_2m22_sampled(F, setup, storage):
    sc, spec, poses, sample = setup
    stor = F.STORAGE_F32 if storage == "f32" else F.STORAGE_BF16
    field = F.Field(spec.origin, spec.res, spec.dims, F.make_params(r_max=X.WAREHOUSE["r_max"]), storage=stor)
    field.build(torch.from_numpy(sc.landmarks).cuda())
    fim, met, st = run_query(F, field, poses, F.Q_METRICS)
    got = X.unpack21(fim[torch.from_numpy(sample).cuda()].cpu().numpy())
    prm = O.make_params(r_max=X.WAREHOUSE["r_max"])
    I_ref, st_ref, *_ = O.query_from_landmarks(sc.landmarks, X.oracle_grid(spec), prm, poses[sample])
    tau = X.TAU_F32 if storage == "f32" else X.TAU_BF16
    err = X.rel_fro(got, I_ref)
    assert err.max() <= tau, err.max()
    np.testing.assert_array_equal(st[torch.from_numpy(sample).cuda()].cpu().numpy() & 3, st_ref & 3)
    m = met[torch.from_numpy(sample).cuda()].cpu().numpy()
    if storage == "f32":
        mo = O.metrics(I_ref)
        t_tr, t_lm, _ = X.metric_tolerances(I_ref, tau)
        assert np.all(np.abs(m[:, 0] - mo[:, 0]) <= t_tr)
        assert np.all(np.abs(m[:, 2] - mo[:, 3]) <= t_lm)
    # the metric arithmetic alone, on the FIMs the launch returned (read back as float32 and
    # evaluated in FP64 by the oracle): lambda_min to 1e-9 ||I||, log|det| to 1e-12 ||I|| ||I^-1||
    I = got                     # the float32 FIM entries, exact in float64
    mo = O.metrics(I)
    n = X.fro(I)
    inv = np.array([X.fro(np.linalg.pinv(M)) for M in I])
    assert np.all(np.abs(m[:, 2] - mo[:, 3]) <= 1e-9 * n), np.max(np.abs(m[:, 2] - mo[:, 3]) / n)
    ok = mo[:, 2] != 0
    assert np.all(np.abs(m[ok, 1] - mo[ok, 1]) <= 1e-12 * n[ok] * inv[ok] + 5e-7)


def test_warehouse_gp_query_2m22_sampled(F, setup):
    """GP field (N_s = 70, length scale fitted as the bench does), 2^22 poses, 48 sampled poses
    against the oracle: corner coefficients from the oracle's sigmoid basis D (node frame), moved
    to the world frame and to the paper's basis C = W D (both exact, pinned on the CPU), then
    the oracle's GP query.  Tolerance as in tests/test_gpu_gp.py end to end: max(1e-5, 2e-5 kappa);
    then the oracle's D written into the field at those poses' corner nodes and the same launch
    again, within the query's own bounds: max(1e-5, 16 u kappa) with the single-precision
    contraction, max(1e-5, 2 u kappa) with the compensated one."""
    sc, spec, poses, sample = setup
    axes = synth.fibonacci_sphere(70)
    l = F.gp_fit_length_scale(axes, synth.sphere_points(7, 2000))
    gp = F.GPModel(axes, l)
    field = F.Field(spec.origin, spec.res, spec.dims, F.make_params(r_max=X.WAREHOUSE["r_max"]),
                    storage=F.STORAGE_GP, gp=gp)
    field.build(torch.from_numpy(sc.landmarks).cuda())
    fim, met, st = run_query(F, field, poses, F.Q_METRICS)
    sub = sample[np.linspace(0, len(sample) - 1, 48).astype(int)]
    got = X.unpack21(fim[torch.from_numpy(sub).cuda()].cpu().numpy())
    del fim, met, st
    ogp = O.GP(axes, l)
    grid = X.oracle_grid(spec)
    nodes, w, _, _ = O.query_cells(grid, poses[sub])
    uniq, inv = np.unique(nodes.reshape(-1), return_inverse=True)
    D = O.field_nodes_gp(sc.landmarks, grid, O.make_params(r_max=X.WAREHOUSE["r_max"]), ogp, uniq, about_node=True,
                         basis="sigmoid")
    nx, ny = spec.dims[0], spec.dims[1]
    # node coordinates exactly as the build and the oracle round them: fl(origin + fl(res * i))
    ijk = np.stack([uniq % nx, (uniq // nx) % ny, uniq // (nx * ny)], axis=1).astype(np.float32)
    c = (np.float32(spec.res) * ijk + np.asarray(spec.origin, np.float32)).astype(np.float64)
    Mc = np.tile(np.eye(6), (len(uniq), 1, 1))
    S = np.zeros((len(uniq), 3, 3))
    S[:, 0, 1], S[:, 0, 2], S[:, 1, 2] = -c[:, 2], c[:, 1], -c[:, 0]
    S[:, 1, 0], S[:, 2, 0], S[:, 2, 1] = c[:, 2], -c[:, 1], c[:, 0]
    Mc[:, :3, 3:] = -S
    Dw = np.einsum("nji,ngjk,nkl->ngil", Mc, D, Mc)
    Cw = np.einsum("gh,nhij->ngij", ogp.W, Dw)
    I_ref = O.query_gp(Cw[inv].reshape(len(sub), 8, 70, 6, 6), w, poses[sub], ogp)
    # kappa from the node-frame D, as in tests/test_gpu_gp.py
    Dn = np.sqrt((D ** 2).sum(axis=(2, 3)))
    kap = np.zeros(len(sub))
    for i, p in enumerate(poses[sub].astype(np.float64)):
        a = ogp.W @ ogp.vr(O.quat_to_rot(p[3:])[:, 2])
        s = 0.0
        for j in range(8):
            u = inv.reshape(len(sub), 8)[i, j]
            s += w[i, j] * (1 + np.linalg.norm(c[u] - p[:3])) ** 2 * (np.abs(a) @ Dn[u])
        kap[i] = s / max(X.fro(I_ref[i]), 1e-300)
    tau = np.maximum(X.TAU_F32, 2 * X.TAU_F32 * kap)
    err = X.rel_fro(got, I_ref)
    # the query's own arithmetic in the same 2^22-pose launch: the oracle's D written into the
    # field at every node these poses touch, bound max(1e-5, 2 u kappa) as in tests/test_gpu_gp.py
    from tests.test_gpu_gp import pack_gp
    field.coeffs[torch.from_numpy(uniq).cuda()] = torch.from_numpy(
        pack_gp(D, F.gp_row_stride(70), F.gp_stride(70))).cuda()
    u = 2.0 ** -24
    errs = {}
    for comp in (False, True):
        fim, _, _ = run_query(F, field, poses, F.Q_METRICS | (F.Q_GP_COMPENSATED if comp else 0))
        errs[comp] = X.rel_fro(X.unpack21(fim[torch.from_numpy(sub).cuda()].cpu().numpy()), I_ref)
        del fim
    del field
    torch.cuda.empty_cache()
    msg = (f"GP query N_s = 70, 2^22 poses, {len(sub)} sampled poses; kappa median {np.median(kap):.1f} p99 "
           f"{np.percentile(kap, 99):.1f} max {kap.max():.1f}; GPU build + query: error max {err.max():.2e} p99 "
           f"{np.percentile(err, 99):.2e} median {np.median(err):.2e}")
    for comp, e in errs.items():
        msg += (f"; oracle D + GPU query, {'compensated' if comp else 'single-precision'}: error max {e.max():.2e} "
                f"p99 {np.percentile(e, 99):.2e}, max error / (u kappa) {(e / (u * kap)).max():.2f}")
    print(msg)
    assert np.all(err <= tau), (err.max(), (err / tau).max())
    assert np.median(err) <= X.TAU_F32
    assert np.all(errs[False] <= np.maximum(X.TAU_F32, 16 * u * kap)), msg
    assert np.all(errs[True] <= np.maximum(X.TAU_F32, 2 * u * kap)), msg
