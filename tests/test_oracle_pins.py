"""Pins of the FP64 oracle against what the paper and the mathematics fix.

No GPU.  Each test compares the oracle with something other than itself: a closed form,
finite differences, a brute-force evaluation of the paper's explicit matrices, a
textbook library routine, or an invariant the derivation implies.  The docstrings cite
the passage that fixes the expected value."""
import math

import numpy as np
import pytest

import oracle as O
from paper_2008_03324_gb300 import synth
from tests import _np_geom as G

RNG = np.random.default_rng(12345)


def rand_unit(n=None):
    v = RNG.standard_normal(3 if n is None else (n, 3))
    return v / np.linalg.norm(v, axis=-1, keepdims=True)


def rand_R():
    return G.R_from_quat(RNG.standard_normal(4))


# ---------------------------------------------------------------------------
# quadratic visibility (Sec. V-B-1)
# ---------------------------------------------------------------------------

@pytest.mark.parametrize("alpha,va", [(math.pi / 4, 0.5), (math.pi / 4, 0.8), (math.pi / 6, 0.3),
                                      (1.2, 0.9), (0.4, 0.5)])
def test_quad_coeffs_meet_conditions(alpha, va):
    """Eq. quadratic_conditions: v(0) = 1, v(pi) = 0, v(alpha) = v_alpha."""
    k0, k1, k2 = O.quad_coeffs(alpha, va)
    v = lambda th: k2 * math.cos(th) ** 2 + k1 * math.cos(th) + k0
    assert v(0.0) == pytest.approx(1.0, abs=1e-14)
    assert v(math.pi) == pytest.approx(0.0, abs=1e-14)
    assert v(alpha) == pytest.approx(va, abs=1e-14)


def test_quad_coeffs_golden():
    """Closed form of the 3x3 system (solved by hand): k1 = 1/2,
    k2 = (v_a - 1/2 - cos(a)/2)/(cos^2 a - 1), k0 = 1/2 - k2; the stored values for the
    90-degree field of view of Sec. VII-A (alpha = 45 deg) with v_alpha = 0.5 and 0.8."""
    rows = np.loadtxt(__file__.replace("test_oracle_pins.py", "golden/quad_coeffs.txt"))
    for alpha_deg, va, k0, k1, k2 in rows:
        k = O.quad_coeffs(math.radians(alpha_deg), va)
        np.testing.assert_allclose(k, [k0, k1, k2], rtol=0, atol=5e-12)


def test_quad_min_matches_figure_note():
    """Fig. sim_quad_vis: v_alpha = 0.5 goes negative behind the camera; the parabola's
    vertex is at cos(theta) = -k1/(2 k2) = -0.35355 with value -0.29550."""
    k0, k1, k2 = O.quad_coeffs(math.pi / 4, 0.5)
    c = np.linspace(-1, 1, 200001)
    v = k2 * c ** 2 + k1 * c + k0
    assert c[np.argmin(v)] == pytest.approx(-0.35355, abs=2e-5)
    assert v.min() == pytest.approx(-0.29550, abs=2e-5)


def test_vr_vp_dot_is_quadratic():
    """Eq. quad_vis_component: v_r(z)^T v_p(p) = k2 (z.p)^2 + k1 (z.p) + k0."""
    k = O.quad_coeffs(math.pi / 4, 0.5)
    for _ in range(50):
        z, p = rand_unit(), rand_unit()
        c = z @ p
        assert O.vr(z, k) @ O.vp(p) == pytest.approx(k[2] * c * c + k[1] * c + k[0], abs=1e-14)


def test_vr_grad_matches_fd():
    k = O.quad_coeffs(math.pi / 4, 0.8)
    z = rand_unit()
    g = O.vr_grad(z, k)
    h = 1e-6
    for a in range(3):
        e = np.zeros(3)
        e[a] = h
        fd = (O.vr(z + e, k) - O.vr(z - e, k)) / (2 * h)
        np.testing.assert_allclose(g[a], fd, atol=1e-9)


# ---------------------------------------------------------------------------
# Jacobians and the per-landmark FIM (Sec. V-A)
# ---------------------------------------------------------------------------

def test_global_jacobian_matches_fd():
    """Eq. jac_pose_global equals the derivative of the bearing under T <- exp(xi^) T
    (first form of Eq. deriv_se3), xi = (rho, phi)."""
    for _ in range(20):
        R, t = rand_R(), RNG.uniform(-5, 5, 3)
        p = t + R @ (rand_unit() * RNG.uniform(1, 8) * np.sign(1))
        J = O.jac_global(p, R, t)
        h = 1e-6
        fd = np.zeros((3, 6))
        for a in range(6):
            xi = np.zeros(6)
            xi[a] = h
            Rp, tp = G.se3_exp(xi)
            Rm, tm = G.se3_exp(-xi)
            fp = G.bearing(Rp @ R, Rp @ t + tp, p)
            fm = G.bearing(Rm @ R, Rm @ t + tm, p)
            fd[:, a] = (fp - fm) / (2 * h)
        np.testing.assert_allclose(J, fd, atol=1e-8)


def test_local_jacobian_matches_fd():
    """Second form of Eq. deriv_se3: T <- T exp(xi^)."""
    for _ in range(20):
        R, t = rand_R(), RNG.uniform(-5, 5, 3)
        p = t + rand_unit() * RNG.uniform(1, 8)
        J = O.jac_local(p, R, t)
        h = 1e-6
        fd = np.zeros((3, 6))
        for a in range(6):
            xi = np.zeros(6)
            xi[a] = h
            Rp, tp = G.se3_exp(xi)
            Rm, tm = G.se3_exp(-xi)
            fp = G.bearing(R @ Rp, R @ tp + t, p)
            fm = G.bearing(R @ Rm, R @ tm + t, p)
            fd[:, a] = (fp - fm) / (2 * h)
        np.testing.assert_allclose(J, fd, atol=1e-8)


def test_fim_gauss_is_JtJ_over_sigma2():
    """Eq. fim_gaussian."""
    J = RNG.standard_normal((3, 6))
    np.testing.assert_allclose(O.fim_gauss(J, 0.5), J.T @ J / 0.25, rtol=1e-14)


def test_single_landmark_rank2_closed_form():
    """One bearing: the projector I - f f^T has rank 2 (Eq. jac_f), so the camera-frame FIM
    has rank 2 with both non-zero eigenvalues (1 + 1/n^2)/sigma^2 (derived by hand)."""
    for sigma in (1.0, 0.01):
        for _ in range(10):
            R, t = rand_R(), RNG.uniform(-5, 5, 3)
            n = RNG.uniform(0.2, 9)
            p = t + R @ (rand_unit() * n)
            I = O.fim_gauss(O.jac_local(p, R, t), sigma)
            ev = np.linalg.eigvalsh(I)
            lam = (1 + 1 / n ** 2) / sigma ** 2
            np.testing.assert_allclose(ev[:4], 0.0, atol=1e-12 * lam)
            np.testing.assert_allclose(ev[4:], lam, rtol=1e-12)
            assert np.trace(I) == pytest.approx(2 * lam, rel=1e-13)
            # the closed-form block matrix [[P/n^2, -[u]x/n], [[u]x/n, P]] in the camera frame
            u = R.T @ (p - t) / n
            np.testing.assert_allclose(I * sigma ** 2, G.landmark_info_closed_form(u, n), atol=1e-12)


def test_global_fim_rotation_invariant():
    """Eq. global_fim_eq: with the global perturbation the FIM does not depend on R."""
    for _ in range(10):
        t = RNG.uniform(-5, 5, 3)
        p = t + rand_unit() * RNG.uniform(0.5, 8)
        I1 = O.fim_gauss(O.jac_global(p, rand_R(), t))
        I2 = O.fim_gauss(O.jac_global(p, rand_R(), t))
        np.testing.assert_allclose(I1, I2, atol=1e-13 * np.abs(I1).max())


def test_camera_frame_is_adjoint_of_world():
    """Sec. V-A: the two perturbations are related by the SE(3) adjoint:
    I_local = Ad^T I_global Ad with Ad = [[R, [t]x R], [0, R]]."""
    for _ in range(10):
        R, t = rand_R(), RNG.uniform(-20, 20, 3)
        p = t + rand_unit() * RNG.uniform(0.5, 8)
        Iw = O.fim_gauss(O.jac_global(p, R, t))
        Ic = O.fim_gauss(O.jac_local(p, R, t))
        A = G.Ad(R, t)
        np.testing.assert_allclose(A.T @ Iw @ A, Ic, atol=1e-10 * np.abs(Ic).max())


def test_reference_point_shift():
    """Moving the rotation reference point from the origin to o: C_0 = M_o^T C_o M_o."""
    for _ in range(10):
        R, t = rand_R(), RNG.uniform(-20, 20, 3)
        o = RNG.uniform(-30, 30, 3)
        p = t + rand_unit() * RNG.uniform(0.5, 8)
        I0 = O.fim_gauss(O.jac_global(p, R, t))
        Io = O.fim_gauss(O.jac_global(p, R, t, o))
        M = G.M_shift(o)
        np.testing.assert_allclose(M.T @ Io @ M, I0, atol=1e-10 * np.abs(I0).max())


def test_quat_to_rot_matches_hamilton_product():
    for _ in range(20):
        q = RNG.standard_normal(4)
        np.testing.assert_allclose(O.quat_to_rot(q), G.R_from_quat(q), atol=1e-14)


# ---------------------------------------------------------------------------
# single-precision decisions
# ---------------------------------------------------------------------------

def test_shell_decision_matches_float32_numpy():
    pts = RNG.uniform(-12, 12, (20000, 3)).astype(np.float32)
    x = np.array([0.125, 0.375, 0.625], np.float32)
    got = np.array([O.in_shell_f32(p, x, 0.1, 10.0) for p in pts])
    np.testing.assert_array_equal(got, G.shell_f32(pts, x, 0.1, 10.0))


def test_pinhole_decision_matches_projection():
    """Eq. exact_vis_func: visible iff the projection falls inside the 640 x 640 image;
    the division-free single-precision test agrees with the float64 projection for
    every landmark further than 1e-3 px from the image border."""
    lib = O.lib()
    import ctypes
    pose = np.concatenate([RNG.uniform(0, 5, 3), RNG.standard_normal(4)]).astype(np.float32)
    R = G.R_from_quat(pose[3:].astype(np.float64))
    pts = (pose[:3] + RNG.uniform(-10, 10, (20000, 3))).astype(np.float32)
    pc = (pts.astype(np.float64) - pose[:3].astype(np.float64)) @ R
    u = 320 * pc[:, 0] / pc[:, 2] + 320
    v = 320 * pc[:, 1] / pc[:, 2] + 320
    ref = (pc[:, 2] > 0) & (u >= 0) & (u < 640) & (v >= 0) & (v < 640)
    far = (np.minimum.reduce([np.abs(u), np.abs(u - 640), np.abs(v), np.abs(v - 640)]) > 1e-3) | (pc[:, 2] <= 0)
    got = np.array([lib.or_pinhole_visible_f32(p.ctypes.data_as(ctypes.POINTER(ctypes.c_float)),
                                               pose.ctypes.data_as(ctypes.POINTER(ctypes.c_float)),
                                               320.0, 320.0, 320.0, 320.0, 640.0, 640.0) for p in pts]).astype(bool)
    assert far.mean() > 0.99
    np.testing.assert_array_equal(got[far], ref[far])


# ---------------------------------------------------------------------------
# point-cloud FIM (Sec. IV)
# ---------------------------------------------------------------------------

def _small_scene(n=300, seed=3):
    sc = synth.room_landmarks(seed=seed, n=n)
    return sc.landmarks


def test_pc_fim_is_sum_of_closed_forms():
    """Eq. cost_info: I_T = sum over V of the per-landmark FIMs; with v = 1 the
    camera-frame sum equals the sum of the closed-form blocks over the range shell."""
    lm = _small_scene()
    poses = synth.random_poses(7, 5, (1, 1, 0.5), (9, 9, 2.5))
    prm = O.make_params(r_max=6.0)
    got = O.pc_fim(lm, poses, prm, vis=O.VIS_ONE, frame=O.FRAME_CAMERA)
    for j, pose in enumerate(poses):
        R = G.R_from_quat(pose[3:].astype(np.float64))
        t = pose[:3].astype(np.float64)
        mask = G.shell_f32(lm, pose[:3], 0.1, 6.0)
        ref = np.zeros((6, 6))
        for p in lm[mask].astype(np.float64):
            pc = R.T @ (p - t)
            n = np.linalg.norm(pc)
            ref += G.landmark_info_closed_form(pc / n, n)
        np.testing.assert_allclose(got[j], ref, rtol=1e-11, atol=1e-11 * np.abs(ref).max())


def test_pc_fim_pinhole_subset_and_psd():
    """Exact visibility keeps a subset of the shell; every FIM is symmetric PSD."""
    sc = synth.room_landmarks(seed=1, n=2000)
    poses = synth.random_poses(2, 20, (0.5, 0.5, 0.5), (9.5, 9.5, 2.5))
    prm = O.make_params(r_max=8.0)
    a, b = O.pc_counts(sc.landmarks, poses, prm)
    assert np.all(b <= a) and np.all(a > 0)
    I = O.pc_fim(sc.landmarks, poses, prm, vis=O.VIS_PINHOLE)
    np.testing.assert_allclose(I, np.transpose(I, (0, 2, 1)), atol=1e-9)
    for M in I:
        ev = np.linalg.eigvalsh(M)
        assert ev[0] >= -1e-10 * ev[-1]


def test_pc_fim_world_camera_same_det():
    """det Ad = 1: the determinant is the same in the world and camera frames."""
    lm = _small_scene(400)
    poses = synth.random_poses(9, 6, (2, 2, 1), (8, 8, 2))
    prm = O.make_params(r_max=8.0)
    Ic = O.pc_fim(lm, poses, prm, vis=O.VIS_CONE, frame=O.FRAME_CAMERA)
    Iw = O.pc_fim(lm, poses, prm, vis=O.VIS_CONE, frame=O.FRAME_WORLD)
    for a, b in zip(Ic, Iw):
        sa, la = np.linalg.slogdet(a)
        sb, lb = np.linalg.slogdet(b)
        assert sa == sb and la == pytest.approx(lb, abs=1e-8)


# ---------------------------------------------------------------------------
# field build (Sec. VI-A-1) and query (Eq. fim_separation)
# ---------------------------------------------------------------------------

def _tiny_map():
    lm = np.array([[0.3, 0.1, 0.2], [1.7, 0.4, 0.9], [-0.6, 1.3, 0.5], [0.9, -0.8, 1.6],
                   [1.1, 1.2, -0.7]], np.float32)
    grid = O.make_grid((0.0, 0.0, 0.0), 0.5, (2, 2, 2))
    return lm, grid


def test_field_brute_force_tiny_map():
    """Eq. general_info_pif and Eq. fim_separation with the paper's explicit matrices:
    C_I = sum_i diag6(v_p,i) I_i (6N_v x 6), V_I = diag6(v_r^T) (6 x 6N_v), and the query at a
    node is V_I C_I = sum_i (v_r^T v_p,i) I_i, with I_i from the closed form moved to the
    world origin."""
    lm, grid = _tiny_map()
    prm = O.make_params(r_max=3.0)
    field = O.full_field(lm, grid, prm, about_node=False)
    k = O.quad_coeffs(math.pi / 4, 0.5)
    for node in range(8):
        c = np.array([node & 1, (node >> 1) & 1, (node >> 2) & 1], float) * 0.5
        CI = np.zeros((60, 6))
        for p in lm.astype(np.float64):
            if not G.shell_f32(p, c, 0.1, 3.0):
                continue
            d = p - c
            n = np.linalg.norm(d)
            Ii = G.M_shift(c).T @ G.landmark_info_closed_form(d / n, n) @ G.M_shift(c)
            vp = np.array([*(d / n) ** 2, d[0] * d[1] / n ** 2, d[0] * d[2] / n ** 2, d[1] * d[2] / n ** 2, *(d / n), 1.0])
            D6 = np.kron(np.eye(6), vp.reshape(-1, 1))   # diag6(v_p): 6 N_v x 6
            CI += D6 @ Ii
        # oracle block k, (r, c)  <->  C_I[(r, k), c]
        got = field[node].transpose(1, 0, 2).reshape(60, 6)
        np.testing.assert_allclose(got, CI, atol=1e-10 * np.abs(CI).max())
        z = rand_unit()
        vr = np.array([k[2] * z[0] ** 2, k[2] * z[1] ** 2, k[2] * z[2] ** 2, 2 * k[2] * z[0] * z[1],
                       2 * k[2] * z[0] * z[2], 2 * k[2] * z[1] * z[2], k[1] * z[0], k[1] * z[1], k[1] * z[2], k[0]])
        VI = np.kron(np.eye(6), vr.reshape(1, -1))       # diag6(v_r^T): 6 x 6 N_v
        R = np.eye(3)
        R[:, 2] = z
        R[:, 0] = np.cross([0.3, 0.5, 0.8], z)
        R[:, 0] /= np.linalg.norm(R[:, 0])
        R[:, 1] = np.cross(z, R[:, 0])
        pose = np.concatenate([c, G.quat_from_R(R)])
        Iq, st, *_ = O.query_from_landmarks(lm, grid, prm, pose[None], interp=O.INTERP_NEAREST,
                                            frame=O.FRAME_WORLD, field=field)
        np.testing.assert_allclose(Iq[0], VI @ CI, atol=1e-10 * np.abs(CI).max())


def test_field_vis_one_equals_point_cloud_sum():
    """Visibility held at 1 (k2 = k1 = 0, k0 = 1 so v_r = e_10): the field at a node is the
    direct point-cloud sum over the shell (Eq. fim_separation with v = 1)."""
    sc = synth.room_landmarks(seed=1, n=2000)
    grid = O.make_grid((0, 0, 0), 0.5, (21, 21, 7))
    prm = O.make_params(r_max=8.0)
    nodes = RNG.choice(grid.nx * grid.ny * grid.nz, 12, replace=False)
    F = O.field_nodes(sc.landmarks, grid, prm, nodes)
    for node, Fk in zip(nodes, F):
        i, j, kk = node % 21, (node // 21) % 21, node // 441
        pose = np.array([[0.5 * i, 0.5 * j, 0.5 * kk, 1, 0, 0, 0]], np.float32)
        ref = O.pc_fim(sc.landmarks, pose, prm, vis=O.VIS_ONE, frame=O.FRAME_WORLD)[0]
        np.testing.assert_allclose(Fk[9], ref, rtol=1e-12, atol=1e-12 * np.abs(ref).max())


def test_field_node_frame_relation():
    """Node-local coefficients C' relate to the paper's world-frame ones by C^w = M_c^T C' M_c."""
    sc = synth.room_landmarks(seed=1, n=2000)
    grid = O.make_grid((0, 0, 0), 0.5, (21, 21, 7))
    prm = O.make_params(r_max=8.0)
    nodes = RNG.choice(grid.nx * grid.ny * grid.nz, 6, replace=False)
    Fw = O.field_nodes(sc.landmarks, grid, prm, nodes, about_node=False)
    Fl = O.field_nodes(sc.landmarks, grid, prm, nodes, about_node=True)
    for node, a, b in zip(nodes, Fw, Fl):
        c = 0.5 * np.array([node % 21, (node // 21) % 21, node // 441], float)
        M = G.M_shift(c)
        for kk in range(10):
            np.testing.assert_allclose(M.T @ b[kk] @ M, a[kk], atol=1e-10 * np.abs(a[kk]).max())


def test_field_additive_in_landmarks():
    """Sec. VI-A-1: the factor is a sum over landmarks, so build(A u B) = build(A) + build(B)."""
    sc = synth.room_landmarks(seed=4, n=1000)
    A, B = sc.landmarks[:600], sc.landmarks[600:]
    grid = O.make_grid((0, 0, 0), 0.5, (21, 21, 7))
    prm = O.make_params(r_max=8.0)
    nodes = RNG.choice(grid.nx * grid.ny * grid.nz, 8, replace=False)
    F = O.field_nodes(sc.landmarks, grid, prm, nodes)
    FA = O.field_nodes(A, grid, prm, nodes)
    FB = O.field_nodes(B, grid, prm, nodes)
    np.testing.assert_allclose(F, FA + FB, atol=1e-10 * np.abs(F).max())


def test_query_at_node_equals_quadratic_weighted_point_cloud():
    """Eq. fim_separation, first line: at a node the query is exactly
    sum_i v_quad(theta_i) I_i, the point-cloud FIM weighted by the quadratic visibility."""
    sc = synth.room_landmarks(seed=1, n=2000)
    grid = O.make_grid((0, 0, 0), 0.5, (21, 21, 7))
    for va in (0.5, 0.8):
        prm = O.make_params(r_max=8.0, v_alpha=va)
        for _ in range(5):
            node = (RNG.integers(0, 21), RNG.integers(0, 21), RNG.integers(0, 7))
            q = RNG.standard_normal(4)
            q = q / np.linalg.norm(q)
            pose = np.array([[0.5 * node[0], 0.5 * node[1], 0.5 * node[2], *q]], np.float32)
            for frame in (O.FRAME_WORLD, O.FRAME_CAMERA):
                Iq, *_ = O.query_from_landmarks(sc.landmarks, grid, prm, pose, frame=frame)
                ref = O.pc_fim(sc.landmarks, pose, prm, vis=O.VIS_QUAD, frame=frame)[0]
                np.testing.assert_allclose(Iq[0], ref, rtol=1e-10, atol=1e-10 * np.abs(ref).max())


def test_query_psd_for_nonnegative_visibility():
    """v_alpha = 0.8 keeps v_quad >= 0 on [0, pi], so every queried FIM is PSD."""
    sc = synth.room_landmarks(seed=1, n=2000)
    grid = O.make_grid((0, 0, 0), 0.5, (21, 21, 7))
    prm = O.make_params(r_max=8.0, v_alpha=0.8)
    poses = synth.random_poses(11, 30, (0, 0, 0), (10, 10, 3))
    I, *_ = O.query_from_landmarks(sc.landmarks, grid, prm, poses)
    for M in I:
        ev = np.linalg.eigvalsh(M)
        assert ev[0] >= -1e-10 * ev[-1]


def test_query_optical_axis_invariance():
    """v depends on R only through z = R e3 (Sec. V-B-2), so R -> R Rz(psi) leaves the world
    FIM unchanged, and the camera-frame trace, determinant and lambda_min unchanged."""
    sc = synth.room_landmarks(seed=1, n=2000)
    grid = O.make_grid((0, 0, 0), 0.5, (21, 21, 7))
    prm = O.make_params(r_max=8.0)
    poses = synth.random_poses(12, 10, (0, 0, 0), (10, 10, 3)).astype(np.float64)
    rot = poses.copy()
    for p in rot:
        R = G.R_from_quat(p[3:]) @ G.so3_exp([0, 0, RNG.uniform(-3, 3)])
        p[3:] = G.quat_from_R(R)
    Iw1, *_ = O.query_from_landmarks(sc.landmarks, grid, prm, poses, frame=O.FRAME_WORLD)
    Iw2, *_ = O.query_from_landmarks(sc.landmarks, grid, prm, rot, frame=O.FRAME_WORLD)
    np.testing.assert_allclose(Iw1, Iw2, atol=1e-9 * np.abs(Iw1).max())
    Ic1, *_ = O.query_from_landmarks(sc.landmarks, grid, prm, poses)
    Ic2, *_ = O.query_from_landmarks(sc.landmarks, grid, prm, rot)
    m1, m2 = O.metrics(Ic1), O.metrics(Ic2)
    np.testing.assert_allclose(m1, m2, rtol=1e-9, atol=1e-9)


def test_trilinear_interpolation_properties():
    """Interpolation over the 8 surrounding nodes (Sec. VII-A-1): weights sum to 1, the value
    at a node is that node's, and along a cell edge the field is linear."""
    sc = synth.room_landmarks(seed=1, n=500)
    grid = O.make_grid((0, 0, 0), 0.5, (21, 21, 7))
    prm = O.make_params(r_max=8.0)
    field = O.full_field(sc.landmarks, grid, prm)
    poses = synth.random_poses(13, 50, (0, 0, 0), (10, 10, 3))
    nodes, w, dw, st = O.query_cells(grid, poses)
    np.testing.assert_allclose(w.sum(1), 1.0, atol=1e-14)
    np.testing.assert_allclose(dw.sum(1), 0.0, atol=1e-12)
    assert np.all(st == 0)
    q = np.array([1, 0, 0, 0.0])
    a = np.array([2.0, 3.0, 1.0])
    ts = [a + np.array([s * 0.5, 0, 0]) for s in (0.0, 0.25, 1.0)]
    P = np.array([np.concatenate([t, q]) for t in ts])
    I, *_ = O.query_from_landmarks(sc.landmarks, grid, prm, P, frame=O.FRAME_WORLD, field=field)
    np.testing.assert_allclose(I[1], 0.75 * I[0] + 0.25 * I[2], atol=1e-10 * np.abs(I).max())
    node = 4 + 21 * (6 + 21 * 2)
    k = O.quad_coeffs(prm.half_fov, prm.v_alpha)
    ref = np.einsum("k,kij->ij", O.vr([0, 0, 1], k), field[node])
    np.testing.assert_allclose(I[0], ref, atol=1e-12 * np.abs(ref).max())
    # outside the lattice: status 1
    out = np.array([[-0.1, 5, 1, 1, 0, 0, 0], [5, 5, 3.2, 1, 0, 0, 0]])
    assert list(O.query_cells(grid, out)[3]) == [1, 1]


# ---------------------------------------------------------------------------
# metrics (Sec. IV)
# ---------------------------------------------------------------------------

def test_metrics_match_library_routines():
    """trace, log|det| with its sign, and lambda_min against numpy (LAPACK)."""
    for _ in range(40):
        A = RNG.standard_normal((6, 6))
        S = A @ A.T if RNG.random() < 0.5 else A + A.T
        S *= 10 ** RNG.uniform(-3, 4)
        m = O.metrics(S[None])[0]
        s, la = np.linalg.slogdet(S)
        assert m[0] == pytest.approx(np.trace(S), rel=1e-13, abs=1e-13 * np.abs(S).max())
        assert m[1] == pytest.approx(la, abs=1e-10)
        assert m[2] == s
        ev = np.linalg.eigvalsh(S)
        assert m[3] == pytest.approx(ev[0], abs=1e-12 * np.abs(ev).max())
        ev2, V = O.eig(S)
        np.testing.assert_allclose(ev2[0], ev, atol=1e-12 * np.abs(ev).max())
        np.testing.assert_allclose(S @ V[0], V[0] * ev2[0], atol=1e-11 * np.abs(ev).max())


def test_inverse6_matches_library():
    A = RNG.standard_normal((6, 6))
    np.testing.assert_allclose(O.inverse6(A), np.linalg.inv(A), rtol=1e-10, atol=1e-10)


# ---------------------------------------------------------------------------
# gradient of the metrics with respect to the pose
# ---------------------------------------------------------------------------

def _fd_grad(landmarks, grid, prm, field, pose, which, h_t=1e-6, h_r=1e-6):
    def metric(p):
        I, *_ = O.query_from_landmarks(landmarks, grid, prm, p[None], field=field)
        m = O.metrics(I)[0]
        return [m[0], m[1], m[3]][which]

    g = np.zeros(6)
    for a in range(3):
        e = np.zeros(3)
        e[a] = h_t
        pp, pm = pose.copy(), pose.copy()
        pp[:3] += e
        pm[:3] -= e
        g[a] = (metric(pp) - metric(pm)) / (2 * h_t)
    R = G.R_from_quat(pose[3:])
    for a in range(3):
        e = np.zeros(3)
        e[a] = h_r
        pp, pm = pose.copy(), pose.copy()
        pp[3:] = G.quat_from_R(R @ G.so3_exp(e))
        pm[3:] = G.quat_from_R(R @ G.so3_exp(-e))
        g[3 + a] = (metric(pp) - metric(pm)) / (2 * h_r)
    return g


@pytest.mark.parametrize("which", [0, 1, 2])
def test_query_gradient_matches_central_differences(which):
    """Analytic oracle gradient (trace, log|det|, lambda_min) vs central differences in t and
    in a right so(3) perturbation; the component about the optical axis vanishes."""
    sc = synth.room_landmarks(seed=1, n=800)
    grid = O.make_grid((0, 0, 0), 0.5, (21, 21, 7))
    prm = O.make_params(r_max=8.0, v_alpha=0.8)
    field = O.full_field(sc.landmarks, grid, prm)
    k = O.quad_coeffs(prm.half_fov, prm.v_alpha)
    poses = synth.random_poses(21, 6, (0.6, 0.6, 0.6), (9.4, 9.4, 2.4)).astype(np.float64)
    gm = np.zeros((len(poses), 3))
    gm[:, which] = 1.0
    nodes, w, dw, st = O.query_cells(grid, poses)
    g = O.query_grad(field[nodes], w, dw, poses, k, gm)
    for p, ga in zip(poses, g):
        fd = _fd_grad(sc.landmarks, grid, prm, field, p, which)
        scale = np.abs(fd).max()
        np.testing.assert_allclose(ga, fd, atol=2e-6 * scale + 1e-9)
        assert abs(ga[5]) <= 1e-9 * scale + 1e-12
