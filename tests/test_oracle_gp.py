"""Pins of the FP64 oracle's GP visibility model (Sec. V-B-2) against what the paper and the
mathematics fix: the sigmoid's half value at the field-of-view edge and its symmetry, GP
interpolation of the training samples, the log marginal likelihood against scipy's Gaussian
density, a brute-force evaluation of the paper's explicit matrices with numpy's solver, the
separation identity at a node against the GP-weighted point-cloud sum, and the optical-axis
invariance.  No GPU."""
import math

import numpy as np
import pytest

import oracle as O
from paper_2008_03324_gb300 import synth
from tests import _np_geom as G

RNG = np.random.default_rng(2008)

# length scales that maximise the marginal likelihood of 2000 random bearings (seed 7) for
# spherical-Fibonacci sample axes; test_fitted_length_scales_are_likelihood_maxima pins them
FITTED = {30: 0.89754, 50: 0.67813, 70: 0.61302}


def _gp(ns, **kw):
    return O.GP(synth.fibonacci_sphere(ns), FITTED[ns], **kw)


def _rotation_with_axis(z):
    z = np.asarray(z, float) / np.linalg.norm(z)
    a = np.cross([0.3, 0.5, 0.8], z)
    a /= np.linalg.norm(a)
    R = np.stack([a, np.cross(z, a), z], axis=1)
    return R


# ---------------------------------------------------------------------------
# the sigmoid visibility (Eq. sigmoid_vis_func)
# ---------------------------------------------------------------------------

@pytest.mark.parametrize("alpha", [math.pi / 4, math.pi / 6, 1.1])
def test_sigmoid_is_half_at_the_fov_edge_and_symmetric(alpha):
    """v_sig(theta) = 1/2 at theta = alpha, and v(cos alpha + d) + v(cos alpha - d) = 1 (a
    logistic function is point-symmetric about its midpoint)."""
    axes = np.array([[0.0, 0.0, 1.0]])
    for d in (0.0, 0.01, 0.1, 0.3):
        c1, c2 = math.cos(alpha) + d, math.cos(alpha) - d
        if abs(c1) > 1 or abs(c2) > 1:
            continue
        P = np.array([[math.sqrt(1 - c1 * c1), 0, c1], [0, math.sqrt(1 - c2 * c2), c2]])
        y = O.gp_training(axes, 15.0, alpha, P)[:, 0]
        if d == 0.0:
            assert y[0] == pytest.approx(0.5, abs=1e-15)
        assert y[0] + y[1] == pytest.approx(1.0, abs=1e-14)
        assert y[0] >= 0.5 >= y[1]


def test_sigmoid_tends_to_the_fov_step():
    """Large k_s turns the sigmoid into the indicator of the field of view (Eq.
    theta_vis_func), which k_s = 15 smooths."""
    alpha = math.pi / 4
    axes = np.array([[0.0, 0.0, 1.0]])
    th = np.linspace(0, math.pi, 181)
    P = np.stack([np.sin(th), np.zeros_like(th), np.cos(th)], axis=1)
    y = O.gp_training(axes, 400.0, alpha, P)[:, 0]
    inside, outside = th < alpha - 0.05, th > alpha + 0.05
    assert np.all(y[inside] > 1 - 1e-4) and np.all(y[outside] < 1e-4)
    y15 = O.gp_training(axes, 15.0, alpha, P)[:, 0]
    assert np.all(np.diff(y15) <= 0)            # decreasing in theta
    assert 0.9 < y15[0] < 1.0 and y15[-1] < 1e-10


# ---------------------------------------------------------------------------
# GP regression (Sec. III-B, Eq. gp_regress; Eq. gp_vis_approx)
# ---------------------------------------------------------------------------

@pytest.mark.parametrize("ns", [30, 70])
def test_gp_interpolates_the_samples(ns):
    """Kriging with a 1e-10 nugget reproduces the training values at the sample axes:
    v_gp(z_g) = v^s_g up to noise * |W v^s|."""
    gp = _gp(ns)
    for _ in range(5):
        p = RNG.standard_normal(3)
        p /= np.linalg.norm(p)
        vs = O.gp_training(gp.axes, gp.ks, math.pi / 4, p[None])[0]
        got = np.array([gp.visibility(gp.axes[g], p) for g in range(ns)])
        bound = 1e-10 * np.abs(gp.vp(p)).max() + 1e-12
        assert np.abs(got - vs).max() <= 10 * bound


def test_gp_weights_invert_the_kernel_matrix():
    """W (K^s + noise I) = I, K^s from the SE kernel k(a, b) = exp(-|a - b|^2 / 2 l^2)."""
    gp = _gp(50)
    d2 = ((gp.axes[:, None, :] - gp.axes[None, :, :]) ** 2).sum(-1)
    K = np.exp(-d2 / (2 * gp.l ** 2)) + 1e-10 * np.eye(50)
    np.testing.assert_allclose(gp.W @ K, np.eye(50), atol=1e-9)
    np.testing.assert_allclose(gp.W, gp.W.T, atol=1e-9)


@pytest.mark.parametrize("ns,l", [(30, 0.8), (50, 0.5), (20, 1.3)])
def test_log_marginal_matches_scipy(ns, l):
    """Rasmussen & Williams Eq. 2.30 for independent draws: the sum of Gaussian log densities
    of the training vectors under N(0, K^s + noise I)."""
    scipy_stats = pytest.importorskip("scipy.stats")
    axes = synth.fibonacci_sphere(ns)
    P = synth.sphere_points(11, 40)
    Y = O.gp_training(axes, 15.0, math.pi / 4, P)
    noise = 1e-4            # a larger nugget keeps scipy's own factorisation well posed
    d2 = ((axes[:, None, :] - axes[None, :, :]) ** 2).sum(-1)
    cov = np.exp(-d2 / (2 * l * l)) + noise * np.eye(ns)
    ref = scipy_stats.multivariate_normal(mean=np.zeros(ns), cov=cov).logpdf(Y).sum()
    got = O.gp_log_marginal(axes, l, noise, Y)
    assert got == pytest.approx(ref, rel=1e-9)


@pytest.mark.parametrize("ns", [30, 50, 70])
def test_fitted_length_scales_are_likelihood_maxima(ns):
    """The length scale is the maximiser of the marginal likelihood (Sec. V-B-2): the oracle
    likelihood at l +- 1 % is below its value at the tabulated l."""
    axes = synth.fibonacci_sphere(ns)
    Y = O.gp_training(axes, 15.0, math.pi / 4, synth.sphere_points(7, 2000))
    l = FITTED[ns]
    f0 = O.gp_log_marginal(axes, l, 1e-10, Y)
    assert O.gp_log_marginal(axes, l * 1.01, 1e-10, Y) < f0
    assert O.gp_log_marginal(axes, l * 0.99, 1e-10, Y) < f0


def test_gp_regresses_the_sigmoid_better_with_more_samples():
    """The GP approximates the sigmoid visibility, and more samples reduce the difference
    (Sec. VII-A: accuracy grows with N_s)."""
    z = synth.sphere_points(21, 300)
    p = synth.sphere_points(22, 300)
    c = (z * p).sum(1)
    vsig = 1.0 / (1.0 + np.exp(-15.0 * (c - math.cos(math.pi / 4))))
    err = {}
    for ns in (30, 70):
        gp = _gp(ns)
        v = np.array([gp.visibility(a, b) for a, b in zip(z, p)])
        err[ns] = np.abs(v - vsig).mean()
    assert err[70] < err[30] < 0.08


# ---------------------------------------------------------------------------
# the GP field (Eq. general_info_pif, Eq. fim_separation with v_r = K_z, v_p = W v^s)
# ---------------------------------------------------------------------------

def _tiny_map():
    lm = np.array([[0.3, 0.1, 0.2], [1.7, 0.4, 0.9], [-0.6, 1.3, 0.5], [0.9, -0.8, 1.6],
                   [1.1, 1.2, -0.7], [0.2, 0.9, 1.4]], np.float32)
    grid = O.make_grid((0.0, 0.0, 0.0), 0.5, (2, 2, 2))
    return lm, grid


def test_gp_field_brute_force_tiny_map():
    """The paper's explicit matrices with numpy's solver in place of the oracle's inverse:
    C_I = sum_i diag6(v_p,i) I_i, v_p = solve(K^s + noise I, v^s); at a node the query is
    V_I C_I with V_I = diag6(K_z^T), and equals sum_i v_gp(z; u_i) I_i."""
    lm, grid = _tiny_map()
    prm = O.make_params(r_max=3.0)
    gp = _gp(30)
    d2 = ((gp.axes[:, None, :] - gp.axes[None, :, :]) ** 2).sum(-1)
    K = np.exp(-d2 / (2 * gp.l ** 2)) + 1e-10 * np.eye(30)
    field = O.field_nodes_gp(lm, grid, prm, gp, np.arange(8))
    for node in range(8):
        c = np.array([node & 1, (node >> 1) & 1, (node >> 2) & 1], float) * 0.5
        CI = np.zeros((6 * 30, 6))
        for p in lm.astype(np.float64):
            if not G.shell_f32(p, c, 0.1, 3.0):
                continue
            d = p - c
            n = np.linalg.norm(d)
            Ii = G.M_shift(c).T @ G.landmark_info_closed_form(d / n, n) @ G.M_shift(c)
            vs = 1.0 / (1.0 + np.exp(-15.0 * (gp.axes @ (d / n) - math.cos(math.pi / 4))))
            vp = np.linalg.solve(K, vs)
            CI += np.kron(np.eye(6), vp.reshape(-1, 1)) @ Ii
        got = field[node].transpose(1, 0, 2).reshape(6 * 30, 6)
        np.testing.assert_allclose(got, CI, atol=1e-9 * np.abs(CI).max())
        z = RNG.standard_normal(3)
        z /= np.linalg.norm(z)
        kz = np.exp(-((gp.axes - z) ** 2).sum(-1) / (2 * gp.l ** 2))
        VI = np.kron(np.eye(6), kz.reshape(1, -1))
        pose = np.concatenate([c, G.quat_from_R(_rotation_with_axis(z))])
        Iq, st, *_ = O.query_gp_from_landmarks(lm, grid, prm, gp, pose[None], interp=O.INTERP_NEAREST,
                                               frame=O.FRAME_WORLD)
        np.testing.assert_allclose(Iq[0], VI @ CI, atol=1e-9 * np.abs(CI).max())


@pytest.mark.parametrize("ns", [30, 70])
def test_gp_query_at_node_equals_gp_weighted_point_cloud(ns):
    """Eq. fim_separation: at a node the GP-field query is exactly the point-cloud FIM with
    every landmark weighted by its GP visibility v_gp(z; u_i), in both frames."""
    sc = synth.room_landmarks(seed=1, n=800)
    grid = O.make_grid((0, 0, 0), 0.5, (21, 21, 7))
    prm = O.make_params(r_max=8.0)
    gp = _gp(ns)
    for _ in range(4):
        node = (RNG.integers(0, 21), RNG.integers(0, 21), RNG.integers(0, 7))
        q = RNG.standard_normal(4)
        q /= np.linalg.norm(q)
        pose = np.array([[0.5 * node[0], 0.5 * node[1], 0.5 * node[2], *q]], np.float32)
        for frame in (O.FRAME_WORLD, O.FRAME_CAMERA):
            Iq, *_ = O.query_gp_from_landmarks(sc.landmarks, grid, prm, gp, pose, frame=frame)
            ref = O.pc_fim_gp(sc.landmarks, pose, prm, gp, frame=frame)[0]
            np.testing.assert_allclose(Iq[0], ref, rtol=1e-9, atol=1e-9 * np.abs(ref).max())


def test_sigmoid_basis_relation_and_node_frame():
    """The sigmoid-value basis D_g = sum_i v^s_g I_i relates to the paper's C by C = W D, and
    node-local coefficients relate to world ones by C^w = M_c^T C' M_c."""
    sc = synth.room_landmarks(seed=2, n=600)
    grid = O.make_grid((0, 0, 0), 0.5, (21, 21, 7))
    prm = O.make_params(r_max=8.0)
    gp = _gp(50)
    nodes = RNG.choice(21 * 21 * 7, 5, replace=False)
    C = O.field_nodes_gp(sc.landmarks, grid, prm, gp, nodes)
    D = O.field_nodes_gp(sc.landmarks, grid, prm, gp, nodes, basis="sigmoid")
    np.testing.assert_allclose(np.einsum("gh,nhij->ngij", gp.W, D), C, atol=1e-10 * np.abs(C).max())
    Dl = O.field_nodes_gp(sc.landmarks, grid, prm, gp, nodes, about_node=True, basis="sigmoid")
    for node, a, b in zip(nodes, D, Dl):
        c = 0.5 * np.array([node % 21, (node // 21) % 21, node // 441], float)
        M = G.M_shift(c)
        np.testing.assert_allclose(np.einsum("ji,gjk,kl->gil", M, b, M), a, atol=1e-10 * np.abs(a).max())
    # every weight of the sigmoid basis is in (0, 1): D_g is PSD
    for Dn in D:
        for Dg in Dn:
            assert np.linalg.eigvalsh(Dg)[0] >= -1e-9 * np.abs(Dg).max()


def test_gp_field_additive_and_optical_axis_invariance():
    """The factor is a sum over landmarks (Sec. VI-A-1); the GP visibility depends on R only
    through z = R e3, so R -> R Rz(psi) leaves the world FIM unchanged."""
    sc = synth.room_landmarks(seed=4, n=600)
    A, B = sc.landmarks[:350], sc.landmarks[350:]
    grid = O.make_grid((0, 0, 0), 0.5, (21, 21, 7))
    prm = O.make_params(r_max=8.0)
    gp = _gp(30)
    nodes = RNG.choice(21 * 21 * 7, 5, replace=False)
    F = O.field_nodes_gp(sc.landmarks, grid, prm, gp, nodes)
    np.testing.assert_allclose(F, O.field_nodes_gp(A, grid, prm, gp, nodes) + O.field_nodes_gp(B, grid, prm, gp, nodes),
                               atol=1e-10 * np.abs(F).max())
    poses = synth.random_poses(12, 6, (0, 0, 0), (10, 10, 3)).astype(np.float64)
    rot = poses.copy()
    for p in rot:
        p[3:] = G.quat_from_R(G.R_from_quat(p[3:]) @ G.so3_exp([0, 0, RNG.uniform(-3, 3)]))
    I1, *_ = O.query_gp_from_landmarks(sc.landmarks, grid, prm, gp, poses, frame=O.FRAME_WORLD)
    I2, *_ = O.query_gp_from_landmarks(sc.landmarks, grid, prm, gp, rot, frame=O.FRAME_WORLD)
    np.testing.assert_allclose(I1, I2, atol=1e-9 * np.abs(I1).max())
