"""The seeded synthetic inputs follow their stated recipe (no GPU): surface landmarks lie on the
surfaces they were drawn from with the stated jitter and area shares, poses are uniform in
position and rotation, planner requests have log-uniform lengths and bounded pitch, arrivals are
Poisson, threshold sets fill the field-of-view cone uniformly in volume, and the B-spline basis
is a partition of unity.  Every generator is deterministic in its seed."""
import math

import numpy as np
import pytest

from paper_2008_03324_gb300 import synth


def test_generators_are_deterministic():
    a = synth.warehouse(seed=3, n=5000)
    b = synth.warehouse(seed=3, n=5000)
    assert np.array_equal(a.landmarks, b.landmarks)
    assert not np.array_equal(a.landmarks, synth.warehouse(seed=4, n=5000).landmarks)
    assert np.array_equal(synth.random_poses(9, 100, (0, 0, 0), (1, 1, 1)),
                          synth.random_poses(9, 100, (0, 0, 0), (1, 1, 1)))


def test_room_landmarks_on_walls_and_ceiling():
    """Area-uniform on four 10 x 3 m walls (120 m^2) and the 10 x 10 m ceiling (100 m^2), with
    N(0, 0.02^2) jitter off the surface."""
    sc = synth.room_landmarks(seed=1, n=20000)
    p = sc.landmarks.astype(np.float64)
    d = np.stack([p[:, 0], 10 - p[:, 0], p[:, 1], 10 - p[:, 1], 3 - p[:, 2]], axis=1)
    dmin = np.abs(d).min(axis=1)
    assert np.all(dmin < 0.02 * 6)                       # every point within 6 sigma of a surface
    assert np.std(d[np.arange(len(d)), np.abs(d).argmin(axis=1)]) == pytest.approx(0.02, rel=0.1)
    ceiling = np.abs(d[:, 4]) < 0.1
    assert ceiling.mean() == pytest.approx(100 / 220, abs=0.02)


def test_warehouse_split_and_bounds():
    """60 % of the landmarks on exposed box faces and 40 % on the four outer walls of the
    50 x 50 x 10 m hall; 40 boxes with 1-6 m sides standing on the floor inside the hall."""
    sc = synth.warehouse(seed=2, n=40000)
    p = sc.landmarks.astype(np.float64)
    assert len(sc.boxes) == 40
    for lo, hi in sc.boxes:
        s = hi - lo
        assert lo[2] == 0.0 and np.all(s >= 1.0 - 1e-9) and np.all(s <= 6.0 + 1e-9)
        assert np.all(lo[:2] >= 0.0) and np.all(hi[:2] <= 50.0)
    assert np.all(p[:, :2] > -0.2) and np.all(p[:, :2] < 50.2) and np.all(p[:, 2] > -0.2) and np.all(p[:, 2] < 10.2)
    on_wall = (np.minimum(np.minimum(p[:, 0], 50 - p[:, 0]), np.minimum(p[:, 1], 50 - p[:, 1])) < 0.1)
    assert on_wall.mean() == pytest.approx(0.4, abs=0.03)   # box faces touching a wall add a little


def test_random_poses_uniform():
    """Positions uniform in the box; unit quaternions whose rotations are uniform on SO(3)
    (the mean rotation matrix of a uniform sample vanishes)."""
    P = synth.random_poses(5, 20000, (1, 2, 3), (4, 6, 5)).astype(np.float64)
    t, q = P[:, :3], P[:, 3:]
    assert np.all(t >= [1, 2, 3]) and np.all(t <= [4, 6, 5])
    np.testing.assert_allclose(t.mean(axis=0), [2.5, 4.0, 4.0], atol=0.05)
    np.testing.assert_allclose(np.linalg.norm(q, axis=1), 1.0, atol=1e-6)
    w, x, y, z = q.T
    R00 = 1 - 2 * (y * y + z * z)
    R22 = 1 - 2 * (x * x + y * y)
    R01 = 2 * (x * y - w * z)
    for v in (R00, R22, R01):
        assert abs(v.mean()) < 0.02


def test_request_stream_lengths_and_angles():
    """Lengths round(exp(U[ln 8, ln 4096])): within [8, 4096] with median near sqrt(8 * 4096);
    unit quaternions with |pitch| <= 30 degrees; end points in the free hall."""
    sc = synth.warehouse(seed=2, n=2000)
    reqs = synth.request_stream(4, 400, sc)
    L = np.array([len(r) for r in reqs])
    assert L.min() >= 8 and L.max() <= 4096
    assert np.median(L) == pytest.approx(math.sqrt(8 * 4096), rel=0.3)
    allp = np.concatenate(reqs).astype(np.float64)
    np.testing.assert_allclose(np.linalg.norm(allp[:, 3:], axis=1), 1.0, atol=1e-5)
    w, x, y, z = allp[:, 3:].T
    # optical axis z_c = R e3 (third column of R): its elevation is the pitch
    zc = np.stack([2 * (x * z + w * y), 2 * (y * z - w * x), 1 - 2 * (x * x + y * y)], axis=1)
    elev = np.arcsin(np.clip(zc[:, 2], -1, 1))
    assert np.all(np.abs(elev) <= math.pi / 6 + 1e-4)
    # both end points of every request (the segment's or the spline's interpolated points) lie
    # in free space: 0.5 m inside the hall's walls, 0.5 <= z <= 9.5
    ends = np.concatenate([np.stack([r[0], r[-1]]) for r in reqs]).astype(np.float64)
    assert np.all(ends[:, :2] >= 0.5 - 1e-4) and np.all(ends[:, :2] <= 49.5 + 1e-4)
    assert np.all(ends[:, 2] >= 0.5 - 1e-4) and np.all(ends[:, 2] <= 9.5 + 1e-4)


def test_poisson_arrivals_rate():
    t = synth.poisson_arrivals(3, 50000, 20000.0)
    assert np.all(np.diff(t) > 0)
    gaps = np.diff(np.concatenate([[0.0], t]))
    assert gaps.mean() == pytest.approx(1 / 20000.0, rel=0.02)
    assert gaps.std() == pytest.approx(1 / 20000.0, rel=0.03)   # exponential: std = mean


def test_threshold_sets_fill_the_cone_uniformly():
    """Inside the field-of-view cone (half-angle 45 degrees) between 0.3 and 1 m, uniform in
    volume: cos(theta) and r^3 uniform."""
    S = synth.threshold_sets(7, 200, 100, 0.3, 1.0).reshape(-1, 3).astype(np.float64)
    r = np.linalg.norm(S, axis=1)
    c = S[:, 2] / r
    assert r.min() >= 0.3 - 1e-6 and r.max() <= 1.0 + 1e-6
    assert c.min() >= math.cos(math.pi / 4) - 1e-6
    assert (r ** 3).mean() == pytest.approx((0.3 ** 3 + 1.0) / 2, rel=0.02)
    assert c.mean() == pytest.approx((math.cos(math.pi / 4) + 1) / 2, rel=0.01)


def test_bspline_basis_partition_of_unity():
    B = synth.bspline_basis(32, 128)
    assert B.shape == (128, 32)
    assert np.all(B >= -1e-12)
    np.testing.assert_allclose(B.sum(axis=1), 1.0, atol=1e-12)
    assert np.count_nonzero(B > 1e-12, axis=1).max() <= 4     # cubic: four control points per sample


def test_fibonacci_sphere_is_spread():
    for n in (30, 70, 96):
        A = synth.fibonacci_sphere(n)
        np.testing.assert_allclose(np.linalg.norm(A, axis=1), 1.0, atol=1e-6)
        assert np.linalg.norm(A.mean(axis=0)) < 2.0 / n
        G = A @ A.T - 2 * np.eye(n)
        assert np.arccos(np.clip(G.max(), -1, 1)) > 1.5 / math.sqrt(n)   # no two axes nearly coincide
