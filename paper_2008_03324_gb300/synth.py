"""Seeded synthetic inputs shaped like the paper's workloads.

This module holds no arithmetic of the method: it only draws landmark maps, poses,
request streams and trajectories.  It is the one module that both the CUDA path (tests,
benchmark) and the FP64 oracle consume, so that both sides see bit-identical inputs.

Every generator uses numpy's PCG64 with an explicit seed and returns float32 arrays.

Scenes (sizes from the benchmark configurations; the paper's own environments are a
1000-landmark random box (Sec. VII-A) and a rendered warehouse (Sec. VII-B) that is not
available here, so these stand in for them):

* :func:`room_landmarks`     10 x 10 x 3 m room, landmarks area-uniform on the four walls
                             and the ceiling, isotropic N(0, 0.02^2) jitter.
* :func:`warehouse`          50 x 50 x 10 m hall with 40 axis-aligned boxes of 1-6 m sides;
                             60 % of the landmarks on exposed box faces, 40 % on the walls.
* :func:`building`           100 x 100 x 20 m, 10 x 10 rooms of 10 m with one 1 x 2.2 m
                             doorway per interior wall segment, 200 boxes; landmarks
                             area-proportional over walls (interior walls both sides) and
                             box faces.
* :func:`random_poses`       positions uniform in a box, rotations uniform on SO(3)
                             (normalised 4-D Gaussian quaternion).
* :func:`request_stream`     planner requests of 8-4096 poses (log-uniform) along straight
                             or Catmull-Rom segments, yaw U[-pi, pi), pitch U[-pi/6, pi/6].
* :func:`bspline_batch`      uniform cubic B-spline trajectories with per-sample yaw.

Pose layout everywhere: [tx, ty, tz, qw, qx, qy, qz] with the quaternion giving R_wc.
"""
from __future__ import annotations

import math
from dataclasses import dataclass

import numpy as np


def _rng(seed: int) -> np.random.Generator:
    return np.random.Generator(np.random.PCG64(int(seed)))


# ---------------------------------------------------------------------------
# geometry helpers (no method arithmetic)
# ---------------------------------------------------------------------------

def _sample_rects(rng, rects, weights, n):
    """Area-weighted uniform samples on axis-aligned rectangles.

    rects: [R, 3, 3] rows (corner, edge_u, edge_v); weights: [R] (area x multiplicity)."""
    rects = np.asarray(rects, dtype=np.float64)
    w = np.asarray(weights, dtype=np.float64)
    idx = rng.choice(len(rects), size=n, p=w / w.sum())
    s = rng.random((n, 2))
    r = rects[idx]
    return r[:, 0] + s[:, :1] * r[:, 1] + s[:, 1:] * r[:, 2]


def _rect(corner, u, v):
    return np.array([corner, u, v], dtype=np.float64)


def _box_faces(lo, hi, bottom=False):
    """Faces of an axis-aligned box [lo, hi] (4 sides + top, optionally bottom)."""
    x0, y0, z0 = lo
    x1, y1, z1 = hi
    sx, sy, sz = x1 - x0, y1 - y0, z1 - z0
    faces = [
        _rect((x0, y0, z0), (0, sy, 0), (0, 0, sz)),   # x = x0
        _rect((x1, y0, z0), (0, sy, 0), (0, 0, sz)),   # x = x1
        _rect((x0, y0, z0), (sx, 0, 0), (0, 0, sz)),   # y = y0
        _rect((x0, y1, z0), (sx, 0, 0), (0, 0, sz)),   # y = y1
        _rect((x0, y0, z1), (sx, 0, 0), (0, sy, 0)),   # top
    ]
    if bottom:
        faces.append(_rect((x0, y0, z0), (sx, 0, 0), (0, sy, 0)))
    return faces


def _area(r):
    return float(np.linalg.norm(r[1]) * np.linalg.norm(r[2]))


def _inside_any(points, boxes, margin=1e-6, cell=4.0):
    """True for points strictly inside any of the boxes (boxes bucketed on a 2-D grid of
    `cell`-metre squares so each point is tested against the few boxes near it)."""
    points = np.asarray(points)
    out = np.zeros(len(points), bool)
    if len(boxes) == 0 or len(points) == 0:
        return out
    lo = np.array([b[0] for b in boxes], dtype=np.float64) + margin   # [B, 3]
    hi = np.array([b[1] for b in boxes], dtype=np.float64) - margin
    x0, y0 = lo[:, 0].min(), lo[:, 1].min()
    nx = int(np.ceil((hi[:, 0].max() - x0) / cell)) + 1
    ny = int(np.ceil((hi[:, 1].max() - y0) / cell)) + 1
    buckets = {}
    for b in range(len(boxes)):
        for i in range(int((lo[b, 0] - x0) // cell), int((hi[b, 0] - x0) // cell) + 1):
            for j in range(int((lo[b, 1] - y0) // cell), int((hi[b, 1] - y0) // cell) + 1):
                buckets.setdefault(i + nx * j, []).append(b)
    ix = np.floor((points[:, 0] - x0) / cell).astype(np.int64)
    iy = np.floor((points[:, 1] - y0) / cell).astype(np.int64)
    valid = (ix >= 0) & (ix < nx) & (iy >= 0) & (iy < ny)
    cid = np.where(valid, ix + nx * iy, -1)
    order = np.argsort(cid, kind="stable")
    cs = cid[order]
    starts = np.searchsorted(cs, list(buckets.keys()), side="left")
    stops = np.searchsorted(cs, list(buckets.keys()), side="right")
    for (key, bl), a, z in zip(buckets.items(), starts, stops):
        if z <= a:
            continue
        idx = order[a:z]
        p = points[idx][:, None, :]
        out[idx] = np.any(np.all((p > lo[bl]) & (p < hi[bl]), axis=2), axis=1)
    return out


def _sample_surfaces(rng, rects, weights, n, boxes, jitter):
    """n area-uniform samples on the rectangles, rejecting points hidden inside boxes."""
    out = []
    need = n
    while need > 0:
        cand = _sample_rects(rng, rects, weights, int(need * 1.25) + 16)
        cand = cand[~_inside_any(cand, boxes)]
        out.append(cand[:need])
        need -= len(out[-1])
    pts = np.concatenate(out, axis=0)
    pts = pts + rng.normal(0.0, jitter, size=pts.shape)
    return pts.astype(np.float32)


def random_quaternions(rng, m):
    """Uniform on SO(3): normalised 4-D Gaussian, w >= 0."""
    q = rng.standard_normal((m, 4))
    q /= np.linalg.norm(q, axis=1, keepdims=True)
    q[q[:, 0] < 0] *= -1.0
    return q


def rot_to_quat(R):
    """Unit quaternion (w, x, y, z) of rotation matrices [..., 3, 3] (Shepperd's method)."""
    R = np.asarray(R, dtype=np.float64).reshape(-1, 3, 3)
    q = np.zeros((R.shape[0], 4))
    tr = R[:, 0, 0] + R[:, 1, 1] + R[:, 2, 2]
    for i in range(R.shape[0]):
        m = R[i]
        if tr[i] > 0:
            s = math.sqrt(tr[i] + 1.0) * 2
            q[i] = [0.25 * s, (m[2, 1] - m[1, 2]) / s, (m[0, 2] - m[2, 0]) / s, (m[1, 0] - m[0, 1]) / s]
        elif m[0, 0] > m[1, 1] and m[0, 0] > m[2, 2]:
            s = math.sqrt(1.0 + m[0, 0] - m[1, 1] - m[2, 2]) * 2
            q[i] = [(m[2, 1] - m[1, 2]) / s, 0.25 * s, (m[0, 1] + m[1, 0]) / s, (m[0, 2] + m[2, 0]) / s]
        elif m[1, 1] > m[2, 2]:
            s = math.sqrt(1.0 + m[1, 1] - m[0, 0] - m[2, 2]) * 2
            q[i] = [(m[0, 2] - m[2, 0]) / s, (m[0, 1] + m[1, 0]) / s, 0.25 * s, (m[1, 2] + m[2, 1]) / s]
        else:
            s = math.sqrt(1.0 + m[2, 2] - m[0, 0] - m[1, 1]) * 2
            q[i] = [(m[1, 0] - m[0, 1]) / s, (m[0, 2] + m[2, 0]) / s, (m[1, 2] + m[2, 1]) / s, 0.25 * s]
    q /= np.linalg.norm(q, axis=1, keepdims=True)
    q[q[:, 0] < 0] *= -1.0
    return q


def look_rotation(yaw, pitch):
    """R_wc of a camera whose optical axis has the given yaw/pitch, roll 0, image y down.

    yaw, pitch: [m].  Returns [m, 3, 3] with columns (x_c, y_c, z_c) in the world."""
    yaw = np.asarray(yaw, dtype=np.float64)
    pitch = np.asarray(pitch, dtype=np.float64)
    f = np.stack([np.cos(pitch) * np.cos(yaw), np.cos(pitch) * np.sin(yaw), np.sin(pitch)], axis=-1)
    up = np.array([0.0, 0.0, 1.0])
    x = np.cross(f, up)
    x /= np.linalg.norm(x, axis=-1, keepdims=True)
    y = np.cross(f, x)
    return np.stack([x, y, f], axis=-1)


# ---------------------------------------------------------------------------
# scenes
# ---------------------------------------------------------------------------

@dataclass
class Scene:
    name: str
    landmarks: np.ndarray          # [n, 3] float32
    lo: np.ndarray                 # scene bounds
    hi: np.ndarray
    boxes: list                    # list of (lo, hi) obstacles


def room_landmarks(seed: int = 1, n: int = 2000, size=(10.0, 10.0, 3.0), jitter: float = 0.02) -> Scene:
    """Walls and ceiling of a size[0] x size[1] x size[2] room, area-uniform, Gaussian jitter."""
    rng = _rng(seed)
    L, W, H = size
    rects = [
        _rect((0, 0, 0), (0, W, 0), (0, 0, H)),
        _rect((L, 0, 0), (0, W, 0), (0, 0, H)),
        _rect((0, 0, 0), (L, 0, 0), (0, 0, H)),
        _rect((0, W, 0), (L, 0, 0), (0, 0, H)),
        _rect((0, 0, H), (L, 0, 0), (0, W, 0)),
    ]
    pts = _sample_surfaces(rng, rects, [_area(r) for r in rects], n, [], jitter)
    return Scene("room", pts, np.zeros(3), np.array(size, float), [])


def _random_boxes(rng, count, extent, side=(1.0, 6.0)):
    boxes = []
    for _ in range(count):
        s = rng.uniform(side[0], side[1], size=3)
        cx = rng.uniform(s[0] / 2, extent[0] - s[0] / 2)
        cy = rng.uniform(s[1] / 2, extent[1] - s[1] / 2)
        lo = np.array([cx - s[0] / 2, cy - s[1] / 2, 0.0])
        hi = np.array([cx + s[0] / 2, cy + s[1] / 2, s[2]])
        boxes.append((lo, hi))
    return boxes


def warehouse(seed: int = 2, n: int = 200_000, size=(50.0, 50.0, 10.0), n_boxes: int = 40,
              box_fraction: float = 0.6, jitter: float = 0.02) -> Scene:
    """Hall of size[0] x size[1] x size[2] with n_boxes axis-aligned obstacles on the floor."""
    rng = _rng(seed)
    L, W, H = size
    boxes = _random_boxes(rng, n_boxes, size)
    walls = [
        _rect((0, 0, 0), (0, W, 0), (0, 0, H)),
        _rect((L, 0, 0), (0, W, 0), (0, 0, H)),
        _rect((0, 0, 0), (L, 0, 0), (0, 0, H)),
        _rect((0, W, 0), (L, 0, 0), (0, 0, H)),
    ]
    faces = [f for lo, hi in boxes for f in _box_faces(lo, hi)]
    n_box = int(round(n * box_fraction))
    p_box = _sample_surfaces(rng, faces, [_area(f) for f in faces], n_box, boxes, jitter)
    p_wall = _sample_surfaces(rng, walls, [_area(f) for f in walls], n - n_box, boxes, jitter)
    pts = np.concatenate([p_box, p_wall], axis=0)
    pts = pts[rng.permutation(len(pts))]
    return Scene("warehouse", pts, np.zeros(3), np.array(size, float), boxes)


def building(seed: int = 5, n: int = 2_000_000, size=(100.0, 100.0, 20.0), rooms=(10, 10),
             n_boxes: int = 200, door=(1.0, 2.2), jitter: float = 0.02) -> Scene:
    """Multi-room building: rooms[0] x rooms[1] rooms, one doorway per interior wall segment."""
    rng = _rng(seed)
    L, W, H = size
    rx, ry = L / rooms[0], W / rooms[1]
    rects, weights = [], []
    for r in (_rect((0, 0, 0), (0, W, 0), (0, 0, H)), _rect((L, 0, 0), (0, W, 0), (0, 0, H)),
              _rect((0, 0, 0), (L, 0, 0), (0, 0, H)), _rect((0, W, 0), (L, 0, 0), (0, 0, H))):
        rects.append(r)
        weights.append(_area(r))
    dw, dh = door
    # interior walls x = i*rx, split into segments of length ry, each with one doorway
    for i in range(1, rooms[0]):
        x = i * rx
        for j in range(rooms[1]):
            a = j * ry
            d = rng.uniform(a + 0.5, a + ry - 0.5 - dw)
            for r in (_rect((x, a, 0), (0, d - a, 0), (0, 0, H)),
                      _rect((x, d + dw, 0), (0, a + ry - d - dw, 0), (0, 0, H)),
                      _rect((x, d, dh), (0, dw, 0), (0, 0, H - dh))):
                rects.append(r)
                weights.append(2.0 * _area(r))
    for j in range(1, rooms[1]):
        y = j * ry
        for i in range(rooms[0]):
            a = i * rx
            d = rng.uniform(a + 0.5, a + rx - 0.5 - dw)
            for r in (_rect((a, y, 0), (d - a, 0, 0), (0, 0, H)),
                      _rect((d + dw, y, 0), (a + rx - d - dw, 0, 0), (0, 0, H)),
                      _rect((d, y, dh), (dw, 0, 0), (0, 0, H - dh))):
                rects.append(r)
                weights.append(2.0 * _area(r))
    boxes = _random_boxes(rng, n_boxes, size)
    for lo, hi in boxes:
        for f in _box_faces(lo, hi):
            rects.append(f)
            weights.append(_area(f))
    pts = _sample_surfaces(rng, rects, weights, n, boxes, jitter)
    return Scene("building", pts, np.zeros(3), np.array(size, float), boxes)


# ---------------------------------------------------------------------------
# poses and requests
# ---------------------------------------------------------------------------

def random_poses(seed: int, m: int, lo, hi) -> np.ndarray:
    """m poses, positions uniform in [lo, hi], rotations uniform on SO(3)."""
    rng = _rng(seed)
    lo = np.asarray(lo, dtype=np.float64)
    hi = np.asarray(hi, dtype=np.float64)
    t = lo + rng.random((m, 3)) * (hi - lo)
    q = random_quaternions(rng, m)
    return np.concatenate([t, q], axis=1).astype(np.float32)


def _free_points(rng, scene: Scene, count, zr):
    out = []
    need = count
    while need > 0:
        p = np.stack([rng.uniform(scene.lo[0] + 0.5, scene.hi[0] - 0.5, need * 2),
                      rng.uniform(scene.lo[1] + 0.5, scene.hi[1] - 0.5, need * 2),
                      rng.uniform(zr[0], zr[1], need * 2)], axis=1)
        p = p[~_inside_any(p, scene.boxes)]
        out.append(p[:need])
        need -= len(out[-1])
    return np.concatenate(out, axis=0)


def request_stream(seed: int, count: int, scene: Scene, min_len: int = 8, max_len: int = 4096,
                   zr=(0.5, 9.5), pitch_max: float = math.pi / 6):
    """Planner requests: list of [L, 7] float32 pose arrays.

    Length L = round(exp(U[ln min_len, ln max_len])); half are straight segments (RRT* edges),
    half Catmull-Rom segments (trajectory samples) between free-space points; yaw and pitch
    are drawn uniformly at both ends and interpolated along the request, roll 0."""
    rng = _rng(seed)
    reqs = []
    for _ in range(count):
        L = int(round(math.exp(rng.uniform(math.log(min_len), math.log(max_len)))))
        L = max(min_len, min(max_len, L))
        s = np.linspace(0.0, 1.0, L)[:, None]
        if rng.random() < 0.5:
            a, b = _free_points(rng, scene, 2, zr)
            pos = a + s * (b - a)
        else:
            P = _free_points(rng, scene, 4, zr)
            u = s
            pos = 0.5 * ((2 * P[1]) + (-P[0] + P[2]) * u + (2 * P[0] - 5 * P[1] + 4 * P[2] - P[3]) * u ** 2
                         + (-P[0] + 3 * P[1] - 3 * P[2] + P[3]) * u ** 3)
        yaw = rng.uniform(-math.pi, math.pi, 2)
        pitch = rng.uniform(-pitch_max, pitch_max, 2)
        y = yaw[0] + s[:, 0] * (yaw[1] - yaw[0])
        p = pitch[0] + s[:, 0] * (pitch[1] - pitch[0])
        q = rot_to_quat(look_rotation(y, p))
        reqs.append(np.concatenate([pos, q], axis=1).astype(np.float32))
    return reqs


def poisson_arrivals(seed: int, count: int, rate_per_s: float) -> np.ndarray:
    """Arrival times (s) of a Poisson stream."""
    rng = _rng(seed)
    return np.cumsum(rng.exponential(1.0 / rate_per_s, size=count))


def bspline_basis(n_ctrl: int, n_samples: int) -> np.ndarray:
    """[n_samples, n_ctrl] uniform cubic B-spline basis, samples spread over the valid range."""
    segs = n_ctrl - 3
    u = np.linspace(0.0, segs, n_samples, endpoint=False) + 0.5 * segs / n_samples
    B = np.zeros((n_samples, n_ctrl))
    for r, uu in enumerate(u):
        i = min(int(uu), segs - 1)
        s = uu - i
        b = np.array([(1 - s) ** 3, 3 * s ** 3 - 6 * s ** 2 + 4, -3 * s ** 3 + 3 * s ** 2 + 3 * s + 1, s ** 3]) / 6.0
        B[r, i:i + 4] = b
    return B


def bspline_batch(seed: int, scene: Scene, n_traj: int = 256, n_ctrl: int = 32, n_samples: int = 128,
                  step=(0.5, 1.5), zr=(1.0, 9.0)):
    """Control points of n_traj cubic B-splines (random walks in free space) and yaw controls.

    Returns (ctrl [n_traj, n_ctrl, 3] float64, yaw_ctrl [n_traj, n_ctrl] float64,
    basis [n_samples, n_ctrl] float64)."""
    rng = _rng(seed)
    ctrl = np.zeros((n_traj, n_ctrl, 3))
    start = _free_points(rng, scene, n_traj, zr)
    for i in range(n_traj):
        p = start[i].copy()
        ctrl[i, 0] = p
        for j in range(1, n_ctrl):
            for _ in range(50):
                d = rng.standard_normal(3)
                d /= np.linalg.norm(d)
                q = p + d * rng.uniform(step[0], step[1])
                if (scene.lo[0] + 0.5 < q[0] < scene.hi[0] - 0.5 and scene.lo[1] + 0.5 < q[1] < scene.hi[1] - 0.5
                        and zr[0] < q[2] < zr[1] and not _inside_any(q[None], scene.boxes)[0]):
                    p = q
                    break
            ctrl[i, j] = p
    yaw = np.cumsum(rng.uniform(-0.5, 0.5, (n_traj, n_ctrl)), axis=1) + rng.uniform(-math.pi, math.pi, (n_traj, 1))
    return ctrl, yaw, bspline_basis(n_ctrl, n_samples)


def horizontal_quats(yaw) -> np.ndarray:
    """Quaternions of cameras looking horizontally along yaw (z_c = (cos, sin, 0)), image y = -world z."""
    return rot_to_quat(look_rotation(np.asarray(yaw).reshape(-1), np.zeros(np.size(yaw))))


def fibonacci_sphere(n: int) -> np.ndarray:
    """n nearly uniform unit vectors (spherical Fibonacci lattice), [n, 3] float64: the sample
    optical axes of the GP visibility model."""
    i = np.arange(n, dtype=np.float64) + 0.5
    z = 1.0 - 2.0 * i / n
    r = np.sqrt(np.maximum(0.0, 1.0 - z * z))
    phi = i * math.pi * (3.0 - math.sqrt(5.0))
    return np.stack([r * np.cos(phi), r * np.sin(phi), z], axis=1)


def sphere_points(seed: int, m: int) -> np.ndarray:
    """m uniform unit vectors (normalised 3-D Gaussian), [m, 3] float64."""
    v = _rng(seed).standard_normal((m, 3))
    return v / np.linalg.norm(v, axis=1, keepdims=True)


# ---------------------------------------------------------------------------
# named workloads
# ---------------------------------------------------------------------------

@dataclass
class GridSpec:
    origin: tuple
    res: float
    dims: tuple

    @property
    def n_nodes(self):
        return int(self.dims[0]) * int(self.dims[1]) * int(self.dims[2])

    @property
    def lo(self):
        return np.array(self.origin, dtype=np.float64)

    @property
    def hi(self):
        return np.array(self.origin, dtype=np.float64) + self.res * (np.array(self.dims) - 1)


ROOM_GRID = GridSpec((0.0, 0.0, 0.0), 0.5, (21, 21, 7))
WAREHOUSE_GRID = GridSpec((0.125, 0.125, 0.125), 0.25, (200, 200, 40))
BUILDING_GRID = GridSpec((0.125, 0.125, 0.125), 0.25, (400, 400, 80))


def threshold_sets(seed: int, n: int, m: int, d_min: float = 0.3, d_max: float = 1.0,
                   half_fov: float = math.pi / 4) -> np.ndarray:
    """n sets of m landmarks meeting the localisation specification of the information
    threshold: inside the camera's field of view (a cone of half-angle half_fov about +z) at a
    distance in [d_min, d_max], uniform over that volume (cos theta and r^3 uniform).
    Camera frame, float32 [n, m, 3]."""
    rng = _rng(seed)
    ct = rng.uniform(math.cos(half_fov), 1.0, size=(n, m))
    st = np.sqrt(np.maximum(0.0, 1.0 - ct * ct))
    ph = rng.uniform(0.0, 2.0 * math.pi, size=(n, m))
    r = np.cbrt(rng.uniform(d_min ** 3, d_max ** 3, size=(n, m)))
    return np.stack([r * st * np.cos(ph), r * st * np.sin(ph), r * ct], axis=-1).astype(np.float32)


def random_box(seed: int = 8, n: int = 1000, size=(10.0, 10.0, 5.0)) -> np.ndarray:
    """n landmarks uniform in a size[0] x size[1] x size[2] box at the origin (float32 [n, 3]):
    the random-landmark environment of the paper's accuracy simulation (Sec. VII-A)."""
    rng = _rng(seed)
    return (rng.random((n, 3)) * np.asarray(size)).astype(np.float32)
