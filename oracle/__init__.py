"""FP64 CPU oracle for the Fisher Information Field hot path (arXiv 2008.03324).

TEST INFRASTRUCTURE ONLY.  The product library never imports, links or executes
anything in this package; only ``tests/``, ``__graft_entry__.smoke()`` and the
CPU-baseline / reference legs of ``bench.py`` do.  The oracle shares no code with the
CUDA path: the arithmetic lives in ``fif_oracle.c`` (plain C, double precision,
OpenMP over independent nodes or poses) and this module only marshals numpy arrays.

Functions and the passages of the paper they follow:

* :func:`quad_coeffs` -- Eq. quadratic_conditions (Sec. V-B-1)
* :func:`vr`, :func:`vp` -- Eq. quad_vis_component
* :func:`jac_global`, :func:`jac_local` -- Eq. jac_f, Eq. jac_pose_global, both forms of Eq. deriv_se3
* :func:`fim_gauss` -- Eq. fim_gaussian
* :func:`pc_fim` -- Eq. cost_info (Sec. IV) with Eq. exact_vis_func / theta_vis_func / quad_vis_approx
* :func:`field_nodes` -- Eq. general_info_pif (Sec. VI-A-1)
* :func:`query_cells`, :func:`query` -- Eq. fim_separation, Eq. general_info_query, trilinear
  interpolation over the 8 surrounding voxels (Sec. VII-A-1)
* :func:`metrics` -- trace, log|det| (LU), lambda_min (cyclic Jacobi) (Sec. IV)
* :func:`query_grad` -- analytic gradient of the metrics with respect to the pose

All of them are pinned by ``tests/test_oracle_*.py`` (closed forms, finite differences,
brute force, invariants and textbook routines).
"""
from __future__ import annotations

import ctypes
import math
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "fif_oracle.c")
_LIB_PATH = os.path.join(_HERE, "liboracle.so")
_lock = threading.Lock()
_lib = None

VIS_PINHOLE, VIS_CONE, VIS_QUAD, VIS_ONE = 0, 1, 2, 3
FRAME_CAMERA, FRAME_WORLD = 0, 1
INTERP_TRILINEAR, INTERP_NEAREST = 0, 1


def build(force: bool = False) -> str:
    """Compile fif_oracle.c into liboracle.so next to it (gcc, OpenMP, no FMA contraction)."""
    with _lock:
        if (not force and os.path.exists(_LIB_PATH)
                and os.path.getmtime(_LIB_PATH) >= os.path.getmtime(_SRC)):
            return _LIB_PATH
        tmp = _LIB_PATH + f".tmp{os.getpid()}"
        cmd = ["gcc", "-O2", "-std=gnu11", "-fopenmp", "-ffp-contract=off", "-fno-fast-math",
               "-fPIC", "-shared", _SRC, "-o", tmp, "-lm"]
        subprocess.run(cmd, check=True)
        os.replace(tmp, _LIB_PATH)
        return _LIB_PATH


class Grid(ctypes.Structure):
    _fields_ = [("origin", ctypes.c_double * 3), ("res", ctypes.c_double),
                ("nx", ctypes.c_int32), ("ny", ctypes.c_int32), ("nz", ctypes.c_int32),
                ("pad_", ctypes.c_int32)]


class Params(ctypes.Structure):
    _fields_ = [("half_fov", ctypes.c_double), ("v_alpha", ctypes.c_double),
                ("r_min", ctypes.c_double), ("r_max", ctypes.c_double), ("sigma", ctypes.c_double),
                ("fx", ctypes.c_double), ("fy", ctypes.c_double), ("cx", ctypes.c_double),
                ("cy", ctypes.c_double), ("width", ctypes.c_int32), ("height", ctypes.c_int32)]


def make_grid(origin, res, dims) -> Grid:
    g = Grid()
    for a in range(3):
        g.origin[a] = float(np.float32(origin[a]))
    g.res = float(np.float32(res))
    g.nx, g.ny, g.nz = (int(d) for d in dims)
    return g


def make_params(half_fov=np.pi / 4, v_alpha=0.5, r_min=0.1, r_max=8.0, sigma=1.0,
                fx=320.0, fy=320.0, cx=320.0, cy=320.0, width=640, height=640) -> Params:
    p = Params()
    p.half_fov, p.v_alpha, p.r_min, p.r_max, p.sigma = half_fov, v_alpha, r_min, r_max, sigma
    p.fx, p.fy, p.cx, p.cy = fx, fy, cx, cy
    p.width, p.height = int(width), int(height)
    return p


_D = ctypes.POINTER(ctypes.c_double)
_F = ctypes.POINTER(ctypes.c_float)
_L = ctypes.POINTER(ctypes.c_int64)
_I = ctypes.POINTER(ctypes.c_int32)


def lib():
    global _lib
    if _lib is None:
        build()
        L = ctypes.CDLL(_LIB_PATH)
        sig = {
            "or_num_threads": (ctypes.c_int, []),
            "or_quat_to_rot": (None, [_D, _D]),
            "or_quad_coeffs": (None, [ctypes.c_double, ctypes.c_double, _D]),
            "or_vr": (None, [_D, _D, _D]),
            "or_vr_grad": (None, [_D, _D, _D]),
            "or_vp": (None, [_D, _D]),
            "or_jac_global": (None, [_D, _D, _D, _D, _D]),
            "or_jac_local": (None, [_D, _D, _D, _D]),
            "or_fim_gauss": (None, [_D, ctypes.c_double, _D]),
            "or_in_shell_f32": (ctypes.c_int, [_F, _F, ctypes.c_float, ctypes.c_float]),
            "or_pinhole_visible_f32": (ctypes.c_int, [_F, _F, ctypes.c_float, ctypes.c_float,
                                                      ctypes.c_float, ctypes.c_float,
                                                      ctypes.c_float, ctypes.c_float]),
            "or_pc_fim": (None, [_F, ctypes.c_int64, _F, ctypes.c_int64, ctypes.POINTER(Params),
                                 ctypes.c_int, ctypes.c_int, _D]),
            "or_pc_counts": (None, [_F, ctypes.c_int64, _F, ctypes.c_int64, ctypes.POINTER(Params),
                                    _L, _L]),
            "or_field_nodes": (None, [_F, ctypes.c_int64, ctypes.POINTER(Grid), ctypes.POINTER(Params),
                                      _L, ctypes.c_int64, ctypes.c_int, _D]),
            "or_field_pairs": (ctypes.c_int64, [_F, ctypes.c_int64, ctypes.POINTER(Grid),
                                                ctypes.POINTER(Params), _L, ctypes.c_int64]),
            "or_query_cells": (None, [ctypes.POINTER(Grid), _D, ctypes.c_int64, ctypes.c_int,
                                      _L, _D, _D, _I]),
            "or_query_batch": (None, [_D, _D, _D, ctypes.c_int64, _D, ctypes.c_int, _D]),
            "or_logdet": (None, [_D, _D, _D]),
            "or_inverse6": (ctypes.c_int, [_D, _D]),
            "or_jacobi6": (None, [_D, _D, _D]),
            "or_metrics": (None, [_D, ctypes.c_int64, _D]),
            "or_eig_batch": (None, [_D, ctypes.c_int64, _D, _D]),
            "or_query_grad_batch": (None, [_D, _D, _D, _D, ctypes.c_int64, _D, _D, _D]),
        }
        for name, (res, args) in sig.items():
            fn = getattr(L, name)
            fn.restype = res
            fn.argtypes = args
        _lib = L
    return _lib


def _p(a, ctype):
    return a.ctypes.data_as(ctypes.POINTER(ctype))


def _f64(a):
    return np.ascontiguousarray(a, dtype=np.float64)


def _f32(a):
    return np.ascontiguousarray(a, dtype=np.float32)


def num_threads() -> int:
    return int(lib().or_num_threads())


def quat_to_rot(q) -> np.ndarray:
    q = _f64(q)
    R = np.zeros(9)
    lib().or_quat_to_rot(_p(q, ctypes.c_double), _p(R, ctypes.c_double))
    return R.reshape(3, 3)


def quad_coeffs(half_fov: float, v_alpha: float) -> np.ndarray:
    """(k0, k1, k2) from Eq. quadratic_conditions."""
    k = np.zeros(3)
    lib().or_quad_coeffs(float(half_fov), float(v_alpha), _p(k, ctypes.c_double))
    return k


def vr(z, k) -> np.ndarray:
    z, k = _f64(z), _f64(k)
    out = np.zeros(10)
    lib().or_vr(_p(z, ctypes.c_double), _p(k, ctypes.c_double), _p(out, ctypes.c_double))
    return out


def vr_grad(z, k) -> np.ndarray:
    z, k = _f64(z), _f64(k)
    out = np.zeros(30)
    lib().or_vr_grad(_p(z, ctypes.c_double), _p(k, ctypes.c_double), _p(out, ctypes.c_double))
    return out.reshape(3, 10)


def vp(p) -> np.ndarray:
    p = _f64(p)
    out = np.zeros(10)
    lib().or_vp(_p(p, ctypes.c_double), _p(out, ctypes.c_double))
    return out


def jac_global(pw, R, t, o=(0.0, 0.0, 0.0)) -> np.ndarray:
    pw, R, t, o = _f64(pw), _f64(R), _f64(t), _f64(o)
    J = np.zeros(18)
    lib().or_jac_global(*(_p(a, ctypes.c_double) for a in (pw, R, t, o, J)))
    return J.reshape(3, 6)


def jac_local(pw, R, t) -> np.ndarray:
    pw, R, t = _f64(pw), _f64(R), _f64(t)
    J = np.zeros(18)
    lib().or_jac_local(*(_p(a, ctypes.c_double) for a in (pw, R, t, J)))
    return J.reshape(3, 6)


def fim_gauss(J, sigma=1.0) -> np.ndarray:
    J = _f64(J)
    out = np.zeros(36)
    lib().or_fim_gauss(_p(J, ctypes.c_double), float(sigma), _p(out, ctypes.c_double))
    return out.reshape(6, 6)


def in_shell_f32(p, x, r_min, r_max) -> bool:
    p, x = _f32(p), _f32(x)
    return bool(lib().or_in_shell_f32(_p(p, ctypes.c_float), _p(x, ctypes.c_float),
                                      float(np.float32(r_min * r_min)), float(np.float32(r_max * r_max))))


def pc_fim(landmarks, poses, params: Params, vis=VIS_PINHOLE, frame=FRAME_CAMERA) -> np.ndarray:
    """Direct point-cloud FIM per pose, [m, 6, 6] (Eq. cost_info)."""
    lm, ps = _f32(landmarks).reshape(-1, 3), _f32(poses).reshape(-1, 7)
    out = np.zeros((ps.shape[0], 36))
    lib().or_pc_fim(_p(lm, ctypes.c_float), lm.shape[0], _p(ps, ctypes.c_float), ps.shape[0],
                    ctypes.byref(params), int(vis), int(frame), _p(out, ctypes.c_double))
    return out.reshape(-1, 6, 6)


def pc_counts(landmarks, poses, params: Params):
    lm, ps = _f32(landmarks).reshape(-1, 3), _f32(poses).reshape(-1, 7)
    a = np.zeros(ps.shape[0], np.int64)
    b = np.zeros(ps.shape[0], np.int64)
    lib().or_pc_counts(_p(lm, ctypes.c_float), lm.shape[0], _p(ps, ctypes.c_float), ps.shape[0],
                       ctypes.byref(params), _p(a, ctypes.c_int64), _p(b, ctypes.c_int64))
    return a, b


def field_nodes(landmarks, grid: Grid, params: Params, nodes, about_node=False) -> np.ndarray:
    """Positional information factors of the listed nodes, [cnt, 10, 6, 6] (Eq. general_info_pif)."""
    lm = _f32(landmarks).reshape(-1, 3)
    nd = np.ascontiguousarray(nodes, dtype=np.int64).reshape(-1)
    out = np.zeros((nd.shape[0], 360))
    lib().or_field_nodes(_p(lm, ctypes.c_float), lm.shape[0], ctypes.byref(grid), ctypes.byref(params),
                         _p(nd, ctypes.c_int64), nd.shape[0], int(bool(about_node)),
                         _p(out, ctypes.c_double))
    return out.reshape(-1, 10, 6, 6)


def field_pairs(landmarks, grid: Grid, params: Params, nodes) -> int:
    lm = _f32(landmarks).reshape(-1, 3)
    nd = np.ascontiguousarray(nodes, dtype=np.int64).reshape(-1)
    return int(lib().or_field_pairs(_p(lm, ctypes.c_float), lm.shape[0], ctypes.byref(grid),
                                    ctypes.byref(params), _p(nd, ctypes.c_int64), nd.shape[0]))


def query_cells(grid: Grid, poses, interp=INTERP_TRILINEAR):
    ps = _f64(poses).reshape(-1, 7)
    m = ps.shape[0]
    nodes = np.zeros((m, 8), np.int64)
    w = np.zeros((m, 8))
    dw = np.zeros((m, 8, 3))
    st = np.zeros(m, np.int32)
    lib().or_query_cells(ctypes.byref(grid), _p(ps, ctypes.c_double), m, int(interp),
                         _p(nodes, ctypes.c_int64), _p(w, ctypes.c_double), _p(dw, ctypes.c_double),
                         _p(st, ctypes.c_int32))
    return nodes, w, dw, st


def query(corners, w, poses, k, frame=FRAME_CAMERA) -> np.ndarray:
    """FIM per pose from the world-frame coefficient sets of its 8 corner nodes.

    corners: [m, 8, 10, 6, 6], w: [m, 8].  Returns [m, 6, 6]."""
    c, ww, ps, kk = _f64(corners), _f64(w), _f64(poses).reshape(-1, 7), _f64(k)
    m = ps.shape[0]
    out = np.zeros((m, 36))
    lib().or_query_batch(_p(c, ctypes.c_double), _p(ww, ctypes.c_double), _p(ps, ctypes.c_double), m,
                         _p(kk, ctypes.c_double), int(frame), _p(out, ctypes.c_double))
    return out.reshape(m, 6, 6)


def metrics(I) -> np.ndarray:
    """[m, 4]: trace, log|det|, sign(det), lambda_min."""
    A = _f64(I).reshape(-1, 36)
    out = np.zeros((A.shape[0], 4))
    lib().or_metrics(_p(A, ctypes.c_double), A.shape[0], _p(out, ctypes.c_double))
    return out


def logdet(I):
    A = _f64(I).reshape(36)
    a, s = np.zeros(1), np.zeros(1)
    lib().or_logdet(_p(A, ctypes.c_double), _p(a, ctypes.c_double), _p(s, ctypes.c_double))
    return float(a[0]), float(s[0])


def inverse6(I) -> np.ndarray:
    A = _f64(I).reshape(36)
    out = np.zeros(36)
    if lib().or_inverse6(_p(A, ctypes.c_double), _p(out, ctypes.c_double)) != 0:
        raise np.linalg.LinAlgError("singular")
    return out.reshape(6, 6)


def eig(I):
    A = _f64(I).reshape(-1, 36)
    ev = np.zeros((A.shape[0], 6))
    V = np.zeros((A.shape[0], 36))
    lib().or_eig_batch(_p(A, ctypes.c_double), A.shape[0], _p(ev, ctypes.c_double), _p(V, ctypes.c_double))
    return ev, V.reshape(-1, 6, 6)


def query_grad(corners, w, dw, poses, k, gm) -> np.ndarray:
    """Analytic gradient of sum_m gm[:, m] * (trace, log|det|, lambda_min)(I_c) with respect to
    (t, phi), phi a right perturbation R <- R exp(phi^).  Returns [m, 6]."""
    c, ww, dd = _f64(corners), _f64(w), _f64(dw)
    ps, kk, g = _f64(poses).reshape(-1, 7), _f64(k), _f64(gm).reshape(-1, 3)
    m = ps.shape[0]
    out = np.zeros((m, 6))
    lib().or_query_grad_batch(_p(c, ctypes.c_double), _p(ww, ctypes.c_double), _p(dd, ctypes.c_double),
                              _p(ps, ctypes.c_double), m, _p(kk, ctypes.c_double), _p(g, ctypes.c_double),
                              _p(out, ctypes.c_double))
    return out


# ---------------------------------------------------------------------------
# composite helpers (marshalling only; every number comes from the C routines)
# ---------------------------------------------------------------------------

def full_field(landmarks, grid: Grid, params: Params, about_node=False) -> np.ndarray:
    """Every node of the lattice: [nx*ny*nz, 10, 6, 6]."""
    n = grid.nx * grid.ny * grid.nz
    return field_nodes(landmarks, grid, params, np.arange(n), about_node=about_node)


def query_from_landmarks(landmarks, grid: Grid, params: Params, poses, interp=INTERP_TRILINEAR,
                         frame=FRAME_CAMERA, field=None):
    """Query poses against a field built on demand for only the corner nodes the poses touch.

    Returns (I [m,6,6], status [m], nodes [m,8], w [m,8], dw [m,8,3], corners [m,8,10,6,6])."""
    nodes, w, dw, st = query_cells(grid, poses, interp)
    if field is None:
        uniq, inv = np.unique(nodes.reshape(-1), return_inverse=True)
        blocks = field_nodes(landmarks, grid, params, uniq, about_node=False)
        corners = blocks[inv].reshape(nodes.shape[0], 8, 10, 6, 6)
    else:
        corners = field[nodes]
    k = quad_coeffs(params.half_fov, params.v_alpha)
    I = query(corners, w, poses, k, frame)
    return I, st, nodes, w, dw, corners


# ---------------------------------------------------------------------------
# GP visibility (Sec. V-B-2)
# ---------------------------------------------------------------------------

class _GPStruct(ctypes.Structure):
    _fields_ = [("axes", _D), ("W", _D), ("ns", ctypes.c_int32), ("pad_", ctypes.c_int32),
                ("l", ctypes.c_double), ("ks", ctypes.c_double), ("cos_alpha", ctypes.c_double)]


def _gp_sigs():
    L = lib()
    if getattr(L, "_gp_ready", False):
        return L
    sig = {
        "or_gp_weights": (ctypes.c_int, [_D, ctypes.c_int, ctypes.c_double, ctypes.c_double, _D]),
        "or_gp_vp": (None, [_D, ctypes.c_int, _D, ctypes.c_double, ctypes.c_double, _D, _D]),
        "or_gp_vr": (None, [_D, ctypes.c_int, ctypes.c_double, _D, _D]),
        "or_gp_visibility": (ctypes.c_double, [_D, ctypes.c_int, _D, ctypes.c_double, ctypes.c_double,
                                               ctypes.c_double, _D, _D]),
        "or_gp_log_marginal": (ctypes.c_double, [_D, ctypes.c_int, ctypes.c_double, ctypes.c_double, _D,
                                                 ctypes.c_int]),
        "or_gp_training": (None, [_D, ctypes.c_int, ctypes.c_double, ctypes.c_double, _D, ctypes.c_int, _D]),
        "or_field_nodes_gp": (None, [_F, ctypes.c_int64, ctypes.POINTER(Grid), ctypes.POINTER(Params),
                                     ctypes.POINTER(_GPStruct), _L, ctypes.c_int64, ctypes.c_int, _D]),
        "or_query_gp_batch": (None, [_D, _D, _D, ctypes.c_int64, ctypes.POINTER(_GPStruct), ctypes.c_int, _D]),
        "or_pc_fim_gp": (None, [_F, ctypes.c_int64, _D, ctypes.c_int64, ctypes.POINTER(Params),
                                ctypes.POINTER(_GPStruct), ctypes.c_int, _D]),
        "or_info_threshold": (None, [_F, ctypes.c_int64, ctypes.c_int, ctypes.POINTER(Params), ctypes.c_int,
                                     ctypes.POINTER(_GPStruct), ctypes.c_int, _D, _D]),
        "or_info_cost": (None, [_D, ctypes.c_int64, ctypes.c_double, ctypes.c_double, _D, _D]),
    }
    for name, (res, args) in sig.items():
        fn = getattr(L, name)
        fn.restype = res
        fn.argtypes = args
    L._gp_ready = True
    return L


class GP:
    """GP visibility model: sample optical axes z_g [ns, 3], SE length scale l, noise variance
    added to K^s, sigmoid sharpness k_s and half field of view alpha (Eq. sigmoid_vis_func)."""

    def __init__(self, axes, length_scale, noise=1e-10, ks=15.0, half_fov=math.pi / 4):
        self.axes = np.ascontiguousarray(axes, dtype=np.float64).reshape(-1, 3)
        self.ns = self.axes.shape[0]
        self.l, self.noise, self.ks, self.cos_alpha = float(length_scale), float(noise), float(ks), math.cos(half_fov)
        self.W = np.zeros((self.ns, self.ns))
        if _gp_sigs().or_gp_weights(_p(self.axes, ctypes.c_double), self.ns, self.l, self.noise,
                                    _p(self.W, ctypes.c_double)) != 0:
            raise np.linalg.LinAlgError("singular GP kernel matrix")
        self.s = _GPStruct(_p(self.axes, ctypes.c_double), _p(self.W, ctypes.c_double), self.ns, 0,
                           self.l, self.ks, self.cos_alpha)

    def vp(self, p):
        p = _f64(p)
        out = np.zeros(self.ns)
        _gp_sigs().or_gp_vp(_p(self.axes, ctypes.c_double), self.ns, _p(self.W, ctypes.c_double), self.ks,
                            self.cos_alpha, _p(p, ctypes.c_double), _p(out, ctypes.c_double))
        return out

    def vr(self, z):
        z = _f64(z)
        out = np.zeros(self.ns)
        _gp_sigs().or_gp_vr(_p(self.axes, ctypes.c_double), self.ns, self.l, _p(z, ctypes.c_double),
                            _p(out, ctypes.c_double))
        return out

    def visibility(self, z, p):
        z, p = _f64(z), _f64(p)
        return float(_gp_sigs().or_gp_visibility(_p(self.axes, ctypes.c_double), self.ns,
                                                 _p(self.W, ctypes.c_double), self.l, self.ks, self.cos_alpha,
                                                 _p(z, ctypes.c_double), _p(p, ctypes.c_double)))


def gp_log_marginal(axes, length_scale, noise, Y):
    axes = np.ascontiguousarray(axes, dtype=np.float64)
    Y = np.ascontiguousarray(Y, dtype=np.float64)
    return float(_gp_sigs().or_gp_log_marginal(_p(axes, ctypes.c_double), axes.shape[0], float(length_scale),
                                               float(noise), _p(Y, ctypes.c_double), Y.shape[0]))


def gp_training(axes, ks, half_fov, bearings):
    axes = np.ascontiguousarray(axes, dtype=np.float64)
    P = np.ascontiguousarray(bearings, dtype=np.float64).reshape(-1, 3)
    Y = np.zeros((P.shape[0], axes.shape[0]))
    _gp_sigs().or_gp_training(_p(axes, ctypes.c_double), axes.shape[0], float(ks), math.cos(half_fov),
                              _p(P, ctypes.c_double), P.shape[0], _p(Y, ctypes.c_double))
    return Y


def field_nodes_gp(landmarks, grid: Grid, params: Params, gp: GP, nodes, about_node=False,
                   basis="paper") -> np.ndarray:
    """[cnt, ns, 6, 6].  basis "paper": C_g = sum_i v_p,i[g] I_i with v_p = W v^s (Eq.
    general_info_pif with the GP's v_p); basis "sigmoid": D_g = sum_i v^s_g(u_i) I_i, the same
    sum with W replaced by the identity (so C = W D)."""
    lm = _f32(landmarks).reshape(-1, 3)
    nd = np.ascontiguousarray(nodes, dtype=np.int64).reshape(-1)
    out = np.zeros((nd.shape[0], gp.ns * 36))
    if basis == "paper":
        s = gp.s
    elif basis == "sigmoid":
        eye = np.eye(gp.ns)
        s = _GPStruct(_p(gp.axes, ctypes.c_double), _p(eye, ctypes.c_double), gp.ns, 0, gp.l, gp.ks, gp.cos_alpha)
    else:
        raise ValueError(basis)
    _gp_sigs().or_field_nodes_gp(_p(lm, ctypes.c_float), lm.shape[0], ctypes.byref(grid), ctypes.byref(params),
                                 ctypes.byref(s), _p(nd, ctypes.c_int64), nd.shape[0], int(bool(about_node)),
                                 _p(out, ctypes.c_double))
    return out.reshape(-1, gp.ns, 6, 6)


def query_gp(corners, w, poses, gp: GP, frame=FRAME_CAMERA) -> np.ndarray:
    c, ww, ps = _f64(corners), _f64(w), _f64(poses).reshape(-1, 7)
    out = np.zeros((ps.shape[0], 36))
    _gp_sigs().or_query_gp_batch(_p(c, ctypes.c_double), _p(ww, ctypes.c_double), _p(ps, ctypes.c_double),
                                 ps.shape[0], ctypes.byref(gp.s), int(frame), _p(out, ctypes.c_double))
    return out.reshape(-1, 6, 6)


def pc_fim_gp(landmarks, poses, params: Params, gp: GP, frame=FRAME_CAMERA) -> np.ndarray:
    lm, ps = _f32(landmarks).reshape(-1, 3), _f64(poses).reshape(-1, 7)
    out = np.zeros((ps.shape[0], 36))
    _gp_sigs().or_pc_fim_gp(_p(lm, ctypes.c_float), lm.shape[0], _p(ps, ctypes.c_double), ps.shape[0],
                            ctypes.byref(params), ctypes.byref(gp.s), int(frame), _p(out, ctypes.c_double))
    return out.reshape(-1, 6, 6)


def query_gp_from_landmarks(landmarks, grid: Grid, params: Params, gp: GP, poses, interp=INTERP_TRILINEAR,
                            frame=FRAME_CAMERA):
    """GP-field query of poses, the field built on demand at the corner nodes they touch.

    Returns (I [m,6,6], status [m], nodes [m,8], w [m,8])."""
    nodes, w, _, st = query_cells(grid, poses, interp)
    uniq, inv = np.unique(nodes.reshape(-1), return_inverse=True)
    blocks = field_nodes_gp(landmarks, grid, params, gp, uniq, about_node=False)
    corners = blocks[inv].reshape(nodes.shape[0], 8, gp.ns, 6, 6)
    I = query_gp(corners, w, poses, gp, frame)
    return I, st, nodes, w


# ---------------------------------------------------------------------------
# information threshold and potential cost (Sec. VI-B)
# ---------------------------------------------------------------------------

MODEL_POINTCLOUD, MODEL_QUAD, MODEL_GP = 0, 1, 2


def info_threshold(sets, params: Params, model=MODEL_POINTCLOUD, gp: GP | None = None, exclude_degenerate=True):
    """sets [n, M, 3] camera-frame landmarks -> (metrics [n, 4] = trace, log|det|, sign,
    lambda_min; thresholds [3] = mean trace, log|det|, lambda_min)."""
    S = _f32(sets)
    n, M = S.shape[0], S.shape[1]
    met = np.zeros((n, 4))
    thr = np.zeros(3)
    gps = ctypes.byref(gp.s) if gp is not None else None
    _gp_sigs().or_info_threshold(_p(S, ctypes.c_float), n, M, ctypes.byref(params), int(model), gps,
                                 int(bool(exclude_degenerate)), _p(met, ctypes.c_double), _p(thr, ctypes.c_double))
    return met, thr


def info_cost(v, eps, kq):
    """Eq. info_pot_cost: (c, dc/dv) for metric values v."""
    x = _f64(v).reshape(-1)
    c, dc = np.zeros_like(x), np.zeros_like(x)
    _gp_sigs().or_info_cost(_p(x, ctypes.c_double), x.shape[0], float(eps), float(kq), _p(c, ctypes.c_double),
                            _p(dc, ctypes.c_double))
    return c, dc
