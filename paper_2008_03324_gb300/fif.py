"""ctypes binding of libfif.so (the C ABI in include/fif.h) -- argument marshalling only.

Every function here passes raw device pointers, sizes and the current CUDA stream to the
library; all arithmetic runs in the library's kernels.  There is no CPU fallback: if the
library is missing, :func:`lib` raises.

The same names as the C ABI: :func:`field_bytes`, :func:`field_init`,
:func:`build_workspace_bytes`, :func:`build`, :func:`query`, :func:`query_backward`,
:func:`pointcloud_fim`, :func:`field_save`, :func:`field_load`, :func:`device_error`, and for
the GP visibility model :func:`gp_row_stride`, :func:`gp_stride`, :func:`gp_aux_bytes`,
:func:`gp_upload`, :func:`gp_fit_length_scale`, :func:`gp_field_bytes`, :func:`field_init_gp`
(:class:`GPModel` holds an uploaded model).
:class:`Field` bundles a field with its torch-owned storage, and :class:`FifQuery` is the
autograd function whose backward is the library's hand-written adjoint.
"""
from __future__ import annotations

import ctypes
import math
import os
import threading

import torch

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "libfif.so")

# ---- constants (mirror include/fif.h) -------------------------------------------------
OK, EINVAL, ESIZE, EALIGN, ECUDA, ETIMEOUT, EIO, EFORMAT, ERANGE = 0, -1, -2, -3, -4, -5, -6, -7, -8
POSE_OUTSIDE, POSE_QUAT, POSE_NOT_PD, POSE_NAN = 1, 2, 4, 8
STORAGE_F32, STORAGE_BF16, STORAGE_TRACE, STORAGE_GP = 0, 1, 2, 3
MODEL_POINTCLOUD, MODEL_QUAD, MODEL_GP = 0, 1, 2
GP_MAX_SAMPLES = 96
Q_TRILINEAR, Q_NEAREST, Q_CAMERA, Q_WORLD, Q_GP_COMPENSATED = 0x0, 0x1, 0x0, 0x2, 0x4
Q_TRACE, Q_LOGDET, Q_LMIN, Q_METRICS = 0x10, 0x20, 0x40, 0x70
STRIDE = {STORAGE_F32: 216, STORAGE_BF16: 224, STORAGE_TRACE: 12}


class FifError(RuntimeError):
    def __init__(self, code, what=""):
        self.code = code
        super().__init__(f"{what}: {status_str(code)} ({code})")


class Grid(ctypes.Structure):
    _fields_ = [("origin", ctypes.c_float * 3), ("res", ctypes.c_float),
                ("nx", ctypes.c_int32), ("ny", ctypes.c_int32), ("nz", ctypes.c_int32)]


class Params(ctypes.Structure):
    _fields_ = [("half_fov", ctypes.c_double), ("v_alpha", ctypes.c_double), ("r_min", ctypes.c_double),
                ("r_max", ctypes.c_double), ("sigma", ctypes.c_double), ("bin_size", ctypes.c_float),
                ("reserved", ctypes.c_int32)]


class Pinhole(ctypes.Structure):
    _fields_ = [("fx", ctypes.c_float), ("fy", ctypes.c_float), ("cx", ctypes.c_float), ("cy", ctypes.c_float),
                ("width", ctypes.c_int32), ("height", ctypes.c_int32)]


class GPC(ctypes.Structure):
    _fields_ = [("n_samples", ctypes.c_int32), ("reserved", ctypes.c_int32), ("length_scale", ctypes.c_double),
                ("noise_var", ctypes.c_double), ("k_s", ctypes.c_double),
                ("axes", (ctypes.c_double * 3) * GP_MAX_SAMPLES), ("d_aux", ctypes.c_void_p)]


class FieldC(ctypes.Structure):
    _fields_ = [("grid", Grid), ("params", Params), ("storage", ctypes.c_int32), ("stride", ctypes.c_int32),
                ("coeffs", ctypes.c_void_p), ("bytes", ctypes.c_size_t), ("k", ctypes.c_double * 3),
                ("gp", GPC)]


_lib = None
_lock = threading.Lock()
_VP = ctypes.c_void_p
_I64 = ctypes.c_int64
_I32 = ctypes.c_int32

_SIGS = {
    "fif_version": (_I32, []),
    "fif_status_str": (ctypes.c_char_p, [_I32]),
    "fif_field_bytes": (ctypes.c_size_t, [ctypes.POINTER(Grid), _I32]),
    "fif_field_init": (_I32, [ctypes.POINTER(FieldC), ctypes.POINTER(Grid), ctypes.POINTER(Params), _I32, _VP,
                              ctypes.c_size_t]),
    "fif_build_workspace_bytes": (ctypes.c_size_t, [ctypes.POINTER(FieldC), _I64]),
    "fif_build": (_I32, [ctypes.POINTER(FieldC), _VP, _I64, _VP, ctypes.c_size_t, _VP]),
    "fif_build_static": (_I32, [ctypes.POINTER(FieldC), _VP, _I64, _VP]),
    "fif_build_slab": (_I32, [ctypes.POINTER(FieldC), _I32, _I32, _VP, _I64, _VP, ctypes.c_size_t, _VP]),
    "fif_slab_landmark_band": (_I32, [ctypes.POINTER(FieldC), _I32, _I32, ctypes.POINTER(ctypes.c_float),
                                      ctypes.POINTER(ctypes.c_float)]),
    "fif_build_update": (_I32, [ctypes.POINTER(FieldC), _VP, _I64, _I32, _VP, ctypes.c_size_t, _VP]),
    "fif_query": (_I32, [ctypes.POINTER(FieldC), _VP, _I64, _I32, _VP, _VP, _VP, _VP, _VP]),
    "fif_query_host_staging_bytes": (ctypes.c_size_t, [_I64]),
    "fif_query_host": (_I32, [ctypes.POINTER(FieldC), _VP, _I64, _I32, _VP, _VP, _VP, _VP, _I64, _VP,
                              ctypes.c_size_t, _VP, _VP]),
    "fif_query_backward": (_I32, [ctypes.POINTER(FieldC), _VP, _I64, _I32, _VP, _VP, _VP, _VP]),
    "fif_pointcloud_fim": (_I32, [_VP, _I64, ctypes.POINTER(Params), ctypes.POINTER(Pinhole), _VP, _I64, _I32,
                                  _VP, _VP, _VP, _VP, _VP]),
    "fif_field_save": (_I32, [ctypes.POINTER(FieldC), ctypes.c_char_p, _VP, _VP]),
    "fif_field_load": (_I32, [ctypes.POINTER(FieldC), ctypes.c_char_p, _VP, ctypes.c_size_t, _VP, _VP]),
    "fif_device_error": (_I32, [ctypes.POINTER(_I32), _I32, _VP]),
    "fif_set_wait_limit": (_I32, [ctypes.c_uint64]),
    "fif_gp_row_stride": (_I32, [_I32]),
    "fif_gp_stride": (_I32, [_I32]),
    "fif_gp_aux_bytes": (ctypes.c_size_t, [_I32]),
    "fif_gp_upload": (_I32, [ctypes.POINTER(GPC), _VP, ctypes.c_size_t, _VP]),
    "fif_gp_fit_length_scale": (_I32, [ctypes.POINTER(GPC), ctypes.c_double, ctypes.POINTER(ctypes.c_double), _I32,
                                       ctypes.c_double, ctypes.c_double, ctypes.POINTER(ctypes.c_double)]),
    "fif_gp_field_bytes": (ctypes.c_size_t, [ctypes.POINTER(Grid), _I32]),
    "fif_field_init_gp": (_I32, [ctypes.POINTER(FieldC), ctypes.POINTER(Grid), ctypes.POINTER(Params),
                                 ctypes.POINTER(GPC), _VP, ctypes.c_size_t]),
    "fif_info_threshold": (_I32, [ctypes.POINTER(Params), _I32, ctypes.POINTER(GPC), _VP, _I64, _I32, _I32, _VP, _VP,
                                  _VP, _VP]),
    "fif_info_cost": (_I32, [_VP, _I64, _I64, ctypes.c_double, ctypes.c_double, _VP, _VP, _VP]),
}
SYMBOLS = tuple(_SIGS)


def lib(path: str = LIB_PATH):
    """Load libfif.so (raises if it has not been built -- there is no fallback)."""
    global _lib
    with _lock:
        if _lib is None:
            if not os.path.exists(path):
                raise RuntimeError(f"{path} is missing: build it with `python -m paper_2008_03324_gb300.build`")
            L = ctypes.CDLL(path)
            for name, (res, args) in _SIGS.items():
                fn = getattr(L, name)
                fn.restype = res
                fn.argtypes = args
            _lib = L
    return _lib


def status_str(code: int) -> str:
    try:
        return lib().fif_status_str(int(code)).decode()
    except Exception:  # library not loadable
        return "unknown"


def _check(rc, what):
    if rc != OK:
        raise FifError(rc, what)


def _ptr(t):
    return None if t is None else ctypes.c_void_p(t.data_ptr())


def _stream(stream=None):
    s = stream if stream is not None else torch.cuda.current_stream()
    return ctypes.c_void_p(s.cuda_stream)


def make_grid(origin, res, dims) -> Grid:
    g = Grid()
    for a in range(3):
        g.origin[a] = float(origin[a])
    g.res = float(res)
    g.nx, g.ny, g.nz = (int(d) for d in dims)
    return g


def make_params(half_fov=math.pi / 4, v_alpha=0.5, r_min=0.1, r_max=8.0, sigma=1.0, bin_size=0.0) -> Params:
    p = Params()
    p.half_fov, p.v_alpha, p.r_min, p.r_max, p.sigma = half_fov, v_alpha, r_min, r_max, sigma
    p.bin_size = bin_size
    return p


def make_pinhole(fx=320.0, fy=320.0, cx=320.0, cy=320.0, width=640, height=640) -> Pinhole:
    c = Pinhole()
    c.fx, c.fy, c.cx, c.cy, c.width, c.height = fx, fy, cx, cy, int(width), int(height)
    return c


def field_bytes(grid: Grid, storage=STORAGE_F32) -> int:
    return int(lib().fif_field_bytes(ctypes.byref(grid), int(storage)))


def field_init(grid: Grid, params: Params, storage, coeffs: torch.Tensor) -> FieldC:
    f = FieldC()
    _check(lib().fif_field_init(ctypes.byref(f), ctypes.byref(grid), ctypes.byref(params), int(storage),
                                _ptr(coeffs), coeffs.numel() * coeffs.element_size()), "fif_field_init")
    return f


def gp_row_stride(n_samples: int) -> int:
    return int(lib().fif_gp_row_stride(int(n_samples)))


def gp_stride(n_samples: int) -> int:
    return int(lib().fif_gp_stride(int(n_samples)))


def gp_aux_bytes(n_samples: int) -> int:
    return int(lib().fif_gp_aux_bytes(int(n_samples)))


def gp_field_bytes(grid: Grid, n_samples: int) -> int:
    return int(lib().fif_gp_field_bytes(ctypes.byref(grid), int(n_samples)))


def _gp_struct(axes, length_scale, noise_var, k_s) -> GPC:
    g = GPC()
    ax = [tuple(float(v) for v in row) for row in axes]
    if not 1 <= len(ax) <= GP_MAX_SAMPLES:
        raise FifError(EINVAL, "GP sample count")
    g.n_samples = len(ax)
    g.length_scale, g.noise_var, g.k_s = float(length_scale), float(noise_var), float(k_s)
    for i, row in enumerate(ax):
        for c in range(3):
            g.axes[i][c] = row[c]
    return g


def gp_fit_length_scale(axes, bearings, half_fov=math.pi / 4, k_s=15.0, noise_var=1e-10, l_lo=0.05,
                        l_hi=5.0) -> float:
    """Maximum-marginal-likelihood length scale (fif_gp_fit_length_scale); bearings [m, 3]."""
    g = _gp_struct(axes, 1.0, noise_var, k_s)
    flat = [float(v) for row in bearings for v in row[:3]]
    arr = (ctypes.c_double * len(flat))(*flat)
    out = ctypes.c_double(0.0)
    _check(lib().fif_gp_fit_length_scale(ctypes.byref(g), float(half_fov), arr, len(flat) // 3, float(l_lo),
                                          float(l_hi), ctypes.byref(out)), "fif_gp_fit_length_scale")
    return float(out.value)


def gp_upload(gp: GPC, aux: torch.Tensor, stream=None):
    _check(lib().fif_gp_upload(ctypes.byref(gp), _ptr(aux), aux.numel() * aux.element_size(), _stream(stream)),
           "fif_gp_upload")


def field_init_gp(grid: Grid, params: Params, gp: GPC, coeffs: torch.Tensor) -> FieldC:
    f = FieldC()
    _check(lib().fif_field_init_gp(ctypes.byref(f), ctypes.byref(grid), ctypes.byref(params), ctypes.byref(gp),
                                   _ptr(coeffs), coeffs.numel() * coeffs.element_size()), "fif_field_init_gp")
    return f


class GPModel:
    """GP visibility model (Sec. V-B-2) resident on the device: sample optical axes [N_s, 3],
    SE length scale (fitted by maximum marginal likelihood when None, from `bearings`), noise
    variance on the diagonal of K^s and sigmoid sharpness k_s."""

    def __init__(self, axes, length_scale=None, noise_var=1e-10, k_s=15.0, half_fov=math.pi / 4, bearings=None,
                 device="cuda", stream=None):
        axes = [tuple(float(v) for v in row) for row in axes]
        if length_scale is None:
            if bearings is None:
                raise ValueError("length_scale or bearings is required")
            length_scale = gp_fit_length_scale(axes, bearings, half_fov, k_s, noise_var)
        self.c = _gp_struct(axes, length_scale, noise_var, k_s)
        self.aux = torch.zeros(gp_aux_bytes(len(axes)), dtype=torch.uint8, device=device)
        gp_upload(self.c, self.aux, stream)

    @property
    def n_samples(self):
        return int(self.c.n_samples)

    @property
    def length_scale(self):
        return float(self.c.length_scale)


def gp_struct(axes, length_scale, noise_var=1e-10, k_s=15.0) -> GPC:
    """A host GP model struct (not uploaded): enough for fif_info_threshold."""
    return _gp_struct(axes, length_scale, noise_var, k_s)


def info_threshold(params: Params, sets: torch.Tensor, model=MODEL_POINTCLOUD, gp: GPC | None = None,
                   exclude_degenerate=True, metrics=None, sign=None, threshold=None, stream=None):
    """fif_info_threshold: sets [n, m, 3] camera-frame float32 -> (metrics [n, 3] float64,
    thresholds [3] float64), both on the device."""
    assert sets.is_cuda and sets.dtype == torch.float32 and sets.is_contiguous() and sets.dim() == 3
    n, m = sets.shape[0], sets.shape[1]
    if metrics is None:
        metrics = torch.empty(n, 3, dtype=torch.float64, device=sets.device)
    if threshold is None:
        threshold = torch.empty(3, dtype=torch.float64, device=sets.device)
    _check(lib().fif_info_threshold(ctypes.byref(params), int(model), ctypes.byref(gp) if gp is not None else None,
                                    _ptr(sets), n, m, int(bool(exclude_degenerate)), _ptr(metrics), _ptr(sign),
                                    _ptr(threshold), _stream(stream)), "fif_info_threshold")
    return metrics, threshold


def info_cost(values: torch.Tensor, eps: float, k_q: float, column=None, cost=None, dcost=None, stream=None):
    """fif_info_cost of a float64 vector, or of one column of a contiguous [m, k] float64 matrix
    (column = index).  Returns (cost, dcost) [m] float64."""
    assert values.is_cuda and values.dtype == torch.float64 and values.is_contiguous()
    if column is None:
        m, stride, ptr = values.numel(), 1, values.data_ptr()
    else:
        m, stride = values.shape[0], values.shape[1]
        ptr = values.data_ptr() + 8 * int(column)
    if cost is None:
        cost = torch.empty(m, dtype=torch.float64, device=values.device)
    if dcost is None:
        dcost = torch.empty(m, dtype=torch.float64, device=values.device)
    _check(lib().fif_info_cost(ctypes.c_void_p(ptr), m, stride, float(eps), float(k_q), _ptr(cost), _ptr(dcost),
                               _stream(stream)), "fif_info_cost")
    return cost, dcost


class InfoCost(torch.autograd.Function):
    """cost = InfoCost.apply(metrics [m, 3] float64, column, eps, k_q) -> [m]: the information
    potential cost of one metric column (Eq. info_pot_cost); backward multiplies by dc/dv from
    the same kernel."""

    @staticmethod
    def forward(ctx, metrics, column, eps, k_q):
        met = metrics.detach().contiguous()
        cost, dcost = info_cost(met, eps, k_q, column=column)
        ctx.column = column
        ctx.save_for_backward(dcost)
        ctx.shape = met.shape
        return cost

    @staticmethod
    def backward(ctx, g):
        (dcost,) = ctx.saved_tensors
        grad = torch.zeros(ctx.shape, dtype=torch.float64, device=dcost.device)
        grad[:, ctx.column] = (g.to(torch.float64) * dcost).nan_to_num()
        return grad, None, None, None


def build_workspace_bytes(field: FieldC, n: int) -> int:
    return int(lib().fif_build_workspace_bytes(ctypes.byref(field), int(n)))


def build(field: FieldC, landmarks: torch.Tensor, workspace: torch.Tensor, stream=None):
    assert landmarks.is_cuda and landmarks.dtype == torch.float32 and landmarks.is_contiguous()
    _check(lib().fif_build(ctypes.byref(field), _ptr(landmarks), landmarks.shape[0], _ptr(workspace),
                           workspace.numel() * workspace.element_size(), _stream(stream)), "fif_build")


def build_update(field: FieldC, landmarks: torch.Tensor, sign: int, workspace: torch.Tensor, stream=None):
    """Add (sign=+1) or remove (sign=-1) landmarks' contributions to a built field."""
    assert landmarks.is_cuda and landmarks.dtype == torch.float32 and landmarks.is_contiguous()
    _check(lib().fif_build_update(ctypes.byref(field), _ptr(landmarks), landmarks.shape[0], int(sign),
                                  _ptr(workspace), workspace.numel() * workspace.element_size(), _stream(stream)),
           "fif_build_update")


def build_slab(field: FieldC, k_begin: int, k_end: int, landmarks: torch.Tensor, workspace: torch.Tensor,
               stream=None):
    """fif_build_slab: build only the nodes with k_begin <= k < k_end."""
    assert landmarks.is_cuda and landmarks.dtype == torch.float32 and landmarks.is_contiguous()
    _check(lib().fif_build_slab(ctypes.byref(field), int(k_begin), int(k_end), _ptr(landmarks), landmarks.shape[0],
                                _ptr(workspace), workspace.numel() * workspace.element_size(), _stream(stream)),
           "fif_build_slab")


def slab_landmark_band(field: FieldC, k_begin: int, k_end: int):
    """fif_slab_landmark_band: (z_lo, z_hi) of the landmarks the slab's build can use (host only)."""
    lo, hi = ctypes.c_float(0.0), ctypes.c_float(0.0)
    _check(lib().fif_slab_landmark_band(ctypes.byref(field), int(k_begin), int(k_end), ctypes.byref(lo),
                                        ctypes.byref(hi)), "fif_slab_landmark_band")
    return float(lo.value), float(hi.value)


BUILD_STATIC_SCRATCH_BYTES = 16 << 20


def build_static(field: FieldC, landmarks: torch.Tensor, stream=None):
    """fif_build without a workspace: the scratch is the library's fixed 16 MiB device array
    (for callers that cannot allocate; see include/fif.h).  Calls that overlap on the GPU race."""
    assert landmarks.is_cuda and landmarks.dtype == torch.float32 and landmarks.is_contiguous()
    _check(lib().fif_build_static(ctypes.byref(field), _ptr(landmarks), landmarks.shape[0], _stream(stream)),
           "fif_build_static")


def query(field: FieldC, poses: torch.Tensor, flags=Q_METRICS, fim=None, metrics=None, sign=None, status=None,
          stream=None):
    assert poses.is_cuda and poses.dtype == torch.float32 and poses.is_contiguous()
    _check(lib().fif_query(ctypes.byref(field), _ptr(poses), poses.shape[0], int(flags), _ptr(fim), _ptr(metrics),
                           _ptr(sign), _ptr(status), _stream(stream)), "fif_query")


def query_host_staging_bytes(chunk: int) -> int:
    return int(lib().fif_query_host_staging_bytes(int(chunk)))


def query_host(field: FieldC, poses: torch.Tensor, flags=Q_METRICS, fim=None, metrics=None, sign=None, status=None,
               chunk=1 << 18, staging=None, stream=None, copy_stream=None):
    """fif_query_host: poses and outputs are CPU tensors (pinned for overlapped copies); staging is
    a device uint8 tensor of at least query_host_staging_bytes(chunk) bytes; copy_stream a
    torch.cuda.Stream other than stream."""
    assert not poses.is_cuda and poses.dtype == torch.float32 and poses.is_contiguous()
    for t in (fim, metrics, sign, status):
        assert t is None or (not t.is_cuda and t.is_contiguous())
    assert staging is not None and staging.is_cuda and copy_stream is not None
    _check(lib().fif_query_host(ctypes.byref(field), _ptr(poses), poses.shape[0], int(flags), _ptr(fim), _ptr(metrics),
                                _ptr(sign), _ptr(status), int(chunk), _ptr(staging),
                                staging.numel() * staging.element_size(), _stream(stream), _stream(copy_stream)),
           "fif_query_host")


def query_backward(field: FieldC, poses, fim, grad_metrics, grad_pose, flags=Q_METRICS, stream=None):
    _check(lib().fif_query_backward(ctypes.byref(field), _ptr(poses), poses.shape[0], int(flags), _ptr(fim),
                                    _ptr(grad_metrics), _ptr(grad_pose), _stream(stream)), "fif_query_backward")


def pointcloud_fim(landmarks, params: Params, camera: Pinhole, poses, flags=Q_METRICS, fim=None, metrics=None,
                   sign=None, status=None, stream=None):
    _check(lib().fif_pointcloud_fim(_ptr(landmarks), landmarks.shape[0], ctypes.byref(params), ctypes.byref(camera),
                                    _ptr(poses), poses.shape[0], int(flags), _ptr(fim), _ptr(metrics), _ptr(sign),
                                    _ptr(status), _stream(stream)), "fif_pointcloud_fim")


def field_save(field: FieldC, path: str, stream=None):
    _check(lib().fif_field_save(ctypes.byref(field), path.encode(), None, _stream(stream)), "fif_field_save")


def field_load(path: str, coeffs: torch.Tensor, stream=None) -> FieldC:
    f = FieldC()
    _check(lib().fif_field_load(ctypes.byref(f), path.encode(), _ptr(coeffs), coeffs.numel() * coeffs.element_size(),
                                None, _stream(stream)), "fif_field_load")
    return f


def device_error(reset=True, stream=None) -> int:
    v = _I32(0)
    _check(lib().fif_device_error(ctypes.byref(v), int(bool(reset)), _stream(stream)), "fif_device_error")
    return int(v.value)


def set_wait_limit(limit_ns: int = 0):
    """fif_set_wait_limit: limit of every bounded device wait of the kernels launched afterwards
    (0 restores the default of 2 s)."""
    _check(lib().fif_set_wait_limit(int(limit_ns)), "fif_set_wait_limit")


# ---------------------------------------------------------------------------
# convenience objects
# ---------------------------------------------------------------------------

class Field:
    """A field with torch-owned device storage."""

    def __init__(self, origin, res, dims, params: Params | None = None, storage=STORAGE_F32, device="cuda",
                 gp: GPModel | None = None):
        self.grid = make_grid(origin, res, dims)
        self.params = params if params is not None else make_params()
        n_nodes = int(dims[0]) * int(dims[1]) * int(dims[2])
        self.storage = storage
        self.gp = gp
        self.dims = tuple(int(d) for d in dims)
        if storage == STORAGE_GP:
            if gp is None:
                raise FifError(EINVAL, "a GP field needs a GPModel")
            self.coeffs = torch.zeros(n_nodes, gp_stride(gp.n_samples), dtype=torch.float32, device=device)
            self.c = field_init_gp(self.grid, self.params, gp.c, self.coeffs)
            return
        nbytes = field_bytes(self.grid, storage)
        if nbytes == 0:
            raise FifError(EINVAL, "fif_field_bytes")
        dt = torch.bfloat16 if storage == STORAGE_BF16 else torch.float32
        self.coeffs = torch.zeros(n_nodes, STRIDE[storage], dtype=dt, device=device)
        self.c = field_init(self.grid, self.params, storage, self.coeffs)

    @property
    def n_nodes(self):
        return self.coeffs.shape[0]

    def with_params(self, params: Params) -> "Field":
        """The same coefficient storage queried with other parameters (the stored factor does not
        depend on the visibility coefficients, only the query does)."""
        other = object.__new__(Field)
        other.__dict__.update(self.__dict__)
        other.params = params
        if self.storage == STORAGE_GP:
            other.c = field_init_gp(self.grid, params, self.gp.c, self.coeffs)
        else:
            other.c = field_init(self.grid, params, self.storage, self.coeffs)
        return other

    def build(self, landmarks: torch.Tensor, workspace: torch.Tensor | None = None, stream=None):
        need = build_workspace_bytes(self.c, landmarks.shape[0])
        if workspace is None or workspace.numel() * workspace.element_size() < need:
            workspace = torch.empty(need, dtype=torch.uint8, device=self.coeffs.device)
        build(self.c, landmarks, workspace, stream)
        return workspace

    def query(self, poses, flags=Q_METRICS, want_fim=True, stream=None):
        m = poses.shape[0]
        dev = poses.device
        trace = self.storage == STORAGE_TRACE
        fim = torch.empty(m, 21, dtype=torch.float32, device=dev) if (want_fim and not trace) else None
        met = torch.empty(m, 3, dtype=torch.float64, device=dev)
        sg = None if trace else torch.empty(m, dtype=torch.int8, device=dev)
        st = torch.empty(m, dtype=torch.int32, device=dev)
        if trace:
            flags = Q_TRACE | Q_WORLD | (flags & Q_NEAREST)
        query(self.c, poses, flags, fim, met, sg, st, stream)
        return fim, met, sg, st


def build_stats(workspace: torch.Tensor, field: Field, n_landmarks: int):
    """(in-shell pairs, candidate pairs, dropped landmarks) counted by the last build (reads
    the statistics block at the end of the workspace)."""
    need = build_workspace_bytes(field.c, n_landmarks)
    # the statistics block is the last 256-byte-aligned block of the layout
    raw = workspace[need - 256: need - 256 + 32].view(torch.int64).cpu()
    return int(raw[0]), int(raw[1]), int(raw[2])


class FifQuery(torch.autograd.Function):
    """metrics = FifQuery.apply(t, phi, quat, field, flags) -> [m, 3] (trace, log|det|, lambda_min).

    The pose is (t, R(quat) exp(phi^)) evaluated at phi = 0: `phi` must be a zero [m, 3] tensor
    that only routes the gradient of the right (camera-frame) so(3) perturbation.  Backward
    runs the library's adjoint kernel and returns d/dt [m, 3] and d/dphi [m, 3]."""

    @staticmethod
    def forward(ctx, t, phi, quat, field: Field, flags=Q_METRICS):
        poses = torch.cat([t.detach(), quat.detach()], dim=1).to(torch.float32).contiguous()
        fim, met, sg, st = field.query(poses, flags)
        ctx.field = field
        ctx.flags = flags
        ctx.save_for_backward(poses, fim)
        ctx.mark_non_differentiable(sg, st)
        return met, sg, st

    @staticmethod
    def backward(ctx, g_met, g_sg=None, g_st=None):
        poses, fim = ctx.saved_tensors
        g = g_met.detach().to(torch.float64).contiguous()
        out = torch.empty(poses.shape[0], 6, dtype=torch.float32, device=poses.device)
        query_backward(ctx.field.c, poses, fim, g, out, ctx.flags & (Q_WORLD | Q_METRICS))
        return out[:, :3], out[:, 3:], None, None, None
