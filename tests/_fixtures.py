"""Shared test fixtures: the seeded workloads, oracle results cached per process, and the
packing of an oracle-built field into the library's documented storage layout."""
import functools
import math

import numpy as np

import oracle as O
from paper_2008_03324_gb300 import synth

TAU_F32 = 1e-5    # relative Frobenius bound for single-precision storage
TAU_BF16 = 1e-2   # relative Frobenius bound for bfloat16 storage

# sym packing order of the library (21 upper-triangular entries, row-major)
SYM_RC = [(r, c) for r in range(6) for c in range(r, 6)]
SYM_R = np.array([rc[0] for rc in SYM_RC])
SYM_C = np.array([rc[1] for rc in SYM_RC])
SYM_W = np.where(SYM_R == SYM_C, 1.0, 2.0)   # weight of an entry in the full Frobenius sum


def unpack21(x):
    """[..., 21] -> [..., 6, 6] symmetric."""
    x = np.asarray(x, dtype=np.float64)
    out = np.zeros(x.shape[:-1] + (6, 6))
    out[..., SYM_R, SYM_C] = x
    out[..., SYM_C, SYM_R] = x
    return out


def pack21(M):
    M = np.asarray(M)
    return M[..., SYM_R, SYM_C]


def fro(M):
    M = np.asarray(M, dtype=np.float64)
    return np.sqrt((M ** 2).sum(axis=(-2, -1)))


def rel_fro(A, B):
    """||A - B||_F / ||B||_F per matrix (full symmetric 6x6)."""
    return fro(np.asarray(A) - np.asarray(B)) / np.maximum(fro(B), 1e-300)


U32 = 2.0 ** -24   # unit roundoff of single precision
BLOCK_FLOOR = 16 * U32   # absolute floor of the per-block check, relative to the node's norm


def block_ratio(got, ref, tau, floor=BLOCK_FLOOR):
    """Per node and monomial block k of fields [N, 10, 6, 6] (float64):
    ||got_k - ref_k||_F / max(tau ||ref_k||_F, floor ||ref||_F), where ||ref||_F is the node's norm
    over all 10 blocks.  A block passes at <= 1: within tau of its own norm, or, for a block far
    smaller than its node, within a few single-precision roundings of the node's moments (every
    stored coefficient is a short integer combination of moment sums bounded by the node's
    norm).  A block that is wrong by 1 % at 1e-3 of the node's norm fails."""
    got = np.asarray(got, dtype=np.float64)
    ref = np.asarray(ref, dtype=np.float64)
    d = fro(got - ref)                          # [N, 10]
    rk = fro(ref)                               # [N, 10]
    node = np.sqrt((rk ** 2).sum(axis=1, keepdims=True))
    den = np.maximum(tau * rk, floor * node)
    return np.where(den > 0, d / np.where(den > 0, den, 1.0), np.where(d > 0, np.inf, 0.0))


# elements per monomial block of a node record: 21 for float32 records (stride 216), 22 for
# bfloat16 records (stride 224: entry 21 of each block is a zero pad)
BLOCK = {216: 21, 224: 22}


def pack_field(F_local, stride=216):
    """Oracle node-local coefficients [N, 10, 6, 6] -> library layout [N, stride] float32."""
    N = F_local.shape[0]
    blk = BLOCK[stride]
    out = np.zeros((N, stride), np.float32)
    out[:, :10 * blk].reshape(N, 10, blk)[:, :, :21] = F_local[:, :, SYM_R, SYM_C].astype(np.float32)
    return out


def unpack_field(buf):
    """Library layout [N, stride] (stride 216 or 224) -> [N, 10, 6, 6] float64."""
    buf = np.asarray(buf, dtype=np.float64)
    blk = BLOCK[buf.shape[1]]
    return unpack21(buf[:, :10 * blk].reshape(-1, 10, blk)[:, :, :21])


# ---------------------------------------------------------------------------
# workloads
# ---------------------------------------------------------------------------

ROOM = dict(seed=1, n=2000, grid=synth.ROOM_GRID, r_max=8.0, pose_seed=2, m=1000)
WAREHOUSE = dict(seed=2, n=200_000, grid=synth.WAREHOUSE_GRID, r_max=10.0)


@functools.lru_cache(maxsize=None)
def room_scene():
    return synth.room_landmarks(seed=ROOM["seed"], n=ROOM["n"])


@functools.lru_cache(maxsize=None)
def room_poses(m=1000):
    return synth.random_poses(ROOM["pose_seed"], m, (0, 0, 0), (10, 10, 3))


def oracle_grid(spec):
    return O.make_grid(spec.origin, spec.res, spec.dims)


@functools.lru_cache(maxsize=None)
def room_field_oracle(about_node: bool):
    sc = room_scene()
    return O.full_field(sc.landmarks, oracle_grid(ROOM["grid"]), O.make_params(r_max=ROOM["r_max"]),
                        about_node=about_node)


@functools.lru_cache(maxsize=None)
def warehouse_scene():
    return synth.warehouse(seed=WAREHOUSE["seed"], n=WAREHOUSE["n"])


def metric_tolerances(I_ref, tau):
    """Per-matrix bounds on the metric errors implied by ||dI||_F <= tau ||I||_F:
    |d trace| <= sqrt(6) tau ||I||, |d lambda_min| <= tau ||I||, |d log|det|| <= tau ||I|| ||I^-1||
    (first order, doubled)."""
    n = fro(I_ref)
    inv = np.array([fro(np.linalg.pinv(M)) for M in I_ref])
    return math.sqrt(6) * tau * n, tau * n, 2.0 * tau * n * inv


def round_bf16(x):
    """Round float64/float32 values to the nearest bfloat16 (ties to even), returned as float64."""
    f = np.ascontiguousarray(x, dtype=np.float32)
    u = f.view(np.uint32).astype(np.uint64)
    lsb = (u >> 16) & 1
    u = ((u + 0x7FFF + lsb) >> 16) << 16
    return u.astype(np.uint32).view(np.float32).astype(np.float64)


def local_to_world(F_local, spec, nodes=None):
    """Node-local coefficients [N, 10, 6, 6] -> the paper's world frame, C^w = M_c^T C M_c (FP64);
    row n belongs to lattice node nodes[n] (default: node n)."""
    F_local = np.asarray(F_local, dtype=np.float64)
    N = F_local.shape[0]
    idx = np.arange(N) if nodes is None else np.asarray(nodes, dtype=np.int64).reshape(-1)
    nx, ny = spec.dims[0], spec.dims[1]
    c = np.stack([spec.origin[0] + spec.res * (idx % nx), spec.origin[1] + spec.res * ((idx // nx) % ny),
                  spec.origin[2] + spec.res * (idx // (nx * ny))], axis=1)
    M = np.tile(np.eye(6), (N, 1, 1))
    S = np.zeros((N, 3, 3))
    S[:, 0, 1], S[:, 0, 2], S[:, 1, 2] = -c[:, 2], c[:, 1], -c[:, 0]
    S[:, 1, 0], S[:, 2, 0], S[:, 2, 1] = c[:, 2], -c[:, 1], c[:, 0]
    M[:, :3, 3:] = -S
    return np.einsum("nji,nkjl,nlm->nkim", M, F_local, M)


def build_c_client(out_dir):
    """Compile tests/abi_client.c, a plain C program against include/fif.h, and link it with the
    in-tree libfif.so and the CUDA runtime; returns the executable's path."""
    import os
    import subprocess
    root = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
    pkg = os.path.join(root, "paper_2008_03324_gb300")
    cuda = os.environ.get("CUDA_HOME", "/usr/local/cuda")
    exe = os.path.join(str(out_dir), "abi_client")
    cmd = ["gcc", "-std=c11", "-O2", "-Wall", "-Wextra", "-Werror", "-I", os.path.join(root, "include"),
           "-I", os.path.join(cuda, "include"), os.path.join(root, "tests", "abi_client.c"), "-o", exe,
           "-L", pkg, "-lfif", f"-Wl,-rpath,{pkg}", "-L", os.path.join(cuda, "lib64"), "-lcudart",
           f"-Wl,-rpath,{os.path.join(cuda, 'lib64')}", "-lm"]
    subprocess.run(cmd, check=True, capture_output=True, text=True)
    return exe


class OracleNodes:
    """Coefficient sets of lattice nodes built by the FP64 oracle on demand and cached: for test
    workloads whose lattice is too large to build whole (every node costs a pass over all
    landmarks), only the nodes that the poses under test touch."""

    def __init__(self, landmarks, spec, params):
        self.landmarks = landmarks
        self.spec = spec
        self.grid = oracle_grid(spec)
        self.params = params
        self.cache = {}

    def local(self, nodes):
        """[len(nodes), 10, 6, 6] node-local (about the node) coefficients."""
        nodes = np.asarray(nodes, dtype=np.int64).reshape(-1)
        missing = np.unique(nodes[[n not in self.cache for n in nodes.tolist()]])
        if missing.size:
            blocks = O.field_nodes(self.landmarks, self.grid, self.params, missing, about_node=True)
            for n, b in zip(missing.tolist(), blocks):
                self.cache[n] = b
        return np.stack([self.cache[n] for n in nodes.tolist()]) if nodes.size else np.zeros((0, 10, 6, 6))

    def world(self, nodes):
        nodes = np.asarray(nodes, dtype=np.int64)
        W = local_to_world(self.local(nodes), self.spec, nodes.reshape(-1))
        return W.reshape(nodes.shape + (10, 6, 6))

    def corners(self, poses):
        """(corners [m, 8, 10, 6, 6] world frame, w, dw, nodes) of the trilinear query cells."""
        nodes, w, dw, _ = O.query_cells(self.grid, poses)
        return self.world(nodes), w, dw, nodes
