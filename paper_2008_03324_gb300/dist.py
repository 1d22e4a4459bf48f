"""Multi-process helpers (one process per GPU, launched by torchrun).

The query path shards with no data-path exchange: every rank holds a replica of the field
and answers its own slice of the poses (weak scaling).  The build shards by z-slabs of the
lattice (Sec. VI-A-1: every node is independent): each rank builds its slab from the landmarks
in the slab's band (fif_slab_landmark_band), and one broadcast per rank of its slab, the only
data exchange, completes every replica.  The other collectives are the timing barrier and the
max-over-ranks of the measured time."""
from __future__ import annotations

import os

import torch
import torch.distributed as dist


def world() -> tuple[int, int, int]:
    """(rank, local_rank, world_size) from the torchrun environment (1 process when unset)."""
    return (int(os.environ.get("RANK", 0)), int(os.environ.get("LOCAL_RANK", 0)),
            int(os.environ.get("WORLD_SIZE", 1)))


def init(backend: str | None = None) -> bool:
    rank, local, ws = world()
    if ws <= 1 or dist.is_initialized():
        return ws > 1
    if backend is None:
        backend = "nccl" if torch.cuda.is_available() else "gloo"
    os.environ.setdefault("MASTER_ADDR", "127.0.0.1")
    dist.init_process_group(backend=backend, rank=rank, world_size=ws)
    return True


def shard(total: int, rank: int, world_size: int) -> tuple[int, int]:
    """Contiguous [start, stop) of `total` units for `rank`; sizes differ by at most one."""
    base, extra = divmod(total, world_size)
    start = rank * base + min(rank, extra)
    return start, start + base + (1 if rank < extra else 0)


def barrier():
    if dist.is_available() and dist.is_initialized():
        dist.barrier()


def max_over_ranks(x: float, device=None) -> float:
    if not (dist.is_available() and dist.is_initialized()):
        return float(x)
    t = torch.tensor([float(x)], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def sum_over_ranks(x: float, device=None) -> float:
    if not (dist.is_available() and dist.is_initialized()):
        return float(x)
    t = torch.tensor([float(x)], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.SUM)
    return float(t.item())


def slab_ranges(nz: int, world_size: int, align: int = 4) -> list[tuple[int, int]]:
    """Contiguous z-slabs [k_begin, k_end) of an nz-layer lattice, one per rank, cut at multiples
    of `align` (the build's brick depth, so no brick is shared) while there are enough layers; a
    rank may get an empty slab (k_begin == k_end) when there are more ranks than bricks."""
    bricks = -(-nz // align)
    out = []
    for r in range(world_size):
        b0, b1 = shard(bricks, r, world_size)
        out.append((min(nz, b0 * align), min(nz, b1 * align)))
    return out


def slab_landmarks(landmarks, band):
    """The landmarks whose z lies in band = (z_lo, z_hi), in their input order (numpy [n, 3])."""
    z = landmarks[:, 2]
    return landmarks[(z >= band[0]) & (z <= band[1])]


def gather_slabs(coeffs: torch.Tensor, ranges, nodes_per_layer: int):
    """Complete every rank's copy of the node-major storage coeffs [n_nodes, stride]: rank r
    broadcasts its rows [k_begin * nx ny, k_end * nx ny)."""
    if not (dist.is_available() and dist.is_initialized()):
        return
    for r, (k0, k1) in enumerate(ranges):
        if k1 > k0:
            dist.broadcast(coeffs[k0 * nodes_per_layer:k1 * nodes_per_layer], src=r)
