"""Multi-process host logic on CPU (gloo, world size 2): every rank takes a contiguous shard of
the poses with no data-path exchange, and the reported time is the maximum over ranks; the build
splits into z-slabs whose landmark bands give every node of a slab the same landmark set (and
the same FP64 oracle factors) as the whole map, and the slabs gathered by broadcast complete
every rank's copy of the field."""
import ctypes
import os
import socket

import numpy as np
import pytest
import torch
import torch.multiprocessing as mp

from paper_2008_03324_gb300 import dist


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _worker(rank, world, port, total, out):
    os.environ.update(RANK=str(rank), LOCAL_RANK=str(rank), WORLD_SIZE=str(world), MASTER_ADDR="127.0.0.1",
                      MASTER_PORT=str(port))
    assert dist.init(backend="gloo")
    start, stop = dist.shard(total, rank, world)
    t = 10.0 * (rank + 1)                      # a rank-dependent "time"
    tmax = dist.max_over_ranks(t)
    units = dist.sum_over_ranks(stop - start)
    dist.barrier()
    out.put((rank, start, stop, tmax, units))
    import torch.distributed as tdist
    tdist.destroy_process_group()


def test_shards_cover_everything_once():
    for total in (0, 1, 7, 1000, 4194305):
        for world in (1, 2, 3, 8):
            spans = [dist.shard(total, r, world) for r in range(world)]
            assert spans[0][0] == 0 and spans[-1][1] == total
            assert all(a[1] == b[0] for a, b in zip(spans, spans[1:]))
            sizes = [b - a for a, b in spans]
            assert max(sizes) - min(sizes) <= 1


@pytest.mark.timeout(120)
def test_two_gloo_ranks_max_time_and_units():
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_worker, args=(r, 2, port, 1001, q)) for r in range(2)]
    for p in procs:
        p.start()
    got = sorted(q.get(timeout=90) for _ in range(2))
    for p in procs:
        p.join(timeout=30)
        assert p.exitcode == 0
    (r0, s0, e0, t0, u0), (r1, s1, e1, t1, u1) = got
    assert (s0, e0, s1, e1) == (0, 501, 501, 1001)
    assert t0 == t1 == 20.0 and u0 == u1 == 1001


def test_slab_ranges_cover_the_lattice_once():
    for nz in (1, 2, 5, 7, 40, 80):
        for world in (1, 2, 3, 8):
            r = dist.slab_ranges(nz, world)
            assert r[0][0] == 0 and r[-1][1] == nz
            assert all(a[1] == b[0] for a, b in zip(r, r[1:]))
            assert all(k0 % 4 == 0 for k0, k1 in r if k1 > k0)


def _slab_worker(rank, world, port, out):
    os.environ.update(RANK=str(rank), LOCAL_RANK=str(rank), WORLD_SIZE=str(world), MASTER_ADDR="127.0.0.1",
                      MASTER_PORT=str(port))
    import oracle as O
    from paper_2008_03324_gb300 import fif, synth
    assert dist.init(backend="gloo")
    # a tall lattice (13 layers at 0.5 m) and a 2.5 m range shell, so that the slabs' bands cut the map
    spec = synth.GridSpec((0.0, 0.0, 0.0), 0.5, (9, 9, 13))
    sc = synth.room_landmarks(seed=4, n=3000, size=(4.0, 4.0, 6.0))
    field = fif.FieldC()
    g = fif.make_grid(spec.origin, spec.res, spec.dims)
    prm = fif.make_params(r_max=2.5)
    assert fif.lib().fif_field_init(ctypes.byref(field), ctypes.byref(g), ctypes.byref(prm), 0,
                                    ctypes.c_void_p(256), fif.field_bytes(g, 0)) == 0
    k0, k1 = dist.slab_ranges(spec.dims[2], world)[rank]
    band = fif.slab_landmark_band(field, k0, k1)
    sub = dist.slab_landmarks(sc.landmarks, band)
    # every node of the slab: the same in-shell landmark count and bitwise the same FP64 factor
    nxy = spec.dims[0] * spec.dims[1]
    nodes = np.arange(k0 * nxy, k1 * nxy)
    grid = O.make_grid(spec.origin, spec.res, spec.dims)
    oprm = O.make_params(r_max=2.5)
    same_pairs = O.field_pairs(sub, grid, oprm, nodes) == O.field_pairs(sc.landmarks, grid, oprm, nodes)
    same_field = np.array_equal(O.field_nodes(sub, grid, oprm, nodes), O.field_nodes(sc.landmarks, grid, oprm, nodes))
    # gather: rank r fills its slab rows with r + 1, the broadcasts complete both copies
    coeffs = torch.zeros(spec.n_nodes, 4, dtype=torch.float32)
    coeffs[k0 * nxy:k1 * nxy] = rank + 1
    dist.gather_slabs(coeffs, dist.slab_ranges(spec.dims[2], world), nxy)
    expect = torch.zeros_like(coeffs)
    for r, (a, b) in enumerate(dist.slab_ranges(spec.dims[2], world)):
        expect[a * nxy:b * nxy] = r + 1
    out.put((rank, len(sub) < len(sc.landmarks), same_pairs, same_field, bool(torch.equal(coeffs, expect))))
    import torch.distributed as tdist
    tdist.destroy_process_group()


@pytest.mark.timeout(180)
def test_two_gloo_ranks_slab_build_inputs_and_gather():
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_slab_worker, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    got = sorted(q.get(timeout=150) for _ in range(2))
    for p in procs:
        p.join(timeout=30)
        assert p.exitcode == 0
    for rank, cut, same_pairs, same_field, gathered in got:
        assert cut and same_pairs and same_field and gathered, (rank, cut, same_pairs, same_field, gathered)
