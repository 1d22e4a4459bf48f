"""Multi-process host logic on CPU (gloo, world size 2): every rank takes a contiguous shard of
the poses with no data-path exchange, and the reported time is the maximum over ranks."""
import os
import socket

import pytest
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
