"""The serving loop on the GPU: each request's metrics are bitwise identical alone and inside a
mixed stream of requests (the query of a pose depends on that pose only)."""
import numpy as np
import pytest
import torch

from paper_2008_03324_gb300 import synth
from tests import _fixtures as X

pytestmark = pytest.mark.gpu


def test_alone_equals_mixed_on_gpu():
    from paper_2008_03324_gb300 import build as B
    B.build()
    from paper_2008_03324_gb300 import fif, serve
    spec = X.ROOM["grid"]
    field = fif.Field(spec.origin, spec.res, spec.dims, fif.make_params(r_max=8.0))
    field.coeffs.copy_(torch.from_numpy(X.pack_field(X.room_field_oracle(True))))
    room = synth.Scene("room", X.room_scene().landmarks, np.zeros(3), np.array([10.0, 10.0, 3.0]), [])
    reqs = synth.request_stream(8, 120, room, zr=(0.5, 2.5), max_len=512)
    srv = serve.FifServer(field, max_batch_poses=1 << 14, slots=32, mem_budget_bytes=1 << 20)
    mixed = srv.run(reqs, synth.poisson_arrivals(9, len(reqs), 5000.0))
    assert srv.peak_bytes <= 1 << 20 and srv.batches_launched < len(reqs)
    for i in (0, 17, 63, 119):
        alone = serve.FifServer(field, max_batch_poses=1 << 14).run([reqs[i]])[0]
        np.testing.assert_array_equal(np.nan_to_num(alone.metrics), np.nan_to_num(mixed[i].metrics))
        np.testing.assert_array_equal(alone.sign, mixed[i].sign)
        np.testing.assert_array_equal(alone.status, mixed[i].status)


def test_resident_ring_wraps_and_matches_direct_queries():
    """Requests live in a small device ring from admission to completion: with the ring only a
    few batches long, placements wrap to its start (and a batch can run as two queries); every
    request's metrics equal a direct fif_query of its poses, bitwise."""
    from paper_2008_03324_gb300 import build as B
    B.build()
    from paper_2008_03324_gb300 import fif, serve
    spec = X.ROOM["grid"]
    field = fif.Field(spec.origin, spec.res, spec.dims, fif.make_params(r_max=8.0))
    field.coeffs.copy_(torch.from_numpy(X.pack_field(X.room_field_oracle(True))))
    room = synth.Scene("room", X.room_scene().landmarks, np.zeros(3), np.array([10.0, 10.0, 3.0]), [])
    reqs = synth.request_stream(12, 300, room, zr=(0.5, 2.5), max_len=512)
    srv = serve.FifServer(field, max_batch_poses=2048, slots=128, mem_budget_bytes=64 << 20, ring_poses=3000)
    got = srv.run(reqs, synth.poisson_arrivals(13, len(reqs), 20000.0))
    assert not srv.ex.ring.live and srv.ex.uploads > 0 and srv.kernel_launches >= srv.batches_launched
    allp = torch.from_numpy(np.concatenate(reqs, axis=0)).cuda()
    _, met, sg, st = field.query(allp)
    torch.cuda.synchronize()
    met, sg, st = met.cpu().numpy(), sg.cpu().numpy(), st.cpu().numpy()
    o = 0
    for r, q in zip(got, reqs):
        L = q.shape[0]
        np.testing.assert_array_equal(np.nan_to_num(r.metrics), np.nan_to_num(met[o:o + L]))
        np.testing.assert_array_equal(r.sign, sg[o:o + L])
        np.testing.assert_array_equal(r.status, st[o:o + L])
        o += L
    print(f"ring 3000 poses: {srv.batches_launched} batches, {srv.kernel_launches} queries, {srv.ex.uploads} uploads")
