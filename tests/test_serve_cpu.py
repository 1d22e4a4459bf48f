"""Host-side logic of the continuous-batching loop (no GPU): admission by slots and memory,
batching of requests that arrive while others run, result routing, and the deadline path."""
import numpy as np
import pytest

from paper_2008_03324_gb300 import serve


class FakeExecutor:
    """Completes a batch after `latency` polls; the 'metric' of a pose is a function of that
    pose only, so a request's result must not depend on its batch."""

    def __init__(self, max_batch=1000, n_streams=2, latency=3, never=False):
        self.max_batch, self.n_streams, self.latency, self.never = max_batch, n_streams, latency, never
        self.polls = {}
        self.data = {}
        self.batches = []

    def launch(self, slot, batch):
        poses = np.concatenate(batch, axis=0)
        self.batches.append([b.shape[0] for b in batch])
        self.data[slot] = poses
        self.polls[slot] = 0

    def done(self, slot):
        self.polls[slot] += 1
        return (not self.never) and self.polls[slot] >= self.latency

    def results(self, slot, off, L):
        p = self.data[slot][off:off + L].astype(np.float64)
        met = np.stack([p.sum(1), p[:, 0] * 2, p[:, 1] - p[:, 2]], axis=1)
        return met, np.sign(p[:, 3]).astype(np.int8), np.arange(off, off + L, dtype=np.int32) * 0


class FakeClock:
    def __init__(self, step=1e-4):
        self.t, self.step = 0.0, step

    def __call__(self):
        self.t += self.step
        return self.t

    def sleep(self, dt):
        self.t += dt


def make_requests(seed, n, lo=8, hi=200):
    rng = np.random.default_rng(seed)
    return [rng.standard_normal((int(rng.integers(lo, hi)), 7)).astype(np.float32) for _ in range(n)]


def expected(r):
    p = r.astype(np.float64)
    return np.stack([p.sum(1), p[:, 0] * 2, p[:, 1] - p[:, 2]], axis=1)


def test_results_are_routed_to_their_requests():
    reqs = make_requests(1, 60)
    ex = FakeExecutor()
    sch = serve.Scheduler(ex, slots=16, mem_budget_bytes=1 << 20)
    clk = FakeClock()
    arr = np.cumsum(np.full(60, 2e-4))
    res = sch.run(reqs, arr, clock=clk, sleep=clk.sleep)
    for r, q in zip(res, reqs):
        np.testing.assert_array_equal(r.metrics, expected(q))
        assert r.done >= r.arrival and r.latency >= 0
    assert sum(len(b) for b in ex.batches) == 60


def test_same_result_alone_and_in_a_mix():
    reqs = make_requests(2, 40)
    alone = serve.Scheduler(FakeExecutor(), slots=64).run([reqs[7]])[0]
    mixed = serve.Scheduler(FakeExecutor(), slots=64).run(reqs)[7]
    np.testing.assert_array_equal(alone.metrics, mixed.metrics)
    np.testing.assert_array_equal(alone.sign, mixed.sign)


def test_admission_never_exceeds_slots_or_memory():
    reqs = make_requests(3, 200, 50, 400)
    budget = 30_000
    ex = FakeExecutor(max_batch=500, latency=5)
    sch = serve.Scheduler(ex, slots=4, mem_budget_bytes=budget)
    clk = FakeClock()
    res = sch.run(reqs, None, clock=clk, sleep=clk.sleep)
    assert sch.peak_bytes <= budget and sch.peak_slots <= 4
    assert sch.in_use_bytes == 0 and sch.in_use_slots == 0
    for r, q in zip(res, reqs):
        np.testing.assert_array_equal(r.metrics, expected(q))


def test_requests_arriving_during_a_batch_join_the_next():
    """Continuous batching: with one stream busy, everything that arrives meanwhile goes out
    together in the next batch instead of one launch per request."""
    reqs = make_requests(4, 30, 10, 20)
    ex = FakeExecutor(max_batch=10_000, n_streams=1, latency=50)
    clk = FakeClock(step=1e-4)
    arr = np.linspace(0.0, 0.004, 30)
    serve.Scheduler(ex, slots=64).run(reqs, arr, clock=clk, sleep=clk.sleep)
    assert len(ex.batches) < 30
    assert max(len(b) for b in ex.batches) > 1


def test_oversized_request_is_refused():
    ex = FakeExecutor(max_batch=100)
    with pytest.raises(serve.AdmissionError):
        serve.Scheduler(ex).run([np.zeros((101, 7), np.float32)])
    with pytest.raises(serve.AdmissionError):
        serve.Scheduler(FakeExecutor(max_batch=10_000), mem_budget_bytes=1000).run([np.zeros((100, 7), np.float32)])


def test_deadline_raises_instead_of_hanging():
    ex = FakeExecutor(never=True)
    clk = FakeClock(step=0.01)
    with pytest.raises(TimeoutError):
        serve.Scheduler(ex, deadline_s=0.5).run(make_requests(5, 3), None, clock=clk, sleep=clk.sleep)


def test_request_ring_never_overlaps_live_ranges():
    """Random admissions and out-of-order releases: every range handed out lies inside the ring
    and overlaps no live range; a refusal happens only when no contiguous room exists."""
    rng = np.random.default_rng(11)
    ring = serve.RequestRing(1000)
    live = {}
    for _ in range(5000):
        if live and rng.random() < 0.45:
            off = list(live)[int(rng.integers(len(live)))]
            ring.release(off)
            del live[off]
            continue
        n = int(rng.integers(1, 300))
        off = ring.alloc(n)
        if off is None:
            assert live            # an empty ring takes any request that fits it
            continue
        assert 0 <= off and off + n <= 1000
        for o, m in live.items():
            assert off + n <= o or o + m <= off
        live[off] = n
    assert ring.alloc(1001) is None


def test_contiguous_runs():
    assert serve.contiguous_runs([0, 5, 9, 0, 3], [5, 4, 2, 3, 1]) == [(0, 11), (0, 4)]
    assert serve.contiguous_runs([], []) == []


class FakeResidentExecutor(FakeExecutor):
    """A request lives in a ring from admission to release (as CudaExecutor keeps it on the
    device); a batch reads the ring through the offsets it is given."""

    def __init__(self, ring=600, **kw):
        super().__init__(**kw)
        self.ring = serve.RequestRing(ring)
        self.store = np.zeros((ring, 7), np.float32)
        self.flushed = 0
        self.unflushed = []
        self.copied = set()
        self.runs = []

    def admit(self, poses):
        busy = bool(self.ring.live)
        off = self.ring.alloc(poses.shape[0])
        self.wraps = getattr(self, "wraps", 0) + int(busy and off == 0)
        if off is not None:
            self.store[off:off + poses.shape[0]] = poses
            self.unflushed.append(off)
        return off

    def flush(self):
        self.flushed += len(self.unflushed)
        self.copied.update(self.unflushed)
        self.unflushed = []

    def launch(self, slot, batch, offsets):
        self.flush()                       # the launch copies what is still waiting
        assert all(o in self.copied for o in offsets)
        self.runs.append(serve.contiguous_runs(offsets, [b.shape[0] for b in batch]))
        self.batches.append([b.shape[0] for b in batch])
        self.data[slot] = None
        self.polls[slot] = 0

    def results(self, slot, off, L):
        p = self.store[off:off + L].astype(np.float64)
        met = np.stack([p.sum(1), p[:, 0] * 2, p[:, 1] - p[:, 2]], axis=1)
        return met, np.sign(p[:, 3]).astype(np.int8), np.zeros(L, np.int32)

    def release(self, off, L):
        self.store[off:off + L] = np.nan        # a stale read after release would show
        self.ring.release(off)


def test_resident_requests_route_wrap_and_wait_for_ring_space():
    """Requests placed in a small ring at admission: results come from each request's own
    range (released ranges are poisoned), batches are at most two runs (one wrap), placements
    wrap to the ring start, and admission waits for ring space."""
    reqs = make_requests(5, 150, 20, 200)
    ex = FakeResidentExecutor(ring=600, max_batch=400)
    sch = serve.Scheduler(ex, slots=500, mem_budget_bytes=1 << 30)
    clk = FakeClock()
    res = sch.run(reqs, None, clock=clk, sleep=clk.sleep)      # all at once: the ring fills
    for r, q in zip(res, reqs):
        np.testing.assert_array_equal(r.metrics, expected(q))
    assert ex.flushed == 150 and sum(len(b) for b in ex.batches) == 150
    assert all(len(runs) <= 2 for runs in ex.runs)
    assert ex.wraps > 0                                     # placements wrapped to the ring start
    assert not ex.ring.live
