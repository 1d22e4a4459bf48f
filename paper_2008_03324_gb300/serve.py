"""Continuous-batching request loop for pose-FIM queries on a device-resident field.

Planner requests (RRT* edges, trajectory samples: 8-4096 poses each) arrive over time.  The
loop admits a request when a slot is free and its bytes fit the in-flight memory budget, and
the request then lives on the device: its poses go into a device ring of pose slots (placed at
admission; copied while every stream is busy, on an upload stream that overlaps the batches in
flight, or else by the launch that takes them), and the next batch queries the ring in place
(one fif_query per contiguous run of requests), writing the metrics of each slot straight into
its page-locked host mirror.  Up to `streams` batches are in flight on separate CUDA streams,
so requests that arrive while a batch runs join the next one.  Completion is detected by
polling CUDA events against a deadline (no blocking waits).  Every result is independent of the batch it travelled in: the query of a pose
depends on that pose only.

The scheduler (`Scheduler`) is separate from the executor that owns the streams and buffers
(`CudaExecutor`), so admission, batching and deadlines can be exercised without a GPU.
"""
from __future__ import annotations

import time
from collections import deque
from dataclasses import dataclass

import numpy as np

BYTES_PER_POSE = 7 * 4 + 3 * 8 + 1 + 4   # pose in; metrics, sign, status out


@dataclass
class Result:
    metrics: np.ndarray      # [L, 3] float64: trace, log|det|, lambda_min
    sign: np.ndarray         # [L] int8
    status: np.ndarray       # [L] int32
    arrival: float = 0.0
    admitted: float = 0.0
    done: float = 0.0

    @property
    def latency(self):
        return self.done - self.arrival


class AdmissionError(RuntimeError):
    pass


class RequestRing:
    """Host-side bookkeeping of a ring of `capacity` pose slots in which admitted requests live,
    each in one contiguous range, from admission until its results are read.  Ranges are handed
    out in admission order (wrapping to the start when the end has no room) and come back in
    any order; the space of the oldest range is reused only once it is released."""

    def __init__(self, capacity: int):
        self.cap = int(capacity)
        self.live = deque()      # [offset, length, released] in admission order
        self.by_off = {}         # offset -> its entry in `live`
        self.tail = 0

    def alloc(self, n: int):
        if n > self.cap:
            return None
        if not self.live:
            off = 0
        else:
            head = self.live[0][0]
            if self.tail > head:                   # free: [tail, cap) and [0, head)
                if self.tail + n <= self.cap:
                    off = self.tail
                elif n <= head:
                    off = 0
                else:
                    return None
            else:                                  # wrapped: free [tail, head)
                if self.tail + n <= head:
                    off = self.tail
                else:
                    return None
        e = [off, n, False]
        self.live.append(e)
        self.by_off[off] = e
        self.tail = off + n
        return off

    def release(self, off: int):
        e = self.by_off.pop(off)          # KeyError: no live range there
        e[2] = True
        while self.live and self.live[0][2]:
            self.live.popleft()

    @property
    def in_use(self):
        return sum(e[1] for e in self.live)


def contiguous_runs(offsets, lengths):
    """[(offset, length)] of maximal runs of back-to-back ranges, in the given order."""
    runs = []
    for off, n in zip(offsets, lengths):
        if runs and runs[-1][0] + runs[-1][1] == off:
            runs[-1][1] += n
        else:
            runs.append([off, n])
    return [tuple(r) for r in runs]


class CudaExecutor:
    """Request state resident on the device: a ring of pose slots in device memory with a
    page-locked host mirror, into which the query writes each request's metrics, sign and status
    directly (device-addressable host memory, mapped on every system with unified addressing).
    A request's poses are placed in its ring range when it is admitted; while every stream is
    busy, the placed ranges are copied to the device on an upload stream (once enough poses
    wait), so that they are there when a stream frees; otherwise the launch that takes them
    copies them on its own stream.  A batch is one fif_query per contiguous run of ring ranges
    (one, or two where the batch wraps), reading the ring in place.  `n_streams` batches are in
    flight at once."""

    def __init__(self, fld, max_batch_poses: int, n_streams: int = 2, flags=None, ring_poses: int = 0):
        import torch
        from . import fif
        self.torch, self.fif = torch, fif
        self.field = fld
        self.flags = fif.Q_METRICS if flags is None else flags
        self.max_batch = int(max_batch_poses)
        cap = int(ring_poses) if ring_poses else 4 * self.max_batch
        cap = max(cap, self.max_batch)
        self.ring = RequestRing(cap)
        dev = fld.coeffs.device
        self.d_pose = torch.empty(cap, 7, dtype=torch.float32, device=dev)
        self.h_pose = torch.empty(cap, 7, dtype=torch.float32, pin_memory=True)
        self.h_met = torch.empty(cap, 3, dtype=torch.float64, pin_memory=True)
        self.h_sg = torch.empty(cap, dtype=torch.int8, pin_memory=True)
        self.h_st = torch.empty(cap, dtype=torch.int32, pin_memory=True)
        # numpy views of the pinned mirror: placing and reading a request is one memcpy each
        self.np_pose, self.np_met = self.h_pose.numpy(), self.h_met.numpy()
        self.np_sg, self.np_st = self.h_sg.numpy(), self.h_st.numpy()
        self.up_stream = torch.cuda.Stream(device=dev)
        self.up_event = torch.cuda.Event()      # re-recorded by every upload
        self.uploaded = False
        self.flush_min = 2048
        self.pending = []        # admitted ranges not yet copied to the device
        self.streams = [torch.cuda.Stream(device=dev) for _ in range(n_streams)]
        self.events = [torch.cuda.Event() for _ in range(n_streams)]   # re-recorded by every launch
        self.launches = 0
        self.uploads = 0

    @property
    def n_streams(self):
        return len(self.streams)

    def admit(self, poses):
        """Place an admitted request's poses in the ring; its offset, or None without room."""
        n = poses.shape[0]
        off = self.ring.alloc(n)
        if off is None:
            return None
        self.np_pose[off:off + n] = poses
        self.pending.append((off, n))
        return off

    def _upload(self, stream):
        # the pending ranges, one copy per contiguous run, then the event that later batches wait on
        for off, n in contiguous_runs(*zip(*self.pending)):
            self.d_pose[off:off + n].copy_(self.h_pose[off:off + n], non_blocking=True)
            self.uploads += 1
        self.up_event.record(stream)
        self.uploaded = True
        self.pending = []

    def flush(self):
        """While every stream is busy: copy the admitted ranges to the device on the upload
        stream, overlapping the batches in flight, once at least `flush_min` poses wait (the
        next launch copies whatever is left, on its own stream)."""
        if sum(n for _, n in self.pending) < self.flush_min:
            return
        with self.torch.cuda.stream(self.up_stream):
            self._upload(self.up_stream)

    def launch(self, slot: int, batch, offsets):
        """batch: the requests' [L, 7] arrays; offsets: their ring offsets, in ring order."""
        torch, fif = self.torch, self.fif
        s = self.streams[slot]
        if self.uploaded:
            s.wait_event(self.up_event)
        with torch.cuda.stream(s):
            if self.pending:
                self._upload(s)
            for off, n in contiguous_runs(offsets, [b.shape[0] for b in batch]):
                # the outputs go straight to the page-locked mirror (device-addressable host
                # memory): no device-to-host copy to issue or wait for
                fif.query(self.field.c, self.d_pose[off:off + n], self.flags, None, self.h_met[off:off + n],
                          self.h_sg[off:off + n], self.h_st[off:off + n], stream=s)
                self.launches += 1
            self.events[slot].record(s)

    def done(self, slot: int) -> bool:
        return self.events[slot].query()

    def results(self, slot: int, off: int, L: int):
        return (self.np_met[off:off + L].copy(), self.np_sg[off:off + L].copy(), self.np_st[off:off + L].copy())

    def release(self, off: int, L: int):
        self.ring.release(off)


class Scheduler:
    """Admission by slots and an in-flight memory budget; continuous batching over the
    executor's streams; completion polling with a per-batch deadline."""

    def __init__(self, executor, slots: int = 256, mem_budget_bytes: int = 64 << 20, deadline_s: float = 10.0):
        self.ex = executor
        self.slots = int(slots)
        self.mem_budget = int(mem_budget_bytes)
        self.deadline = float(deadline_s)
        self.in_use_slots = 0
        self.in_use_bytes = 0
        self.peak_bytes = 0
        self.peak_slots = 0
        self.batches_launched = 0

    def _fits(self, n):
        return self.in_use_slots < self.slots and self.in_use_bytes + n * BYTES_PER_POSE <= self.mem_budget

    def _admit(self, n):
        self.in_use_slots += 1
        self.in_use_bytes += n * BYTES_PER_POSE
        self.peak_bytes = max(self.peak_bytes, self.in_use_bytes)
        self.peak_slots = max(self.peak_slots, self.in_use_slots)

    def _release(self, n):
        self.in_use_slots -= 1
        self.in_use_bytes -= n * BYTES_PER_POSE

    def run(self, requests, arrivals=None, clock=time.perf_counter, sleep=time.sleep):
        """Serve `requests` (list of [L, 7] float32 arrays) arriving at `arrivals` seconds (open
        loop; None = all at t = 0).  Returns the list of Result in request order."""
        n_req = len(requests)
        if arrivals is None:
            arrivals = np.zeros(n_req)
        order = np.argsort(arrivals, kind="stable").tolist()
        arr = np.asarray(arrivals, dtype=np.float64).tolist()
        lengths = [int(r.shape[0]) for r in requests]
        for L in lengths:
            if L > self.ex.max_batch or L * BYTES_PER_POSE > self.mem_budget:
                raise AdmissionError(f"request of {L} poses exceeds the batch or memory limit")
        results = [Result(np.zeros((0, 3)), np.zeros(0, np.int8), np.zeros(0, np.int32)) for _ in range(n_req)]
        # executors that keep request state on the device place a request at admission
        # (admit -> handle, or None without room), copy the placed requests with flush, and
        # take the handles back at launch, results and release
        resident = hasattr(self.ex, "admit")
        handle = [None] * n_req
        t0 = clock()
        nxt, done = 0, 0
        waiting, ready = deque(), deque()
        inflight = {}            # stream slot -> (request ids, offsets, launch time)
        while done < n_req:
            now = clock() - t0
            while nxt < n_req and arr[order[nxt]] <= now:
                rid = order[nxt]
                results[rid].arrival = arr[rid]
                waiting.append(rid)
                nxt += 1
            while waiting and self._fits(lengths[waiting[0]]):
                rid = waiting[0]
                if resident:
                    handle[rid] = self.ex.admit(requests[rid])
                    if handle[rid] is None:
                        break
                waiting.popleft()
                self._admit(lengths[rid])
                results[rid].admitted = now
                ready.append(rid)
            for slot in list(inflight):
                rids, offs, launched = inflight[slot]
                if self.ex.done(slot):
                    tdone = clock() - t0
                    for rid, off in zip(rids, offs):
                        L = lengths[rid]
                        r = results[rid]
                        key = handle[rid] if resident else off
                        r.metrics, r.sign, r.status = self.ex.results(slot, key, L)
                        r.done = tdone
                        if resident:
                            self.ex.release(key, L)
                        self._release(L)
                    done += len(rids)
                    del inflight[slot]
                elif now - launched > self.deadline:
                    raise TimeoutError(f"batch on stream {slot} exceeded the {self.deadline} s deadline")
            free = [s for s in range(self.ex.n_streams) if s not in inflight]
            if resident and not (ready and free):
                self.ex.flush()        # copies overlap the batches in flight; a launch copies itself
            if ready and free:
                rids, offs, n = [], [], 0
                while ready and n + lengths[ready[0]] <= self.ex.max_batch:
                    rid = ready.popleft()
                    rids.append(rid)
                    offs.append(n)
                    n += lengths[rid]
                if resident:
                    self.ex.launch(free[0], [requests[r] for r in rids], [handle[r] for r in rids])
                else:
                    self.ex.launch(free[0], [requests[r] for r in rids])
                self.batches_launched += 1
                inflight[free[0]] = (rids, offs, clock() - t0)
            elif not inflight and not ready and not waiting and nxt < n_req:
                dt = arr[order[nxt]] - (clock() - t0)
                if dt > 2e-4:
                    sleep(dt - 1e-4)
        return results


class FifServer(Scheduler):
    """Scheduler + CUDA executor over a device-resident field."""

    def __init__(self, fld, max_batch_poses: int = 1 << 18, slots: int = 256, mem_budget_bytes: int = 64 << 20,
                 streams: int = 2, flags=None, deadline_s: float = 10.0, ring_poses: int = 0):
        # the ring holds every admitted request: the memory budget's worth of poses, at most
        # four batches (beyond that admission waits for ring space), at least one batch
        ring = ring_poses or max(max_batch_poses, min(mem_budget_bytes // BYTES_PER_POSE, 4 * max_batch_poses))
        super().__init__(CudaExecutor(fld, max_batch_poses, streams, flags, ring), slots, mem_budget_bytes,
                         deadline_s)

    @property
    def kernel_launches(self):
        return self.ex.launches


def latency_stats(results):
    lat = np.array([r.latency for r in results])
    return dict(p50_ms=float(np.percentile(lat, 50) * 1e3), p99_ms=float(np.percentile(lat, 99) * 1e3),
                mean_ms=float(lat.mean() * 1e3), max_ms=float(lat.max() * 1e3))
