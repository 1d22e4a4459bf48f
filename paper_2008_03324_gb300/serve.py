"""Continuous-batching request loop for pose-FIM queries on a device-resident field.

Planner requests (RRT* edges, trajectory samples: 8-4096 poses each) arrive over time.  The
loop admits a request when a slot is free and its bytes fit the in-flight memory budget,
packs every admitted request into the next batch (one pinned host buffer, one host-to-device
copy, one fif_query launch, one device-to-host copy of the metrics) and keeps up to `streams`
batches in flight on separate CUDA streams, so requests that arrive while a batch runs join
the next one.  Completion is detected by polling CUDA events against a deadline (no blocking
waits).  Every result is independent of the batch it travelled in: the query of a pose
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


class CudaExecutor:
    """Streams, pinned staging and device buffers for `n_streams` batches in flight."""

    def __init__(self, fld, max_batch_poses: int, n_streams: int = 2, flags=None):
        import torch
        from . import fif
        self.torch, self.fif = torch, fif
        self.field = fld
        self.flags = fif.Q_METRICS if flags is None else flags
        self.max_batch = int(max_batch_poses)
        dev = fld.coeffs.device
        self.bufs = []
        for _ in range(n_streams):
            self.bufs.append(dict(
                stream=torch.cuda.Stream(device=dev),
                h_pose=torch.empty(self.max_batch, 7, dtype=torch.float32, pin_memory=True),
                h_met=torch.empty(self.max_batch, 3, dtype=torch.float64, pin_memory=True),
                h_sg=torch.empty(self.max_batch, dtype=torch.int8, pin_memory=True),
                h_st=torch.empty(self.max_batch, dtype=torch.int32, pin_memory=True),
                d_pose=torch.empty(self.max_batch, 7, dtype=torch.float32, device=dev),
                d_met=torch.empty(self.max_batch, 3, dtype=torch.float64, device=dev),
                d_sg=torch.empty(self.max_batch, dtype=torch.int8, device=dev),
                d_st=torch.empty(self.max_batch, dtype=torch.int32, device=dev),
                event=None,
            ))
        # numpy views of the pinned staging buffers: packing and unpacking a request is one
        # memcpy each, without per-request tensor dispatch
        for b in self.bufs:
            b["np_pose"], b["np_met"] = b["h_pose"].numpy(), b["h_met"].numpy()
            b["np_sg"], b["np_st"] = b["h_sg"].numpy(), b["h_st"].numpy()
        self.launches = 0

    @property
    def n_streams(self):
        return len(self.bufs)

    def launch(self, slot: int, batch):
        """batch: list of [L, 7] float32 arrays packed back to back."""
        torch, fif = self.torch, self.fif
        b = self.bufs[slot]
        n = 0
        dst = b["np_pose"]
        for poses in batch:
            L = poses.shape[0]
            dst[n:n + L] = poses
            n += L
        s = b["stream"]
        with torch.cuda.stream(s):
            b["d_pose"][:n].copy_(b["h_pose"][:n], non_blocking=True)
            fif.query(self.field.c, b["d_pose"][:n], self.flags, None, b["d_met"][:n], b["d_sg"][:n],
                      b["d_st"][:n], stream=s)
            b["h_met"][:n].copy_(b["d_met"][:n], non_blocking=True)
            b["h_sg"][:n].copy_(b["d_sg"][:n], non_blocking=True)
            b["h_st"][:n].copy_(b["d_st"][:n], non_blocking=True)
            ev = torch.cuda.Event()
            ev.record(s)
        b["event"] = ev
        self.launches += 1

    def done(self, slot: int) -> bool:
        return self.bufs[slot]["event"].query()

    def results(self, slot: int, off: int, L: int):
        b = self.bufs[slot]
        return (b["np_met"][off:off + L].copy(), b["np_sg"][off:off + L].copy(), b["np_st"][off:off + L].copy())


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
                rid = waiting.popleft()
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
                        r.metrics, r.sign, r.status = self.ex.results(slot, off, L)
                        r.done = tdone
                        self._release(L)
                    done += len(rids)
                    del inflight[slot]
                elif now - launched > self.deadline:
                    raise TimeoutError(f"batch on stream {slot} exceeded the {self.deadline} s deadline")
            free = [s for s in range(self.ex.n_streams) if s not in inflight]
            if ready and free:
                rids, offs, n = [], [], 0
                while ready and n + lengths[ready[0]] <= self.ex.max_batch:
                    rid = ready.popleft()
                    rids.append(rid)
                    offs.append(n)
                    n += lengths[rid]
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
                 streams: int = 2, flags=None, deadline_s: float = 10.0):
        super().__init__(CudaExecutor(fld, max_batch_poses, streams, flags), slots, mem_budget_bytes, deadline_s)

    @property
    def kernel_launches(self):
        return self.ex.launches


def latency_stats(results):
    lat = np.array([r.latency for r in results])
    return dict(p50_ms=float(np.percentile(lat, 50) * 1e3), p99_ms=float(np.percentile(lat, 99) * 1e3),
                mean_ms=float(lat.mean() * 1e3), max_ms=float(lat.max() * 1e3))
