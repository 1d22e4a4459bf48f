"""Benchmark of the Fisher Information Field hot path on GB300.

Metric: pose-FIM queries/s (+ p99 latency, vs the GPU point-cloud FIM; build pairs/s).

Workload (the warehouse map): 200,000 landmarks on the surfaces of a 50 x 50 x 10 m hall
with 40 box obstacles (60 % on box faces, 40 % on the walls), field of 200 x 200 x 40 nodes
at 0.25 m (1.6M nodes, 1.38 GB in float32), range shell (0.1, 10] m, 90-degree field of
view, v_alpha = 0.5.  The field is built once and stays resident; one timed step is one
fif_query of 2^22 poses drawn uniformly over the lattice with uniform rotations, returning
the FIM and trace / log|det| / lambda_min.  The field (1.38 GB) is ten times the L2, and the
random positions defeat caching, so no L2 flush is needed between steps.

Also reported (same run): the build (pairs/s, FP32 roofline), the point-cloud baseline over
all 200,000 landmarks, end-to-end throughput through host buffers, a short open-loop serving
run (p50/p99 latency), the FP64 CPU oracle on a bounded sample, and SM clocks sampled
during the timed region.

Usage: python bench.py [--gpus N] [--steps K] [--warmup W] [--impl reference]
N > 1 runs under torchrun, one process per GPU, each rank holding a replica of the field and
answering its own 2^22 poses (weak scaling, no exchange on the data path); the field is also
built as z-slabs, one per rank, gathered into every replica by broadcasts (reported apart).
"""
from __future__ import annotations

import argparse
import json
import math
import os
import subprocess
import sys
import threading
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

METRIC = "pose-FIM queries/s + p99 latency vs GPU point-cloud FIM; build pairs/s"
WORKLOAD = ("warehouse 50x50x10 m, 200k landmarks (60% box faces / 40% walls, 40 boxes), "
            "field 200x200x40 nodes @0.25 m (1.6M nodes, fp32 216/node), r in (0.1, 10] m, "
            "FoV 90 deg, v_alpha 0.5; step = fif_query of 2^22 uniform-random poses "
            "(FIM + trace + log|det| + lambda_min)")
# algorithmic bytes of one pose's query: the 8 corner coefficient sets (210 floats each); the pose
# and the outputs are reported beside it
QUERY_BYTES_PER_POSE = 8 * 210 * 4
QUERY_IO_BYTES_PER_POSE = 7 * 4 + 21 * 4 + 3 * 8 + 1 + 4    # pose in; FIM, metrics, sign, status out
BF16_QUERY_BYTES_PER_POSE = 8 * 210 * 2
TRACE_QUERY_BYTES_PER_POSE = 8 * 10 * 4
# shell test 8, rsqrt 1, bearing and 1/n^2 4, products 26, 66 accumulations (46 FMA, 20 FADD) 112
BUILD_FLOPS_PER_PAIR = 151
# DRAM traffic of one query launch per pose, from one ncu capture of query_kernel on a 2^20-pose
# launch over the full warehouse field (read 7.192 GB + write 0.116 GB; traffic per pose does not
# depend on the batch for uniform-random poses; summary under profiles/), valid while the kernel
# sources hash to the recorded digest
QUERY_TRAFFIC = {"bytes_per_pose": (7.192873216e9 + 0.116033280e9) / 1048576,
                 "digest": "4c1b93af14d6619f"}
# the same for the GP query (N_s = 70), captured on the 200 x 200 x 8 lattice (read 11.720 GB +
# write 0.0111 GB for 262,144 poses)
GP_QUERY_TRAFFIC = {"bytes_per_pose": (11.720299264e9 + 0.011119872e9) / 262144, "n_samples": 70,
                    "digest": "ab6462b5c7319dfe"}
# FMA-pipe utilisation of build_kernel (ncu sm__pipe_fma_cycles_active on the 200 x 200 x 8
# lattice), valid while the build sources hash to the recorded digest
BUILD_PIPE = {"fma_pipe_active": 0.732, "digest": "807ecbe98429a5e4"}
# thread instructions per pose-landmark pair of pointcloud_kernel (ncu smsp__inst_executed x 32 /
# pairs on one full-wave launch over the 200,000 warehouse landmarks)
PC_INSTRUCTIONS = {"per_pair": 38000753042 * 32 / (77824 * 200000), "digest": "5e88b65bf0a71852"}
# GP build, per (in-shell pair, sample axis): sigmoid 10 (dot 6, shift 1, exp 1, add 1, rcp 1)
# + 15 moment accumulations 30; per pair: bearing products 16
GP_FLOPS_PER_PAIR_SAMPLE = 40
GP_FLOPS_PER_PAIR = 16
SMS = 152
FP32_LANES = 128
SM_MAX_MHZ = 2070.0
E2E_CHUNK = int(os.environ.get("FIF_E2E_CHUNK", 1 << 20))   # poses per chunk of the host-buffer query
PC_POSES = SMS * 4 * 128   # the point-cloud baseline's launch: one full wave


def query_source_digest(files=("query.cu", "gather.cuh", "fif_common.cuh")):
    """Hash of the kernel sources with // comments and blank lines removed (a comment edit
    leaves the recorded counters valid; any code change invalidates them)."""
    import hashlib
    import re
    h = hashlib.sha256()
    for f in files:
        with open(os.path.join(ROOT, "paper_2008_03324_gb300", "csrc", f)) as fh:
            for line in fh:
                code = re.sub(r"//.*", "", line).rstrip()
                if code:
                    h.update(code.encode() + b"\n")
    return h.hexdigest()[:16]


def _peaks():
    path = os.path.join(ROOT, "MEASURED_PEAKS.json")
    try:
        with open(path) as f:
            d = json.load(f)
        return float(d["hbm_gbs"]), "measured"
    except Exception:
        return 6800.0, "fallback"


class ClockSampler:
    """nvidia-smi clocks and throttle reasons sampled every 100 ms while active.  Entering waits
    (at most 5 s) for the first sample, so that sampling runs before the work starts; mark() and
    summary() keep only the samples taken between the marks (the GPU under load)."""

    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index=0):
        self.gpu = gpu_index
        self.proc = None
        self.lines = []
        self.marks = []

    def __enter__(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", str(self.gpu), f"--query-gpu={self.FIELDS}", "--format=csv,noheader,nounits",
                 "-lms", "100"], stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.t = threading.Thread(target=self._read, daemon=True)
            self.t.start()
            t0 = time.monotonic()
            while not self.lines and self.proc.poll() is None and time.monotonic() - t0 < 5.0:
                time.sleep(0.01)
        except Exception:
            self.proc = None
        return self

    def _read(self):
        for line in self.proc.stdout:
            self.lines.append((time.monotonic(), line.strip()))

    def mark(self):
        self.marks.append(time.monotonic())

    def __exit__(self, *a):
        if self.proc is not None:
            self.proc.terminate()
            try:
                self.proc.wait(timeout=2)
            except Exception:
                self.proc.kill()

    def summary(self):
        sm, mx, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        # the window between the marks, widened by one sampling period so that a window shorter
        # than the period still holds the sample taken as it ran
        lo, hi = (self.marks[0] - 0.1, self.marks[-1] + 0.1) if len(self.marks) >= 2 else (-np.inf, np.inf)
        for t, ln in self.lines:
            if not lo <= t <= hi:
                continue
            parts = [p.strip() for p in ln.split(",")]
            if len(parts) < 9:
                continue
            try:
                sm.append(float(parts[1]))
                mx.append(float(parts[2]))
            except ValueError:
                continue
            for n, v in zip(names, parts[5:9]):
                if v.lower().startswith("active"):
                    reasons.add(n)
        if not sm:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["unsampled"], "samples": 0}
        return {"sm_mhz": float(np.median(sm)), "sm_max_mhz": float(max(mx)), "reasons": sorted(reasons),
                "samples": len(sm)}


def time_events(fn, steps, warmup, stream):
    import torch
    for _ in range(warmup):
        fn()
    torch.cuda.synchronize()
    evs = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(steps)]
    for a, b in evs:
        a.record(stream)
        fn()
        b.record(stream)
    torch.cuda.synchronize()
    return [a.elapsed_time(b) for a, b in evs]


def probe_lib():
    """The benchmark's FP32 FMA throughput probe (libfif_probe.so, built beside the product
    library from csrc/probe/; not part of the product ABI):
    fif_fma_probe(d_sink, blocks, iters, packed, stream) -> status."""
    import ctypes
    from paper_2008_03324_gb300 import build as B
    B.build()
    L = ctypes.CDLL(B.PROBE_LIB)
    L.fif_fma_probe.restype = ctypes.c_int32
    L.fif_fma_probe.argtypes = [ctypes.c_void_p, ctypes.c_int64, ctypes.c_int32, ctypes.c_int32, ctypes.c_void_p]
    return L


def fma_probe(sink, blocks, iters, packed, stream):
    """One probe launch: blocks CTAs of 256 threads, 2 * 8 * iters flops per thread, on `stream`."""
    import ctypes
    assert sink.is_cuda and sink.dtype.itemsize == 4 and sink.numel() >= blocks * 256
    rc = probe_lib().fif_fma_probe(ctypes.c_void_p(sink.data_ptr()), int(blocks), int(iters), int(bool(packed)),
                                   ctypes.c_void_p(stream.cuda_stream))
    if rc != 0:
        raise RuntimeError(f"fif_fma_probe: {rc}")


def fma_probe_tflops(dev, stream, blocks=8 * 152, iters=1 << 14):
    """Measured FP32 FMA throughput of this GPU (fif_fma_probe: eight independent chains per
    thread, scalar or packed f32x2), best of five launches: context for the nominal peak the
    ALU-bound build is reported against."""
    import torch
    sink = torch.empty(blocks * 256, dtype=torch.float32, device=dev)
    out = {}
    for name, packed in (("scalar", False), ("packed_f32x2", True)):
        t = time_events(lambda: fma_probe(sink, blocks, iters, packed, stream), 5, 2, stream)
        out[name] = 2 * 8 * iters * blocks * 256 / (min(t) * 1e-3) / 1e12
    assert bool(torch.isfinite(sink).all())
    return out


def cpu_baseline(scene, spec, r_max, seed=123, n_poses=256, min_query_s=2.0):
    """The FP64 oracle on a bounded sample of the same workload, on the host cores:
    build the corner nodes of `n_poses` random poses (timed: pairs/s), then query them
    repeatedly for at least `min_query_s` (timed: queries/s including the metrics)."""
    import oracle as O
    from paper_2008_03324_gb300 import synth
    O.build()
    poses = synth.random_poses(seed, n_poses, spec.lo, spec.hi)
    grid = O.make_grid(spec.origin, spec.res, spec.dims)
    prm = O.make_params(r_max=r_max, v_alpha=0.5)
    nodes, w, dw, st = O.query_cells(grid, poses)
    uniq, inv = np.unique(nodes.reshape(-1), return_inverse=True)
    t0 = time.perf_counter()
    blocks = O.field_nodes(scene.landmarks, grid, prm, uniq)
    t_build = time.perf_counter() - t0
    pairs = O.field_pairs(scene.landmarks, grid, prm, uniq)
    corners = blocks[inv].reshape(n_poses, 8, 10, 6, 6)
    k = O.quad_coeffs(prm.half_fov, prm.v_alpha)
    reps, t0 = 0, time.perf_counter()
    while True:
        I = O.query(corners, w, poses, k)
        O.metrics(I)
        reps += 1
        if time.perf_counter() - t0 >= min_query_s:
            break
    t_q = time.perf_counter() - t0
    return {
        "value": reps * n_poses / t_q, "unit": "queries/s", "cores": O.num_threads(), "kind": "oracle",
        "sample": (f"{n_poses} uniform-random warehouse poses; the oracle first builds their {len(uniq)} corner "
                   f"nodes over all {len(scene.landmarks)} landmarks ({t_build:.1f} s, "
                   f"{pairs / t_build:.3e} in-shell pairs/s), then queries them {reps} times "
                   f"(FIM + trace + log|det| + lambda_min, FP64)"),
        "build_pairs_per_s": pairs / t_build,
    }


def run_reference(args):
    """Reference arm: the FP64 CPU oracle as it stands, on the host cores."""
    from paper_2008_03324_gb300 import dist
    rank, _, ws = dist.world()
    if rank != 0:
        return 0
    import oracle as O
    from paper_2008_03324_gb300 import synth
    O.build()
    spec = synth.WAREHOUSE_GRID
    scene = synth.warehouse(seed=2, n=200_000)
    n_poses = args.ref_poses
    poses = synth.random_poses(7, n_poses, spec.lo, spec.hi)
    grid = O.make_grid(spec.origin, spec.res, spec.dims)
    prm = O.make_params(r_max=10.0, v_alpha=0.5)
    nodes, w, dw, st = O.query_cells(grid, poses)
    uniq, inv = np.unique(nodes.reshape(-1), return_inverse=True)
    corners = O.field_nodes(scene.landmarks, grid, prm, uniq)[inv].reshape(n_poses, 8, 10, 6, 6)
    k = O.quad_coeffs(prm.half_fov, prm.v_alpha)

    def step():
        I = O.query(corners, w, poses, k)
        O.metrics(I)

    for _ in range(args.warmup):
        step()
    times = []
    for _ in range(args.steps):
        t0 = time.perf_counter()
        step()
        times.append(time.perf_counter() - t0)
    ms = 1e3 * float(np.mean(times))
    val = n_poses / (ms * 1e-3)
    sample = (f"{n_poses} uniform-random warehouse poses per step, corner coefficient sets prebuilt by the oracle "
              f"(FIM + trace + log|det| + lambda_min, FP64)")
    line = {
        "impl": "reference", "metric": METRIC, "value": val, "unit": "queries/s", "n_gpus": args.gpus,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": ms, "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
        "config": {"workload": WORKLOAD + "; reference arm: FP64 CPU oracle, bounded sample", "poses_per_step": n_poses},
        "cpu_baseline": {"value": val, "unit": "queries/s", "cores": O.num_threads(), "kind": "oracle",
                         "sample": sample},
        "e2e": {"value": val, "unit": "queries/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
        "gpu_launches": 0,
    }
    print(json.dumps(line), flush=True)
    return 0


def gp_block(fif, synth, spec, lm, r_max, m, ns, dev, stream, hbm_peak, build_steps=2, query_steps=10):
    """GP-visibility field (Sec. V-B-2): N_s spherical-Fibonacci sample axes, length scale fitted
    by maximum marginal likelihood on 2000 random bearings, build on the lattice, then m
    uniform-random poses."""
    import torch
    t0 = time.perf_counter()
    l = fif.gp_fit_length_scale(synth.fibonacci_sphere(ns), synth.sphere_points(7, 2000))
    fit_s = time.perf_counter() - t0
    gp = fif.GPModel(synth.fibonacci_sphere(ns), l)
    fgp = fif.Field(spec.origin, spec.res, spec.dims, fif.make_params(r_max=r_max), storage=fif.STORAGE_GP, gp=gp)
    ws = torch.empty(fif.build_workspace_bytes(fgp.c, lm.shape[0]), dtype=torch.uint8, device=dev)
    tb = time_events(lambda: fif.build(fgp.c, lm, ws), build_steps, 1, stream)
    ins, cnd, _ = fif.build_stats(ws, fgp, lm.shape[0])
    tb_ms = float(np.mean(tb))
    flops = ins * (GP_FLOPS_PER_PAIR_SAMPLE * ns + GP_FLOPS_PER_PAIR) / (tb_ms * 1e-3) / 1e12
    nominal_fp32 = SMS * FP32_LANES * 2 * SM_MAX_MHZ * 1e6 / 1e12
    poses = torch.from_numpy(synth.random_poses(3000, m, spec.lo, spec.hi)).to(dev)
    met = torch.empty(m, 3, dtype=torch.float64, device=dev)
    sg = torch.empty(m, dtype=torch.int8, device=dev)
    st = torch.empty(m, dtype=torch.int32, device=dev)
    tq = time_events(lambda: fif.query(fgp.c, poses, fif.Q_METRICS, None, met, sg, st), query_steps, 3, stream)
    tq_ms = float(np.mean(tq))
    tc = time_events(lambda: fif.query(fgp.c, poses, fif.Q_METRICS | fif.Q_GP_COMPENSATED, None, met, sg, st),
                     max(3, query_steps // 2), 2, stream)
    tc_ms = float(np.mean(tc))
    bpp = 8 * fif.gp_stride(ns) * 4 + 7 * 4 + 3 * 8 + 1 + 4
    ach = m * bpp / (tq_ms * 1e-3) / 1e9
    assert fif.device_error() == 0
    out = {"n_samples": ns, "length_scale": l, "fit_s": fit_s, "field_bytes": fgp.coeffs.numel() * 4,
           "build_ms": tb_ms, "in_shell_pairs": ins, "build_pairs_per_s": ins / (tb_ms * 1e-3),
           "build_roofline": {"bound": "alu", "achieved": flops, "peak": nominal_fp32, "unit": "TFLOP/s",
                              "frac": flops / nominal_fp32,
                              "flops_per_pair": GP_FLOPS_PER_PAIR_SAMPLE * ns + GP_FLOPS_PER_PAIR},
           "queries_per_s": m / (tq_ms * 1e-3), "query_kernel_ms": tq_ms, "poses": m, "bytes_per_pose": bpp,
           "query_roofline": {"bound": "hbm", "achieved": ach, "peak": hbm_peak, "unit": "GB/s",
                              "frac": ach / hbm_peak,
                              "traffic": (GP_QUERY_TRAFFIC["bytes_per_pose"] * m
                                          if ns == GP_QUERY_TRAFFIC["n_samples"] and GP_QUERY_TRAFFIC["digest"] ==
                                          query_source_digest(("gp_query.cu", "fif_common.cuh")) else None)},
           "compensated_contraction": {"queries_per_s": m / (tc_ms * 1e-3), "query_kernel_ms": tc_ms,
                                       "frac": m * bpp / (tc_ms * 1e-3) / 1e9 / hbm_peak,
                                       "flag": "FIF_Q_GP_COMPENSATED (Dot2 contraction, error within 2 u kappa)"}}
    del fgp, ws, poses
    torch.cuda.empty_cache()
    return out


def method_accuracy(fif, synth, dev, n_poses=200):
    """Accuracy of the field representations against the exact point-cloud FIM (Sec. VII-A,
    Eq. fim_rel_diff): 1000 random landmarks in a 10 x 10 x 5 m box, fields on the 9 x 9 x 4 m
    region inside it at 0.5 m, poses at random nodes with uniform rotations, e = ||I_field -
    I_pc||_F / ||I_pc||_F in the camera frame (the field at its own node isolates the visibility
    model, as the paper's nearest-voxel test does).  Three aggregates over the poses that see a
    landmark: the mean and the median of e, and the ratio of sums sum ||I_field - I_pc|| / sum
    ||I_pc|| (per-pose e has a heavy tail where a landmark just outside the image sits close to
    the camera); two exact cameras with the paper's 90-degree horizontal field of view: the
    library's default 640 x 640 image and a 640 x 480 one.  Context for the paper's table, not a
    parity check."""
    import torch
    lm = synth.random_box(8, 1000)
    spec = synth.GridSpec((0.5, 0.5, 0.5), 0.5, (19, 19, 9))
    rng = np.random.default_rng(9)
    idx = rng.integers(0, spec.dims, size=(n_poses, 3))
    q = rng.standard_normal((n_poses, 4))
    q /= np.linalg.norm(q, axis=1, keepdims=True)
    poses = np.concatenate([np.asarray(spec.origin) + spec.res * idx, q], axis=1).astype(np.float32)
    P = torch.from_numpy(poses).to(dev)
    L = torch.from_numpy(lm).to(dev)
    prm_pc = fif.make_params(r_min=0.1, r_max=30.0)
    cams = {"640x640": fif.make_pinhole(), "640x480": fif.make_pinhole(cy=240.0, height=480)}
    fim_pc = {}
    for cname, cam in cams.items():
        fim_pc[cname] = torch.empty(n_poses, 21, device=dev)
        fif.pointcloud_fim(L, prm_pc, cam, P, 0, fim_pc[cname], None, None, None)
    w = torch.tensor([1.0 if r == c else 2.0 for r in range(6) for c in range(r, 6)], device=dev)
    fro = lambda x: torch.sqrt((w * x.double() ** 2).sum(1))
    out = {}
    models = [("Q-I-0.5", None, 0.5), ("Q-I-0.8", None, 0.8)] + [(f"G-I-{n}", n, 0.5) for n in (30, 50, 70, 96)]
    for name, ns, va in models:
        prm = fif.make_params(v_alpha=va, r_min=0.1, r_max=30.0)
        if ns is None:
            fld = fif.Field(spec.origin, spec.res, spec.dims, prm)
        else:
            axes = synth.fibonacci_sphere(ns)
            gp = fif.GPModel(axes, fif.gp_fit_length_scale(axes, synth.sphere_points(7, 2000)))
            fld = fif.Field(spec.origin, spec.res, spec.dims, prm, storage=fif.STORAGE_GP, gp=gp)
        fld.build(L)
        fim, _, _, _ = fld.query(P, fif.Q_NEAREST)
        out[name] = {}
        for cname in cams:
            ref = fro(fim_pc[cname])
            seen = (ref > 0).cpu().numpy()          # poses whose camera sees at least one landmark
            d = fro(fim - fim_pc[cname]).cpu().numpy()[seen]
            r = ref.cpu().numpy()[seen]
            e = d / r
            out[name][cname] = {"mean_pct": float(100 * e.mean()), "median_pct": float(100 * np.median(e)),
                                "ratio_of_sums_pct": float(100 * d.sum() / r.sum()), "poses": int(seen.sum())}
    out["paper_pct"] = {"Q-I-0.5": 64.26, "Q-I-0.8": 164.92, "G-I-30": 11.15, "G-I-50": 9.88, "G-I-70": 9.49}
    return out


def serving_run(fif, serve, field, reqs, rate, seed):
    srv = serve.FifServer(field, max_batch_poses=1 << 19, slots=512, mem_budget_bytes=256 << 20, streams=2)
    srv.run(reqs[:50], serve_arrivals(seed, 50, rate))   # warm-up
    arr = serve_arrivals(seed + 1, len(reqs), rate)
    t0 = time.perf_counter()
    res = srv.run(reqs, arr)
    wall = time.perf_counter() - t0
    n_poses = sum(r.shape[0] for r in reqs)
    return {"arrival_rate_req_per_s": rate, "requests": len(reqs), "poses": n_poses,
            "served_queries_per_s": n_poses / wall, "batches": srv.batches_launched,
            "peak_inflight_bytes": srv.peak_bytes, **serve.latency_stats(res)}


def serving_sweep(fif, serve, synth, scene, field, field16, n_requests):
    """Poisson request streams at 2k-50k requests/s (8-4096 poses each) on the fp32 and bf16
    fields; the 20k fp32 run is the headline p99."""
    reqs = synth.request_stream(3, n_requests, scene)
    sweep = {}
    for sname, sfield, bpp in (("f32", field, 6720), ("bf16", field16, 3360)):
        for rate in (2_000.0, 5_000.0, 10_000.0, 20_000.0, 50_000.0):
            r = serving_run(fif, serve, sfield, reqs, rate, 4)
            r["effective_gather_gbs"] = r["served_queries_per_s"] * bpp / 1e9
            sweep[f"{sname}@{int(rate)}"] = r
    return {"serving": sweep["f32@20000"],
            "serving_sweep": {k: {kk: v[kk] for kk in ("served_queries_per_s", "p50_ms", "p99_ms",
                                                         "effective_gather_gbs", "batches")}
                              for k, v in sweep.items()}}


def serve_arrivals(seed, count, rate):
    from paper_2008_03324_gb300 import synth
    return synth.poisson_arrivals(seed, count, rate)


def trace_block(fif, spec, lm, params, poses, met, st, wsb, stream, hbm_peak):
    """The positional trace factor (Sec. VI-A-2): build and world-frame trace query of the poses.
    Its field (12 floats per node, 77 MB on the warehouse lattice) stays in the 129 MB L2 while
    the poses stream through, so the query is bound by L2-to-SM sector traffic (8 corners x 64 B
    of sectors per pose), not by HBM; the fraction of the HBM copy bandwidth is reported for
    comparison only."""
    import torch
    m = poses.shape[0]
    ftr = fif.Field(spec.origin, spec.res, spec.dims, params, storage=fif.STORAGE_TRACE)
    ttb = time_events(lambda: fif.build(ftr.c, lm, wsb), 2, 1, stream)
    ttq = time_events(lambda: fif.query(ftr.c, poses, fif.Q_TRACE | fif.Q_WORLD, None, met, None, st), 10, 3,
                      stream)
    btr = TRACE_QUERY_BYTES_PER_POSE
    tq_ms = float(np.mean(ttq))
    res = {"field_bytes": ftr.coeffs.numel() * 4, "build_ms": float(np.mean(ttb)),
           "queries_per_s": m / (tq_ms * 1e-3), "bytes_per_pose": btr,
           "io_bytes_per_pose": 7 * 4 + 8 + 4, "kernel_ms": tq_ms,
           "roofline": {"bound": "l2", "achieved": m * btr / (tq_ms * 1e-3) / 1e9,
                        "peak": hbm_peak, "unit": "GB/s",
                        "frac": m * btr / (tq_ms * 1e-3) / 1e9 / hbm_peak,
                        "note": "the trace field fits in L2; frac is against the HBM copy bandwidth, for "
                                "comparison only (the sector traffic from L2 is 8 x 64 B per pose)",
                        "l2_sector_gbs": m * 8 * 64 / (tq_ms * 1e-3) / 1e9}}
    del ftr
    torch.cuda.empty_cache()
    return res


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=60)
    ap.add_argument("--warmup", type=int, default=5)
    ap.add_argument("--impl", default="gpu", choices=["gpu", "reference"])
    ap.add_argument("--poses", type=int, default=1 << 22)
    ap.add_argument("--phase", default="all", choices=["all", "query", "build", "gp", "pointcloud", "trace", "serve"],
                    help="build: time only the build; query: build once untimed, time only the query; "
                         "gp: only the GP-visibility field block")
    ap.add_argument("--gp-samples", type=int, default=70, help="GP sample axes N_s of the GP block")
    ap.add_argument("--storage", default="f32", choices=["f32", "bf16"],
                    help="field storage of the query phase (the full run times float32 first)")
    ap.add_argument("--build-nz", type=int, default=40, help="lattice z-layers (smaller for profiling)")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-large", action="store_true", help="skip the 2M-landmark building map")
    ap.add_argument("--serve-requests", type=int, default=1500)
    ap.add_argument("--ref-poses", type=int, default=1024,
                    help="poses per step of the reference arm (the FP64 oracle on the host cores)")
    args = ap.parse_args()
    if args.warmup < 3:
        args.warmup = 3
    if args.impl == "reference":
        return run_reference(args)

    import torch
    from paper_2008_03324_gb300 import build as B
    from paper_2008_03324_gb300 import dist, fif, serve, synth

    rank, local, ws = dist.world()
    if ws > 1:
        torch.cuda.set_device(local)
        dist.init()
    if rank == 0:
        B.build()
    dist.barrier()
    B.build()   # up to date by now: a no-op on the other ranks
    dev = torch.device("cuda", torch.cuda.current_device())
    stream = torch.cuda.current_stream()
    hbm_peak, peak_kind = _peaks()

    spec = synth.WAREHOUSE_GRID
    if args.build_nz != spec.dims[2]:
        spec = synth.GridSpec(spec.origin, spec.res, (spec.dims[0], spec.dims[1], args.build_nz))
    scene = synth.warehouse(seed=2, n=200_000)
    r_max = 10.0
    params = fif.make_params(r_max=r_max, v_alpha=0.5)
    lm = torch.from_numpy(scene.landmarks).to(dev)
    if args.phase == "gp":
        gpo = gp_block(fif, synth, spec, lm, r_max, args.poses, args.gp_samples, dev, stream, hbm_peak)
        if rank == 0:
            print(json.dumps({"metric": "GP-field queries/s", "value": gpo["queries_per_s"], "unit": "queries/s",
                              "n_gpus": ws, "config": {"workload": WORKLOAD, "lattice": list(spec.dims)},
                              "gp": gpo}), flush=True)
        return 0
    if args.phase == "serve":
        # the serving sweep alone, on fp32 and bf16 fields of the warehouse map
        sf = fif.Field(spec.origin, spec.res, spec.dims, params)
        sf16 = fif.Field(spec.origin, spec.res, spec.dims, params, storage=fif.STORAGE_BF16)
        sws = torch.empty(fif.build_workspace_bytes(sf.c, lm.shape[0]), dtype=torch.uint8, device=dev)
        fif.build(sf.c, lm, sws)
        fif.build(sf16.c, lm, sws)
        del sws
        so = serving_sweep(fif, serve, synth, scene, sf, sf16, args.serve_requests)
        if rank == 0:
            print(json.dumps({"metric": "served pose-FIM queries/s + p99 latency", "unit": "queries/s",
                              "value": so["serving"]["served_queries_per_s"], "n_gpus": ws,
                              "config": {"workload": WORKLOAD, "lattice": list(spec.dims)}, **so}), flush=True)
        return 0
    if args.phase == "trace":
        # the positional trace factor alone: build, then the world-frame trace query of the poses
        tposes = torch.from_numpy(synth.random_poses(1000 + rank, args.poses, spec.lo, spec.hi)).to(dev)
        tmet = torch.empty(args.poses, 3, dtype=torch.float64, device=dev)
        tst = torch.empty(args.poses, dtype=torch.int32, device=dev)
        tf = fif.Field(spec.origin, spec.res, spec.dims, params, storage=fif.STORAGE_TRACE)
        tws = torch.empty(fif.build_workspace_bytes(tf.c, lm.shape[0]), dtype=torch.uint8, device=dev)
        del tf
        tro = trace_block(fif, spec, lm, params, tposes, tmet, tst, tws, stream, hbm_peak)
        if rank == 0:
            print(json.dumps({"metric": "trace-factor queries/s", "value": tro["queries_per_s"], "unit": "queries/s",
                              "n_gpus": ws, "config": {"workload": WORKLOAD, "lattice": list(spec.dims)},
                              "trace_field": tro}), flush=True)
        return 0
    if args.phase == "pointcloud":
        # the point-cloud baseline alone: one full-wave launch over all landmarks per step
        pposes = torch.from_numpy(synth.random_poses(1000 + rank, PC_POSES, spec.lo, spec.hi)).to(dev)
        pmet = torch.empty(PC_POSES, 3, dtype=torch.float64, device=dev)
        tp = time_events(lambda: fif.pointcloud_fim(lm, params, fif.make_pinhole(), pposes, fif.Q_METRICS, None, pmet,
                                                    None, None), max(1, args.steps), args.warmup, stream)
        if rank == 0:
            print(json.dumps({"metric": "point-cloud FIM poses/s", "unit": "queries/s",
                              "value": PC_POSES / (float(np.mean(tp)) * 1e-3), "kernel_ms": float(np.mean(tp)),
                              "poses": PC_POSES, "landmarks": int(lm.shape[0])}), flush=True)
        return 0
    query_storage = fif.STORAGE_BF16 if (args.phase == "query" and args.storage == "bf16") else fif.STORAGE_F32
    field = fif.Field(spec.origin, spec.res, spec.dims, params, storage=query_storage)
    wsb = torch.empty(fif.build_workspace_bytes(field.c, lm.shape[0]), dtype=torch.uint8, device=dev)

    out = {}
    launches = 0
    # ---------------- build ----------------
    build_steps = 3 if args.phase != "query" else 1
    tb = time_events(lambda: fif.build(field.c, lm, wsb), build_steps, 1 if args.phase != "query" else 0, stream)
    inshell, cand, dropped = fif.build_stats(wsb, field, lm.shape[0])
    tb_ms = float(np.mean(tb))
    nominal_fp32 = SMS * FP32_LANES * 2 * SM_MAX_MHZ * 1e6 / 1e12
    build_tflops = inshell * BUILD_FLOPS_PER_PAIR / (tb_ms * 1e-3) / 1e12
    out["build"] = {
        "ms": tb_ms, "pairs_per_s": inshell / (tb_ms * 1e-3), "in_shell_pairs": inshell, "candidate_pairs": cand,
        "launches_per_build": 7,
        "roofline": {"bound": "alu", "achieved": build_tflops, "peak": nominal_fp32, "unit": "TFLOP/s",
                     "frac": build_tflops / nominal_fp32, "traffic": None,
                     "peak_kind": "nominal FP32: 152 SMs x 128 lanes x 2 x 2070 MHz",
                     "fma_pipe_active_ncu": (BUILD_PIPE["fma_pipe_active"] if BUILD_PIPE["digest"] ==
                                             query_source_digest(("build.cu", "landmark_stream.cuh", "fif_common.cuh"))
                                             else None),
                     "fma_probe_tflops": fma_probe_tflops(dev, stream)},
    }
    # ---------------- slab-partitioned build on N GPUs (Sec. VI-A-1: the nodes are independent) ----------------
    # each rank builds its z-slab from the landmarks in the slab's band; one broadcast per rank then
    # completes every replica (the replica built above is overwritten by the gathered slabs)
    if ws > 1:
        ranges = dist.slab_ranges(spec.dims[2], ws)
        k0, k1 = ranges[rank]
        nxy = spec.dims[0] * spec.dims[1]
        if k1 > k0:
            sub_np = dist.slab_landmarks(scene.landmarks, fif.slab_landmark_band(field.c, k0, k1))
        else:
            sub_np = scene.landmarks[:0]
        sub = torch.from_numpy(np.ascontiguousarray(sub_np)).to(dev)
        wss = torch.empty(fif.build_workspace_bytes(field.c, max(1, sub.shape[0])), dtype=torch.uint8, device=dev)
        ts = time_events(lambda: fif.build_slab(field.c, k0, k1, sub, wss) if k1 > k0 else None, build_steps, 1,
                         stream)
        ins_slab = fif.build_stats(wss, field, sub.shape[0])[0] if k1 > k0 else 0
        field.coeffs[: k0 * nxy].zero_()
        field.coeffs[k1 * nxy:].zero_()
        dist.barrier()
        tg = time_events(lambda: dist.gather_slabs(field.coeffs, ranges, nxy), 1, 0, stream)
        slab_ms = dist.max_over_ranks(float(np.mean(ts)), dev)
        gather_ms = dist.max_over_ranks(float(tg[0]), dev)
        ins_all = dist.sum_over_ranks(float(ins_slab), dev)
        out["build_sharded"] = {
            "ranks": ws, "slabs": ranges, "landmarks_this_rank": int(sub.shape[0]), "slab_ms_max": slab_ms,
            "gather_ms": gather_ms, "in_shell_pairs": ins_all, "pairs_per_s": ins_all / (slab_ms * 1e-3),
            "ms_total": slab_ms + gather_ms,
            "note": "z-slabs cut at multiples of the 4-layer brick; each slab from its landmark band; the "
                    "gathered field equals the one-GPU build bitwise (tested)"}
        del wss, sub

    # ---------------- incremental update (Sec. VI-A-1): add then remove 1,000 landmarks ----------------
    delta = torch.from_numpy(synth.random_box(seed=21, n=1000, size=(50.0, 50.0, 10.0))).to(dev)
    wsu = torch.empty(fif.build_workspace_bytes(field.c, delta.shape[0]), dtype=torch.uint8, device=dev)
    tu = time_events(lambda: (fif.build_update(field.c, delta, +1, wsu), fif.build_update(field.c, delta, -1, wsu)),
                     3, 1, stream)
    u_pairs = fif.build_stats(wsu, field, delta.shape[0])[0]
    u_ms = float(np.mean(tu)) / 2
    out["build"]["update"] = {"landmarks": int(delta.shape[0]), "ms_per_update": u_ms,
                              "in_shell_pairs": int(u_pairs), "pairs_per_s": u_pairs / (u_ms * 1e-3),
                              "note": "add then remove the same 1,000 random landmarks; only nodes within r_max change"}
    del wsu
    assert fif.device_error() == 0
    if args.phase == "build":
        if rank == 0:
            print(json.dumps({"metric": "build pairs/s", "unit": "pairs/s", "value": out["build"]["pairs_per_s"],
                              "n_gpus": ws, "config": {"workload": WORKLOAD, "lattice": list(spec.dims)},
                              "build": out["build"]}), flush=True)
        return 0

    # ---------------- query (the timed step) ----------------
    m = args.poses
    poses = torch.from_numpy(synth.random_poses(1000 + rank, m, spec.lo, spec.hi)).to(dev)
    fim = torch.empty(m, 21, dtype=torch.float32, device=dev)
    met = torch.empty(m, 3, dtype=torch.float64, device=dev)
    sg = torch.empty(m, dtype=torch.int8, device=dev)
    st = torch.empty(m, dtype=torch.int32, device=dev)

    def qstep():
        fif.query(field.c, poses, fif.Q_METRICS, fim, met, sg, st)

    evs = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(args.steps)]
    with ClockSampler(local) as clk:
        clk.mark()
        for _ in range(args.warmup):
            qstep()
        torch.cuda.synchronize()
        dist.barrier()
        torch.cuda.synchronize()
        t_all0 = torch.cuda.Event(enable_timing=True)
        t_all1 = torch.cuda.Event(enable_timing=True)
        t_all0.record(stream)
        for a, b in evs:
            a.record(stream)
            qstep()
            b.record(stream)
        t_all1.record(stream)
        torch.cuda.synchronize()
        clk.mark()
    dist.barrier()
    torch.cuda.synchronize()
    launches += args.steps
    per = [a.elapsed_time(b) for a, b in evs]
    total_ms = t_all0.elapsed_time(t_all1)
    total_ms = dist.max_over_ranks(total_ms, dev)
    ms_step = total_ms / args.steps
    value = m * ws * args.steps / (total_ms * 1e-3)
    kernel_ms = float(np.mean(per))
    achieved = m * QUERY_BYTES_PER_POSE / (kernel_ms * 1e-3) / 1e9
    status = st.cpu().numpy()

    if args.phase == "query":
        if query_storage == fif.STORAGE_BF16:
            achieved = m * BF16_QUERY_BYTES_PER_POSE / (kernel_ms * 1e-3) / 1e9
        if rank == 0:
            print(json.dumps({"metric": METRIC, "value": value, "unit": "queries/s", "n_gpus": ws,
                              "steps": args.steps, "warmup": args.warmup, "ms_per_step": ms_step,
                              "kernel_ms": kernel_ms, "roofline_achieved_gbs": achieved, "storage": args.storage,
                              "config": {"workload": WORKLOAD, "poses_per_step": m}}), flush=True)
        return 0

    # ---------------- end to end through host buffers ----------------
    h_poses = torch.from_numpy(synth.random_poses(2000 + rank, m, spec.lo, spec.hi)).pin_memory()
    h_fim = torch.empty(m, 21, dtype=torch.float32).pin_memory()
    h_met = torch.empty(m, 3, dtype=torch.float64).pin_memory()
    h_sg = torch.empty(m, dtype=torch.int8).pin_memory()
    h_st = torch.empty(m, dtype=torch.int32).pin_memory()

    # fif_query_host on page-locked buffers: the query reads the poses from and writes the outputs
    # to host memory in place over the host link (pageable buffers would go through the staged
    # chunks of E2E_CHUNK poses, copies on a second stream)
    copy_stream = torch.cuda.Stream(device=dev)
    staging = torch.empty(fif.query_host_staging_bytes(E2E_CHUNK), dtype=torch.uint8, device=dev)

    def e2e_step():
        fif.query_host(field.c, h_poses, fif.Q_METRICS, h_fim, h_met, h_sg, h_st, chunk=E2E_CHUNK, staging=staging,
                       stream=stream, copy_stream=copy_stream)

    e2e_steps = max(3, args.steps // 2)
    te = time_events(e2e_step, e2e_steps, 2, stream)
    launches += 0
    e2e_ms = dist.max_over_ranks(float(np.mean(te)), dev)
    e2e = {"value": m * ws / (e2e_ms * 1e-3), "unit": "queries/s", "h2d_bytes_per_step": m * 28,
           "d2h_bytes_per_step": m * (84 + 24 + 1 + 4), "ms_per_step": e2e_ms,
           "api": ("fif_query_host, page-locked host buffers queried in place (poses read and outputs written "
                   "over the host link by the query kernel); the same outputs as the timed step (FIM, trace / "
                   "log|det| / lambda_min, sign, status)")}
    del staging

    # ---------------- point-cloud baseline (all 200k landmarks) ----------------
    # ---------------- the same step at v_alpha = 0.8 (non-negative visibility: PSD FIMs) ----------------
    f08 = field.with_params(fif.make_params(r_max=r_max, v_alpha=0.8))
    t08 = time_events(lambda: fif.query(f08.c, poses, fif.Q_METRICS, fim, met, sg, st), 10, 3, stream)
    ms08 = float(np.mean(t08))
    st08 = st.cpu().numpy()
    out["v_alpha_0.8"] = {"queries_per_s": m / (ms08 * 1e-3), "kernel_ms": ms08,
                          "roofline_frac": m * QUERY_BYTES_PER_POSE / (ms08 * 1e-3) / 1e9 / hbm_peak,
                          "status_counts": {"outside": int(((st08 & 1) != 0).sum()),
                                            "not_pd": int(((st08 & 4) != 0).sum())}}
    del f08

    # one thread per pose, 128-thread CTAs, 4 resident per SM: 152 x 4 CTAs fill the GPU once
    mp = PC_POSES
    tp = time_events(lambda: fif.pointcloud_fim(lm, params, fif.make_pinhole(), poses[:mp], fif.Q_METRICS,
                                                fim, met, sg, st), 3, 1, stream)
    pc_ms = float(np.mean(tp))
    pc_rate = mp / (pc_ms * 1e-3)
    pc_pairs_s = mp * int(lm.shape[0]) / (pc_ms * 1e-3)
    ipp = (PC_INSTRUCTIONS["per_pair"] if PC_INSTRUCTIONS["digest"] ==
           query_source_digest(("pointcloud.cu", "fif_common.cuh")) else None)
    out["pointcloud"] = {"queries_per_s": pc_rate, "landmarks": int(lm.shape[0]), "poses": mp,
                         "launch": f"{mp} poses = {mp // 128} CTAs of 128 threads (4 per SM on 152 SMs)",
                         "kernel_ms": pc_ms, "pose_landmark_pairs_per_s": pc_pairs_s,
                         "instructions_per_pair_ncu": ipp,
                         "issue_rate_fraction": (ipp * pc_pairs_s / (SMS * 4 * 32 * SM_MAX_MHZ * 1e6)
                                                 if ipp else None),
                         "field_speedup": (value / ws) / pc_rate}

    # ---------------- bfloat16 storage (same map, same poses) ----------------
    field16 = fif.Field(spec.origin, spec.res, spec.dims, params, storage=fif.STORAGE_BF16)
    fif.build(field16.c, lm, wsb)
    t16 = time_events(lambda: fif.query(field16.c, poses, fif.Q_METRICS, fim, met, sg, st), 10, 3, stream)
    ms16 = float(np.mean(t16))
    b16 = BF16_QUERY_BYTES_PER_POSE
    out["bf16"] = {"queries_per_s": m / (ms16 * 1e-3), "kernel_ms": ms16, "bytes_per_pose": b16,
                   "io_bytes_per_pose": QUERY_IO_BYTES_PER_POSE,
                   "roofline": {"bound": "hbm", "achieved": m * b16 / (ms16 * 1e-3) / 1e9, "peak": hbm_peak,
                                "unit": "GB/s", "frac": m * b16 / (ms16 * 1e-3) / 1e9 / hbm_peak}}
    torch.cuda.empty_cache()

    # ---------------- positional trace factor (10 floats per node, world-frame trace) ----------------
    out["trace_field"] = trace_block(fif, spec, lm, params, poses, met, st, wsb, stream, hbm_peak)

    # ---------------- GP visibility field (N_s = 70, the paper's choice) ----------------
    out["gp"] = gp_block(fif, synth, spec, lm, r_max, m, args.gp_samples, dev, stream, hbm_peak)

    # ---------------- information threshold and potential cost (Sec. VI-B) ----------------
    # 10,000 sets of 200 landmarks at 0.3-1.0 m in the field of view (the paper's specification)
    sets = torch.from_numpy(synth.threshold_sets(21, 10_000, 200, 0.3, 1.0)).to(dev)
    thr_out = {}
    gpc = fif.gp_struct(synth.fibonacci_sphere(args.gp_samples), out["gp"]["length_scale"])
    for name, model in (("pointcloud", fif.MODEL_POINTCLOUD), ("quad", fif.MODEL_QUAD), ("gp", fif.MODEL_GP)):
        tmet = torch.empty(10_000, 3, dtype=torch.float64, device=dev)
        tthr = torch.empty(3, dtype=torch.float64, device=dev)
        tt = time_events(lambda: fif.info_threshold(params, sets, model, gpc if model == fif.MODEL_GP else None,
                                                    metrics=tmet, threshold=tthr), 5, 2, stream)
        thr_out[name] = {"ms": float(np.mean(tt)), "thresholds": [float(x) for x in tthr.cpu()]}
    cst = torch.empty(m, dtype=torch.float64, device=dev)
    dcst = torch.empty(m, dtype=torch.float64, device=dev)
    eps_ld = thr_out["quad"]["thresholds"][1]
    tc = time_events(lambda: fif.info_cost(met, eps_ld, 0.05, column=1, cost=cst, dcost=dcst), 10, 3, stream)
    tc_ms = float(np.mean(tc))
    out["info"] = {"sets": 10_000, "landmarks_per_set": 200, "threshold": thr_out,
                   "cost_ms": tc_ms, "cost_values_per_s": m / (tc_ms * 1e-3),
                   "cost_roofline": {"bound": "hbm", "achieved": m * 24 / (tc_ms * 1e-3) / 1e9, "peak": hbm_peak,
                                     "unit": "GB/s", "frac": m * 24 / (tc_ms * 1e-3) / 1e9 / hbm_peak}}
    del sets

    # ---------------- differentiable trajectory batch (256 x 128 samples) ----------------
    from paper_2008_03324_gb300 import traj
    ctrl_np, yaw_np, basis_np = synth.bspline_batch(6, scene, 256, 32, 128)
    field08 = field.with_params(fif.make_params(r_max=r_max, v_alpha=0.8))
    B_t = torch.from_numpy(basis_np.astype(np.float32)).to(dev)
    yaw_t = torch.from_numpy(yaw_np.astype(np.float32)).to(dev)
    ctrl_t = torch.from_numpy(ctrl_np.astype(np.float32)).to(dev).requires_grad_(True)

    def traj_step():
        ctrl_t.grad = None
        loss, phi, tm, tsg = traj.neg_logdet_objective(ctrl_t, yaw_t, B_t, field08)
        loss.backward()

    ttj = time_events(traj_step, 10, 3, stream)
    # the same step captured once in a CUDA graph and replayed (traj.GraphedObjective)
    gobj = traj.GraphedObjective(ctrl_t, yaw_t, B_t, field08)
    ttg = time_events(lambda: gobj.step(), 10, 3, stream)
    out["trajopt"] = {"trajectories": 256, "samples": 128, "poses": 256 * 128, "v_alpha": 0.8,
                      "ms_forward_backward": float(np.mean(ttj)),
                      "poses_per_s": 256 * 128 / (float(np.mean(ttj)) * 1e-3),
                      "ms_forward_backward_graphed": float(np.mean(ttg)),
                      "poses_per_s_graphed": 256 * 128 / (float(np.mean(ttg)) * 1e-3)}
    del gobj

    # ---------------- large map: 2M landmarks, 400 x 400 x 80 nodes (12.8M), r_max 12 m ----------------
    if not args.no_large:
        del field08
        bscene = synth.building(seed=5, n=2_000_000)
        bspec = synth.BUILDING_GRID
        blm = torch.from_numpy(bscene.landmarks).to(dev)
        large = {"landmarks": int(blm.shape[0]), "field_nodes": bspec.n_nodes, "r_max": 12.0}
        for storage, name in ((fif.STORAGE_F32, "f32"), (fif.STORAGE_BF16, "bf16")):
            bf = fif.Field(bspec.origin, bspec.res, bspec.dims, fif.make_params(r_max=12.0, v_alpha=0.5),
                           storage=storage)
            bws = torch.empty(fif.build_workspace_bytes(bf.c, blm.shape[0]), dtype=torch.uint8, device=dev)
            tbl = time_events(lambda: fif.build(bf.c, blm, bws), 1, 0, stream)
            ins, cnd, _ = fif.build_stats(bws, bf, blm.shape[0])
            bposes = torch.from_numpy(synth.random_poses(77, m, bspec.lo, bspec.hi)).to(dev)
            tql = time_events(lambda: fif.query(bf.c, bposes, fif.Q_METRICS, fim, met, sg, st), 5, 2, stream)
            large[name] = {"build_ms": float(tbl[0]), "in_shell_pairs": ins, "build_pairs_per_s": ins / (tbl[0] * 1e-3),
                           "field_bytes": bf.coeffs.numel() * bf.coeffs.element_size(),
                           "queries_per_s": m / (float(np.mean(tql)) * 1e-3)}
            if rank == 0 and args.serve_requests > 0:
                breqs = synth.request_stream(13, min(600, args.serve_requests), bscene, zr=(0.5, 19.5))
                large[name]["serving"] = serving_run(fif, serve, bf, breqs, 20_000.0, 14)
            del bf, bws, bposes
            torch.cuda.empty_cache()
        out["large"] = large
        assert fif.device_error() == 0

    # ---------------- serving (rank 0) ----------------
    if rank == 0 and args.serve_requests > 0:
        # Poisson request streams at 2k-50k requests/s (8-4096 poses each) on the fp32 and bf16
        # fields; the 20k fp32 run is the headline p99
        out.update(serving_sweep(fif, serve, synth, scene, field, field16, args.serve_requests))
    del field16
    if rank == 0:
        out["method_accuracy"] = method_accuracy(fif, synth, dev)

    # ---------------- CPU oracle baseline (rank 0, N = 1) ----------------
    cpu = None
    if rank == 0 and ws == 1 and not args.no_cpu_baseline:
        cpu = cpu_baseline(scene, spec, r_max)

    if rank == 0:
        clocks = clk.summary()
        line = {
            "metric": METRIC, "value": value, "unit": "queries/s", "n_gpus": ws, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": ms_step, "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "f32", "data": "synthetic",
            "config": {"workload": WORKLOAD, "poses_per_step": m, "field_nodes": field.n_nodes,
                       "landmarks": int(lm.shape[0]),
                       "l2": "inputs larger than L2: 1.38 GB field gathered at uniform-random positions",
                       "parallelism": f"replicas x{ws}"},
            "roofline": {"bound": "hbm", "achieved": achieved, "peak": hbm_peak, "unit": "GB/s",
                         "frac": achieved / hbm_peak,
                         "traffic": (QUERY_TRAFFIC["bytes_per_pose"] * m
                                     if QUERY_TRAFFIC["digest"] == query_source_digest() else None),
                         "traffic_note": "ncu dram read+write bytes per launch of query_kernel (summary in profiles/)",
                         "peak_kind": f"{peak_kind} (MEASURED_PEAKS hbm_gbs)",
                         "bytes_per_pose": QUERY_BYTES_PER_POSE, "io_bytes_per_pose": QUERY_IO_BYTES_PER_POSE,
                         "kernel_ms": kernel_ms},
            "cpu_baseline": cpu,
            "e2e": e2e,
            "gpu_launches": launches,
            "clocks": clocks,
            "p99_latency_ms": out.get("serving", {}).get("p99_ms"),
            "status_counts": {"outside": int(((status & 1) != 0).sum()), "not_pd": int(((status & 4) != 0).sum())},
            **out,
        }
        print(json.dumps(line), flush=True)
    dist.barrier()
    return 0


if __name__ == "__main__":
    sys.exit(main())
