#!/usr/bin/env python3
"""Benchmark of the procedural ray tracer: Mrays/s and frame latency, batched vs plain.

Headline workload: a batch of 64 render requests (each its own instanced
procedural scene of 1..10 000 instances of the 8 primitive types, resolution
256^2..2048^2, orbit camera). One step = one pass of the whole hot path over
the batch: the device LBVH build of every request's scene (BLASes, instance
boxes, TLAS) and one batched launch (CUDA graph, autotuned launch shape) that
renders every request (primary and shadow rays through two-level traversal,
Eq. 1 dispatch, intersection and closest-hit shaders). Beside it, the plain
form: the same builds and one pr_trace launch per request.

Extra blocks: the teaser scene at 1920x1080 (build + frame), the tiny
analytic scene as 4096 frames per launch, the 100 000-instance field at
3840x2160 (build + frame), and the serving loop under Poisson arrivals.

  python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]

N > 1 runs N independent replicas (one per GPU, launched by torchrun); the
path needs no collective. Prints one JSON line on rank 0.
"""
from __future__ import annotations

import argparse
import json
import os
import statistics
import subprocess
import sys
import threading
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

import scenes  # noqa: E402

L2_FLUSH_BYTES = 256 << 20   # > 126 MB L2
BATCH = "batch64"
SINGLE = ("analytic_64x64", "teaser_1080p", "field_100k_2160p")
# default timed steps per workload: about 0.5-1.5 s of GPU work on a B300
DEFAULT_STEPS = {BATCH: 20, "analytic_64x64": 2000, "teaser_1080p": 2000, "field_100k_2160p": 150}
SERVE_RATES = [10.0, 30.0, 100.0, 300.0, 1000.0, 2000.0]
# continuous batching: while at most this many requests wait for rows, the oldest runs alone
# through pr_trace (batching pays when requests queue)
SERVE_SOLO_MAX_WAITING = 2
BATCH_DESC = ("batch of 64 render requests: instanced procedural fields of 1..10000 instances "
              "(8 primitive types, log-uniform count), resolutions from {256^2, 512^2, 1024^2, 2048^2}, orbit cameras")


TLAS_FORMATS = {"greedy4": lambda pr: 0, "parity4": lambda pr: pr.PR_BUILD_TLAS_PARITY4,
                "bvh8": lambda pr: pr.PR_BUILD_TLAS_BVH8, "bvh8_f32": lambda pr: pr.PR_BUILD_TLAS_BVH8_F32}


def workload_by_name(name: str):
    if name == "analytic_64x64":
        return scenes.small_analytic()
    if name == "teaser_1080p":
        return scenes.teaser()
    if name == "field_100k_2160p":
        return scenes.field()
    raise SystemExit(f"unknown workload {name}")


def workload_config(name: str, w) -> dict:
    return {"workload": {"analytic_64x64": "tiny analytic scene, 4 AABB primitives, one BLAS",
                         "teaser_1080p": "teaser scene: 2 pac-men + quaternion Julia + Mandelbulb + mirror slab",
                         "field_100k_2160p": "instanced field, 100000 instances of 8 procedural types"}[name],
            "config": name, "width": w.params.width, "height": w.params.height,
            "instances": int(len(w.scene.inst_blas)), "max_depth": w.params.max_depth,
            "rays_per_pixel_max": 1 + 1 + (1 if w.params.max_depth >= 2 else 0),
            "step": "device LBVH build + one frame", "output": "rgb float32 image, 12 B/pixel",
            "l2": "flushed between timed steps (256 MB write)", "parallelism": "replicas"}


class ClockSampler:
    """nvidia-smi clocks / throttle reasons sampled during the timed region.

    Samples carry nvidia-smi's own timestamps; only those between begin() and
    end() (host wall clock) are summarised, so idle time around the region does
    not enter the median."""

    FIELDS = ("timestamp,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")
    BAD = ("hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown")

    def __init__(self, gpu_index: int):
        self.gpu = gpu_index
        self.proc = None
        self.lines = []
        self.t0 = self.t1 = None

    def start(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", str(self.gpu), f"--query-gpu={self.FIELDS}", "--format=csv,noheader,nounits",
                 "-lms", "50"], stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.thread = threading.Thread(target=self._read, daemon=True)
            self.thread.start()
            deadline = time.time() + 3.0
            while not self.lines and time.time() < deadline:   # sampling has begun
                time.sleep(0.01)
        except (OSError, FileNotFoundError):
            self.proc = None

    def begin(self):
        self.t0 = time.time()

    def end(self):
        self.t1 = time.time()

    def _read(self):
        for line in self.proc.stdout:
            self.lines.append(line.strip())

    def stop(self) -> dict:
        if not self.proc:
            return None
        time.sleep(0.12)                      # the sample that covers the region's end
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except subprocess.TimeoutExpired:
            self.proc.kill()
        import datetime
        rows = []
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for ln in self.lines:
            parts = [p.strip() for p in ln.split(",")]
            if len(parts) < 9:
                continue
            try:
                ts = datetime.datetime.strptime(parts[0], "%Y/%m/%d %H:%M:%S.%f").timestamp()
                sm, smax = float(parts[1]), float(parts[2])
            except ValueError:
                continue
            rows.append((ts, sm, smax, {nm for nm, v in zip(names, parts[5:9]) if v.lower() == "active"}))
        if not rows:
            return None
        inside = [r for r in rows if self.t0 is not None and self.t0 - 0.06 <= r[0] <= self.t1 + 0.06]
        use = inside or [min(rows, key=lambda r: abs(r[0] - (self.t0 or r[0])))]
        reasons = set().union(*[r[3] for r in use])
        return {"sm_mhz": float(statistics.median([r[1] for r in use])), "sm_max_mhz": float(max(r[2] for r in use)),
                "samples": len(use), "samples_in_region": len(inside), "reasons": sorted(reasons)}

    @classmethod
    def rejected(cls, c) -> bool:
        """A run to measure again: a slowdown reason, or SM clocks well below
        their maximum with no reason given (a leftover clock lock)."""
        if not c:
            return False
        if set(c["reasons"]) & set(cls.BAD):
            return True
        return c["sm_mhz"] < 0.8 * c["sm_max_mhz"] and not c["reasons"]


def aggregate_over_ranks(total_ms: float, rays: int, world: int, device) -> tuple:
    """Replicas: the job's time is the slowest rank's, its work the sum over ranks."""
    if world <= 1:
        return total_ms, rays
    import torch
    import torch.distributed as dist
    t = torch.tensor([total_ms], dtype=torch.float64, device=device)
    r = torch.tensor([rays], dtype=torch.int64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    dist.all_reduce(r, op=dist.ReduceOp.SUM)
    return float(t.item()), int(r.item())


# DRAM traffic of one timed trace launch (dram__bytes_read.sum + dram__bytes_write.sum from
# one ncu capture, L2 flushed before the launch as in the timed loop), per workload and traversal
# mode. A figure holds only for the kernel sources it was taken on: it is keyed by the SHA-1 of
# its kernel's sources (the single-request kernel's, or those plus the batched kernels') and
# reported as null once they change.
TRACE_SOURCES = ["paper_2012_10357_b300/csrc/trace.cu", "paper_2012_10357_b300/csrc/tracer.cuh",
                 "paper_2012_10357_b300/csrc/shaders.cuh", "paper_2012_10357_b300/csrc/pr_device.cuh",
                 "include/proceduray.h"]
BATCH_SOURCES = TRACE_SOURCES + ["paper_2012_10357_b300/csrc/wavefront.cu", "paper_2012_10357_b300/csrc/wavefront.h"]
TRACE_TRAFFIC = {   # {sha1 of the kernel's sources: {workload: bytes per launch}}
    # ncu captures of dram__bytes_read.sum + dram__bytes_write.sum (profiles/), taken on the sources
    # keyed 2b0b46fc... / 4cb63c66...; carried to these keys because the one change since is a
    # comment in the header (trace.cu and wavefront.cu compile to identical cubins)
    "85af754dc87822a3d87e7a60e915ab3a56176c38": {"teaser_1080p": 97_024 + 2_048,
                                                 "field_100k_2160p": 5_900_544 + 46_041_600,
                                                 "analytic_64x64_x4096": 494_080 + 162_999_552},
    # batch64: the 8-request batch's 142.63 MB scaled by pixels to the 64-request batch
    # (83 623 936 / 15 859 712)
    "abf4bde15585571a06aa3a20d81ea90dfd6b1a8e": {"batch64": 752_037_702},
}


def sources_sha1(sources) -> str:
    import hashlib
    h = hashlib.sha1()
    for rel in sources:
        with open(os.path.join(ROOT, rel), "rb") as f:
            h.update(f.read())
    return h.hexdigest()


def trace_traffic(workload: str, binary_tlas: bool = False):
    if binary_tlas:
        return None
    key = sources_sha1(BATCH_SOURCES if workload == "batch64" else TRACE_SOURCES)
    return TRACE_TRAFFIC.get(key, {}).get(workload)


def measured_peaks() -> dict:
    p = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(p):
        with open(p) as f:
            return json.load(f)
    return {}


def _events(torch, n):
    return [torch.cuda.Event(enable_timing=True) for _ in range(n)]


def roofline(work, torch, counters_list, kernel_s: float, kernel: str, traffic_key: str, clocks=None,
             probe_tflops=None, binary_tlas: bool = False) -> dict:
    """FP32 roofline of a trace kernel: FMA-pipe FLOPs of the launch (work counters x
    per-unit counts) over its mean CUDA-event duration, against SMs x 128 x 2 x clock;
    ALU-pipe and special-function operation rates beside it."""
    props = torch.cuda.get_device_properties(torch.cuda.current_device())
    n_sm = props.multi_processor_count
    peaks = measured_peaks()
    sm_max = float(peaks.get("sm_max_mhz", 2032.0))
    fma = sum(work.frame_fma_flops(c) for c in counters_list)
    alu = sum(work.frame_alu_ops(c) for c in counters_list)
    spec = sum(work.frame_special_ops(c) for c in counters_list)
    peak = work.fp32_peak_tflops(n_sm, sm_max)
    achieved = fma / kernel_s / 1e12
    roof = {"bound": "alu", "achieved": achieved, "peak": peak, "unit": "TFLOP/s", "frac": achieved / peak,
            "traffic": trace_traffic(traffic_key, binary_tlas), "kernel": kernel,
            "flops_per_launch": fma, "launch_ms": kernel_s * 1e3,
            "flop_count": "FMA-pipe FLOPs (FFMA 2, FADD/FMUL 1) from the work counters; min/max/compares "
                          "(ALU pipe) and rcp/sqrt/log (special) are reported beside, not in the FLOPs",
            "alu_ops_per_launch": alu, "alu_gops_per_s": alu / kernel_s / 1e9,
            "special_ops_per_launch": spec, "special_gops_per_s": spec / kernel_s / 1e9,
            "peak_basis": f"{n_sm} SMs x 128 FP32 lanes x 2 x {sm_max:.0f} MHz (sm_max_mhz of measured)"}
    if clocks:
        roof["peak_at_sampled_clock"] = work.fp32_peak_tflops(n_sm, clocks["sm_mhz"])
        roof["frac_at_sampled_clock"] = achieved / roof["peak_at_sampled_clock"]
    sustained = (peaks.get("clocks_under_load") or {}).get("sm_mhz_median")
    if sustained:
        # the SM clock the driver saw under a seconds-long dense GEMM at the power cap
        roof["peak_at_measured_sustained_clock"] = work.fp32_peak_tflops(n_sm, float(sustained))
        roof["frac_at_measured_sustained_clock"] = achieved / roof["peak_at_measured_sustained_clock"]
    if roof["traffic"]:
        roof["traffic_gbs"] = roof["traffic"] / kernel_s / 1e9
        if peaks.get("hbm_gbs"):
            roof["traffic_frac_of_hbm"] = roof["traffic_gbs"] / float(peaks["hbm_gbs"])
    if probe_tflops:
        roof["peak_fma_probe"] = probe_tflops
        roof["frac_of_fma_probe"] = achieved / probe_tflops
    return roof


def timed(torch, stream, flush, steps, body, sampler=None):
    """K timed steps on `stream`, L2 flushed before each (outside the events).
    body(k) enqueues one step and returns its list of events to record between
    phases; returns [(ev_start, [ev_phase...])]."""
    out = []
    if sampler:
        sampler.begin()
    with torch.cuda.stream(stream):
        for k in range(steps):
            flush.fill_(float(k))
            e0 = torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            out.append((e0, body(k)))
    stream.synchronize()
    torch.cuda.synchronize()
    if sampler:
        sampler.end()
    return out


def bench_scene(pr, work, torch, stream, flush, name: str, steps: int, warmup: int, probe=None,
                binary_tlas: bool = False, sampler=None, build_flags: int = 0) -> dict:
    """One scene, one frame per step: device BVH build (LBVH; the TLAS by PLOC with
    PR_BUILD_TLAS_PLOC) + pr_trace."""
    w = workload_by_name(name)
    H, W = w.params.height, w.params.width
    with torch.cuda.stream(stream):
        scene = pr.Scene(w.scene, stream=stream, build_flags=build_flags)
        out = torch.empty((H, W, 3), dtype=torch.float32, device="cuda")
        counter = torch.zeros(1, dtype=torch.int64, device="cuda")

    def step(k):
        e1, e2 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        scene.build_bvh(stream, build_flags)
        e1.record(stream)
        scene.trace(w.camera, w.params, out=out, ray_counter=counter, stream=stream, binary_tlas=binary_tlas)
        e2.record(stream)
        return [e1, e2]

    with torch.cuda.stream(stream):
        for k in range(warmup):
            step(k)
    stream.synchronize()
    counter.zero_()
    torch.cuda.synchronize()
    if sampler:
        sampler.start()
    ev = timed(torch, stream, flush, steps, step, sampler)
    clocks = sampler.stop() if sampler else None
    step_ms = [e0.elapsed_time(p[1]) for e0, p in ev]
    build_ms = [e0.elapsed_time(p[0]) for e0, p in ev]
    trace_ms = [p[0].elapsed_time(p[1]) for e0, p in ev]
    rays = int(counter.item())
    n_build, n_trace = scene.kernel_launches()
    counters = scene.trace_work(w.camera, w.params, stream=stream, binary_tlas=binary_tlas)
    torch.cuda.synchronize()
    config = workload_config(name, w)
    ploc = bool(build_flags & pr.PR_BUILD_TLAS_PLOC) and len(w.scene.inst_blas) > 1024
    config["tlas_builder"] = "ploc" if ploc else "lbvh"
    config["tlas_format"] = next((k for k, f in TLAS_FORMATS.items() if f(pr) and build_flags & f(pr)), "greedy4")
    if ploc:
        config["step"] = "device build (BLAS: LBVH, TLAS: PLOC) + one frame"
    n_rays = max(1, counters.get("rays", 0))
    block = {"workload": config["workload"], "config": config,
             "value": rays / (sum(step_ms) / 1e3) / 1e6, "unit": "Mrays/s", "steps": steps,
             "ms_per_step": sum(step_ms) / steps, "rays_per_step": rays / steps,
             "latency_ms": {"p50": float(np.percentile(step_ms, 50)), "p99": float(np.percentile(step_ms, 99)),
                            "build_p50": float(np.percentile(build_ms, 50)),
                            "trace_p50": float(np.percentile(trace_ms, 50))},
             "gpu_launches_per_step": n_build + n_trace,
             "roofline": roofline(work, torch, [counters], statistics.mean(trace_ms) / 1e3, "k_trace (megakernel)",
                                  name, clocks, probe, binary_tlas),
             "device_error_word": scene.error_word(stream),
             "traversal_per_ray": {k: counters.get(k, 0) / n_rays
                                   for k in ("tlas_nodes8q", "tlas_nodes8", "tlas_nodes4", "tlas_nodes", "instances",
                                             "blas_nodes", "leaves")}}
    block["roofline"]["trace_share_of_step"] = sum(trace_ms) / sum(step_ms)
    block["roofline"]["work_counters"] = {k: v for k, v in counters.items() if v}
    if clocks:
        block["clocks"] = clocks
    block["_scene"], block["_w"], block["_out"] = scene, w, out
    return block


def bench_tlas_variants(pr, work, torch, stream, flush, steps: int, warmup: int, probe=None) -> dict:
    """The 100 000-instance field with every TLAS builder (LBVH, PLOC) x wide format (greedy
    4-wide, depth-parity 4-wide, 8-wide quantised, 8-wide float): build and trace time, node
    and instance visits per ray, and whether the image equals the default build's."""
    rows, ref = [], None
    for builder in ("lbvh", "ploc"):
        for fmt, flag in TLAS_FORMATS.items():
            flags = (pr.PR_BUILD_TLAS_PLOC if builder == "ploc" else 0) | flag(pr)
            b = bench_scene(pr, work, torch, stream, flush, "field_100k_2160p", steps, warmup, probe,
                            build_flags=flags)
            if ref is None:
                ref = b["_out"].clone()
            t = b["traversal_per_ray"]
            rows.append({"builder": builder, "format": fmt, "mrays": b["value"],
                         "trace_ms": b["latency_ms"]["trace_p50"], "build_ms": b["latency_ms"]["build_p50"],
                         "step_ms": b["latency_ms"]["p50"],
                         "wide_nodes_per_ray": t["tlas_nodes4"] + t["tlas_nodes8"] + t["tlas_nodes8q"],
                         "instances_per_ray": t["instances"], "image_equals_default": bool(torch.equal(b["_out"], ref)),
                         "device_error_word": b["device_error_word"], "fma_frac": b["roofline"]["frac"],
                         "alu_gops_per_s": b["roofline"]["alu_gops_per_s"]})
            b["_scene"].close()
    return {"workload": "instanced field, 100000 instances, 3840x2160, TLAS builder x wide format",
            "steps": steps, "rows": rows}


def scene_e2e(pr, torch, stream, block, n_steps: int, warmup: int, world: int) -> dict:
    """End to end through the public API: host description -> device (pinned staging, one
    copy), build, frame, image -> pinned host memory, every step; the readback of frame k
    overlaps frame k+1 (second stream, double-buffered image)."""
    scene, w, out = block["_scene"], block["_w"], block["_out"]
    e2e_counter = torch.zeros(1, dtype=torch.int64, device="cuda")
    outs = [out, torch.empty_like(out)]
    hosts = [torch.empty(tuple(out.shape), dtype=torch.float32, pin_memory=True) for _ in range(2)]
    copy_stream = torch.cuda.Stream()
    traced = [torch.cuda.Event(), torch.cuda.Event()]
    copied = [torch.cuda.Event(), torch.cuda.Event()]

    def frame(k):
        i = k % 2
        if k >= 2:
            copied[i].synchronize()
        scene.upload(w.scene, stream)
        scene.build_bvh(stream)
        scene.trace(w.camera, w.params, out=outs[i], ray_counter=e2e_counter, stream=stream)
        traced[i].record(stream)
        copy_stream.wait_event(traced[i])
        with torch.cuda.stream(copy_stream):
            hosts[i].copy_(outs[i], non_blocking=True)
        copied[i].record(copy_stream)

    serial = []
    for k in range(warmup + n_steps):
        torch.cuda.synchronize()
        if k == warmup:
            e2e_counter.zero_()
            torch.cuda.synchronize()
        t0 = time.perf_counter()
        frame(k)
        copied[k % 2].synchronize()
        if k >= warmup:
            serial.append(time.perf_counter() - t0)
    serial_rays = int(e2e_counter.item())
    for k in range(warmup):
        frame(k)
    torch.cuda.synchronize()
    e2e_counter.zero_()
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    for k in range(n_steps):
        frame(k)
    torch.cuda.synchronize()
    pipe_ms, rays = aggregate_over_ranks((time.perf_counter() - t0) * 1e3, int(e2e_counter.item()), world, "cuda")
    serial_ms, serial_rays = aggregate_over_ranks(sum(serial) * 1e3, serial_rays, world, "cuda")
    return {"value": rays / (pipe_ms / 1e3) / 1e6, "unit": "Mrays/s",
            "h2d_bytes_per_step": int(scene.desc_bytes), "d2h_bytes_per_step": int(out.numel() * 4),
            "ms_per_step": pipe_ms / n_steps,
            "mode": f"{n_steps} consecutive frames, each: description to the device, BVH build, frame, image to "
                    "pinned host memory; the image copy of frame k overlaps frame k+1",
            "serial": {"value": serial_rays / (serial_ms / 1e3) / 1e6, "unit": "Mrays/s",
                       "ms_per_step": serial_ms / n_steps, "mode": "one frame at a time, synchronised after each"}}


def bench_analytic_frames(pr, work, torch, stream, flush, frames=4096, reps=5, probe=None) -> dict:
    """The tiny analytic scene as a throughput run: 4096 eye-jittered 64x64 frames in one launch."""
    w = scenes.small_analytic()
    cams = pr.CameraArray(scenes.small_analytic_cameras(0, frames))   # marshalled once
    with torch.cuda.stream(stream):
        scene = pr.Scene(w.scene, stream=stream)
        out = torch.empty((frames, 64, 64, 3), dtype=torch.float32, device="cuda")
        counter = torch.zeros(1, dtype=torch.int64, device="cuda")
    for _ in range(3):
        scene.trace_frames(cams, w.params, out=out, stream=stream)
    stream.synchronize()
    ev = _events(torch, 2 * reps)
    with torch.cuda.stream(stream):
        for k in range(reps):
            flush.fill_(float(k))
            ev[2 * k].record(stream)
            scene.trace_frames(cams, w.params, out=out, ray_counter=counter, stream=stream)
            ev[2 * k + 1].record(stream)
    stream.synchronize()
    ms = [ev[2 * k].elapsed_time(ev[2 * k + 1]) for k in range(reps)]
    rays = int(counter.item()) / reps
    counters = scene.trace_work(None, w.params, cameras=cams, stream=stream)
    avg_s = statistics.mean(ms) / 1e3
    _, n_trace = scene.kernel_launches()
    scene.close()
    roof = roofline(work, torch, [counters], avg_s, "k_trace (megakernel)", "analytic_64x64_x4096", None, probe)
    roof["work_counters"] = {k: v for k, v in counters.items() if v}
    return {"workload": "tiny analytic scene: 4096 eye-jittered 64x64 frames, one pr_trace_frames launch",
            "value": rays / avg_s / 1e6, "unit": "Mrays/s", "ms_per_launch": statistics.mean(ms),
            "rays_per_launch": rays, "gpu_launches_per_step": n_trace, "roofline": roof}


class BatchBench:
    """The 64-request batch: scenes, outputs, the batch object and its tuning."""

    def __init__(self, pr, torch, stream, n_requests=64, tuning=None, ws=None):
        self.pr, self.torch, self.stream = pr, torch, stream
        self.ws = ws if ws is not None else scenes.batch_requests(0, n_requests)
        n_requests = len(self.ws)
        self.n = n_requests
        self.total_px = sum(w.params.width * w.params.height for w in self.ws)
        with torch.cuda.stream(stream):
            self.objs = [pr.Scene(w.scene, stream=stream) for w in self.ws]
            self.out_b = [torch.empty((w.params.height, w.params.width, 3), device="cuda") for w in self.ws]
            self.out_p = [torch.empty((w.params.height, w.params.width, 3), device="cuda") for w in self.ws]
            self.counter = torch.zeros(1, dtype=torch.int64, device="cuda")
        self.batch = pr.Batch(n_requests, self.total_px)
        items = [(o, w.camera, w.params, out) for o, w, out in zip(self.objs, self.ws, self.out_b)]
        tune_path = os.path.join(ROOT, "paper_2012_10357_b300", "tuning_cache.json")
        key = f"{torch.cuda.get_device_name()}|batch|{n_requests}|{self.total_px}"
        cache = json.load(open(tune_path)) if os.path.exists(tune_path) else {}
        if tuning is not None:
            self.batch.set_tuning(**tuning)
            self.tuned = {"tuning": tuning, "ms": None, "from_cache": False, "given": True}
        elif key in cache:
            self.batch.set_tuning(**cache[key]["tuning"])
            self.tuned = dict(cache[key], from_cache=True)
        else:
            best, best_ms = self.batch.autotune(items, stream=stream)
            self.tuned = {"tuning": best, "ms": best_ms, "from_cache": False}
            cache[key] = {"tuning": best, "ms": best_ms}
            with open(tune_path, "w") as f:
                json.dump(cache, f, indent=1)
        self.prepared = self.batch.prepare(items)
        # kernels of the batched launch per tuning mode: four stages, or one megakernel
        self.trace_launches = {0: 4, 1: 1, 2: 2, 3: 8, 4: 2}[self.tuned["tuning"]["megakernel"]]

    def build_all(self):
        # the 64 scenes' builds run concurrently (pr_build_bvh_many: internal streams
        # forked from and joined back into the bench stream)
        self.pr.build_bvh_many(self.objs, self.stream)

    def batched_step(self, k):
        e1, e2 = self.torch.cuda.Event(enable_timing=True), self.torch.cuda.Event(enable_timing=True)
        self.build_all()
        e1.record(self.stream)
        self.batch.trace(prepared=self.prepared, ray_counter=self.counter, stream=self.stream, graph=True)
        e2.record(self.stream)
        return [e1, e2]

    def plain_step(self, k):
        ev = _events(self.torch, 1 + self.n)
        self.build_all()
        ev[0].record(self.stream)
        for q, (o, w, out) in enumerate(zip(self.objs, self.ws, self.out_p)):
            o.trace(w.camera, w.params, out=out, ray_counter=self.counter, stream=self.stream)
            ev[1 + q].record(self.stream)
        return ev

    def build_launches(self) -> int:
        return sum(o.kernel_launches()[0] for o in self.objs)

    def close(self):
        self.batch.close()
        for o in self.objs:
            o.close()


def bench_batch(pr, work, torch, stream, flush, steps: int, warmup: int, world: int, probe=None, sampler=None,
                n_requests: int = 64, tuning=None, ws=None):
    """Headline: step = the LBVH builds of the 64 requests' scenes + one batched launch (CUDA
    graph). The plain form (same builds, one pr_trace per request) is timed beside it."""
    B = BatchBench(pr, torch, stream, n_requests, tuning, ws)
    with torch.cuda.stream(stream):
        for k in range(warmup):
            B.batched_step(k)
            B.plain_step(k)
    stream.synchronize()
    B.counter.zero_()
    torch.cuda.synchronize()
    if sampler:
        sampler.start()
    if world > 1:
        import torch.distributed as dist
        dist.barrier()
    torch.cuda.synchronize()
    ev = timed(torch, stream, flush, steps, B.batched_step, sampler)
    if world > 1:
        dist.barrier()
    clocks = sampler.stop() if sampler else None
    rays = int(B.counter.item())
    step_ms = [e0.elapsed_time(p[1]) for e0, p in ev]
    build_ms = [e0.elapsed_time(p[0]) for e0, p in ev]
    trace_ms = [p[0].elapsed_time(p[1]) for e0, p in ev]
    total_ms, rays_all = aggregate_over_ranks(sum(step_ms), rays, world, "cuda")
    # plain form, same steps
    B.counter.zero_()
    torch.cuda.synchronize()
    evp = timed(torch, stream, flush, steps, B.plain_step)
    plain_rays = int(B.counter.item())
    p_step = [e0.elapsed_time(p[-1]) for e0, p in evp]
    p_trace = [p[0].elapsed_time(p[-1]) for e0, p in evp]
    p_lat = [e0.elapsed_time(e) for e0, p in evp for e in p[1:]]        # each request's completion
    identical = all(torch.equal(a, b) for a, b in zip(B.out_b, B.out_p))
    counters = [o.trace_work(w.camera, w.params, stream=stream) for o, w in zip(B.objs, B.ws)]
    torch.cuda.synchronize()
    kernel = {0: "k_wf_primary/shadow/mirror/resolve (wavefront stages)", 1: "k_batch_mega (persistent)",
              2: "k_batch_mega_tiles (one CTA per tile)",
              3: "k_rg_* (regrouped stages with march jobs)",
              4: "k_batch_mega_tiles (one one-warp CTA per quarter tile)"}[B.tuned["tuning"]["megakernel"]]
    roof = roofline(work, torch, counters, statistics.mean(trace_ms) / 1e3, kernel, BATCH, clocks, probe)
    roof["trace_share_of_step"] = sum(trace_ms) / sum(step_ms)
    res = {"value": rays_all / (total_ms / 1e3) / 1e6, "total_ms": total_ms, "rays": rays,
           "step_ms": step_ms, "build_ms": build_ms, "trace_ms": trace_ms, "clocks": clocks, "roofline": roof,
           "gpu_launches_per_step": B.build_launches() + B.trace_launches,
           "plain": {"value": plain_rays / (sum(p_step) / 1e3) / 1e6, "unit": "Mrays/s",
                     "ms_per_step": sum(p_step) / steps, "trace_ms_per_step": sum(p_trace) / steps,
                     "latency_ms": {"p50": float(np.percentile(p_lat, 50)), "p99": float(np.percentile(p_lat, 99))},
                     "gpu_launches_per_step": B.build_launches() + B.n,
                     "form": "the same 64 builds, then one pr_trace launch per request (64 launches)"},
           "images_identical_to_plain": identical, "autotune": B.tuned,
           "batch_device_bytes": B.batch.device_bytes(), "B": B}
    return res


def batch_e2e(pr, torch, stream, B, n_steps: int, warmup: int, world: int) -> dict:
    """End to end through the public API with host buffers: every step uploads the 64 scene
    descriptions from host memory (pinned staging, one copy per scene), builds the 64 BVHs,
    renders the batch in one graph launch and copies the 64 images to pinned host memory.
    Pipelined over double-buffered images: the readback of batch k-1 is issued after batch k's
    uploads and builds and overlaps batch k's trace (a 1 GB device-to-host copy saturates the
    bus and slows the uploads and launches it overlaps, so it is kept off them), and batch k's
    trace waits on the device for the readback that last used its image buffers."""
    outs = [B.out_b, [torch.empty_like(o) for o in B.out_b]]
    prepared = [B.prepared, B.batch.prepare([(o, w.camera, w.params, out)
                                             for o, w, out in zip(B.objs, B.ws, outs[1])])]
    hosts = [[torch.empty(tuple(o.shape), dtype=torch.float32, pin_memory=True) for o in B.out_b] for _ in range(2)]
    copy_stream = torch.cuda.Stream()
    built = [torch.cuda.Event(), torch.cuda.Event()]
    copied = [torch.cuda.Event(), torch.cuda.Event()]
    last = torch.cuda.Event()
    counter = torch.zeros(1, dtype=torch.int64, device="cuda")

    def read_back(j, after):
        copy_stream.wait_event(after)
        with torch.cuda.stream(copy_stream):
            for h, d in zip(hosts[j], outs[j]):
                h.copy_(d, non_blocking=True)
        copied[j].record(copy_stream)

    def step(k):
        i = k % 2
        for o, w in zip(B.objs, B.ws):
            o.upload(w.scene, stream)
        pr.build_bvh_many(B.objs, stream)
        built[i].record(stream)
        if k >= 1:
            read_back(1 - i, built[i])         # batch k-1's images, behind batch k's builds
        if k >= 2:
            stream.wait_event(copied[i])      # batch k-2's readback of these buffers is done
        B.batch.trace(prepared=prepared[i], ray_counter=counter, stream=stream, graph=True)

    def run(n):
        for k in range(n):
            step(k)
        last.record(stream)
        read_back((n - 1) % 2, last)
        copy_stream.synchronize()
        torch.cuda.synchronize()

    run(warmup)
    counter.zero_()
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    run(n_steps)
    pipe_ms, rays = aggregate_over_ranks((time.perf_counter() - t0) * 1e3, int(counter.item()), world, "cuda")
    return {"value": rays / (pipe_ms / 1e3) / 1e6, "unit": "Mrays/s",
            "h2d_bytes_per_step": int(sum(o.desc_bytes for o in B.objs)),
            "d2h_bytes_per_step": int(sum(o.numel() * 4 for o in B.out_b)),
            "ms_per_step": pipe_ms / n_steps,
            "mode": f"{n_steps} consecutive batches, each: 64 scene descriptions from host memory to the device, "
                    "64 BVH builds, one batched graph launch, 64 RGB images to pinned host memory; the readback "
                    "of batch k-1 overlaps batch k's trace (the timed region ends with the last batch's readback)"}


def batch_cpu_baseline(ws, fraction: int = 64, seed: int = 4) -> dict:
    """The FP64 oracle, as it stands, on a seeded 1/64 pixel sample of every request."""
    import oracle
    threads = os.cpu_count() or 1
    rays = px = 0
    t0 = time.perf_counter()
    for q, w in enumerate(ws):
        n = max(1, w.params.width * w.params.height // fraction)
        ref = oracle.render(w, pixels=scenes.sample_pixels(w.params.width, w.params.height, n, seed=seed + q),
                            threads=threads)
        rays += int(ref["rays"].sum())
        px += n
    dt = time.perf_counter() - t0
    return {"value": rays / dt / 1e6, "unit": "Mrays/s", "cores": threads, "kind": "oracle",
            "sample": f"seeded 1/{fraction} pixel sample of each of the {len(ws)} requests ({px} pixels, {rays} "
                      f"rays, {dt:.1f} s, FP64); Mrays/s of the sample, extrapolated to the whole batch"}


class _RequestPool:
    """Serving request stream: scene descriptions cached by (kind, seed) so the
    generator runs once per scene, as a client holding its scenes would."""

    def __init__(self, seed: int):
        self.rng = np.random.default_rng(seed)
        self.descs = {}

    def next(self):
        kind, sseed, wl = scenes.serving_request(self.rng, build=lambda k, s: self.descs.get((k, s)))
        self.descs.setdefault((kind, sseed), wl.scene)
        key = (kind << 32) | sseed
        return key, self.descs[(kind, sseed)], wl.camera, wl.params


def bench_serving(pr, torch, rates, n_requests, mode, tuning=None, max_seconds=40.0, seed=0) -> list:
    """Poisson arrivals at each rate; per-request latency = completion - submission."""
    out_rows = []
    ring = [torch.empty(1920 * 1080 * 4, dtype=torch.float32, device="cuda") for _ in range(128)]
    for lam in rates:
        pool = _RequestPool(seed)
        n = int(min(n_requests, max(20, lam * max_seconds)))
        reqs = [pool.next() for _ in range(n)]
        gaps = np.random.default_rng(seed + 1).exponential(1.0 / lam, n)
        srv = pr.Server(mode=mode, max_active=64, mem_budget_bytes=100 << 30, max_batch_pixels=16 << 20,
                        tuning=tuning, solo_max_waiting=SERVE_SOLO_MAX_WAITING)
        tickets = []
        t0 = time.perf_counter()
        due = t0
        for k, (key, desc, cam, tp) in enumerate(reqs):
            due += gaps[k]
            while True:
                now = time.perf_counter()
                if now >= due:
                    break
                time.sleep(min(due - now, 0.0005))
            if k >= len(ring):      # the ring slot's previous request must be done
                while not srv.poll(tickets[k - len(ring)])[0]:
                    time.sleep(0.0002)
            out = ring[k % len(ring)][: tp.width * tp.height * 4].view(tp.height, tp.width, 4)
            tickets.append(srv.submit(key, desc, cam, tp, out))
        srv.drain(600.0)
        st = [srv.poll(t)[1] for t in tickets]
        stats = srv.stats()
        srv.close()
        lat = np.array([s["t_done"] - s["t_submit"] for s in st]) * 1e3
        span = max(s["t_done"] for s in st) - min(s["t_submit"] for s in st)
        ok = sum(1 for s in st if s["status"] == 0)
        # where the latency goes: waiting for the scene (a build on a miss) and a slot, waiting
        # for the first launch, and from the first launch to completion
        phase = lambda a, b: np.array([s[b] - s[a] for s in st if s["status"] == 0]) * 1e3
        breakdown = {name: {"p50": float(np.percentile(v, 50)), "p99": float(np.percentile(v, 99))}
                     for name, v in (("admit_ms", phase("t_submit", "t_admit")),
                                     ("launch_wait_ms", phase("t_admit", "t_first_launch")),
                                     ("in_flight_ms", phase("t_first_launch", "t_done"))) if len(v)}
        hits = np.array([s["cache_hit"] for s in st], bool)
        loads = np.array([s["t_load_end"] - s["t_load_start"] for s in st if s["t_load_end"] > 0]) * 1e3
        if len(loads):
            breakdown["scene_load_ms"] = {"p50": float(np.percentile(loads, 50)), "p99": float(np.percentile(loads, 99)),
                                          "max": float(loads.max()), "n": int(len(loads))}
        out_rows.append({"rate_per_s": lam, "requests": n, "ok": ok, "mode": "continuous" if mode == 0 else "plain",
                         "p50_ms": float(np.percentile(lat, 50)), "p99_ms": float(np.percentile(lat, 99)),
                         "p99_ms_cache_hits": float(np.percentile(lat[hits], 99)) if hits.any() else None,
                         "value": stats["rays"] / span / 1e6, "unit": "Mrays/s", "makespan_s": span,
                         "iterations": stats["iterations"], "cache_hits": stats["cache_hits"],
                         "cache_misses": stats["cache_misses"], "scene_loads": stats["scene_loads"],
                         "breakdown": breakdown})
    return out_rows


def serving_tuning(tuning: dict) -> dict:
    """The batch's tuned shape for the server's iterations, but never a persistent mode: persistent
    CTAs (wavefront, persistent megakernel and regrouped stages) hold every SM for a whole iteration,
    so the loader's scene builds on the high-priority stream wait for its end (measured: scene loads
    of 3 / 15 ms p50 / p99 and an admission p99 of 47 ms at 1000 requests/s with the persistent
    megakernel); one CTA per tile lets them run between tiles."""
    t = dict(tuning)
    if t.get("megakernel") not in (2, 4):
        t.update(tile_w=16, tile_h=8, megakernel=2)
    return t


def serving_block(pr, torch, rates, n_requests, max_seconds, tuning) -> dict:
    tuning = serving_tuning(tuning)
    rows = []
    for mode in (pr.PR_SERVE_CONTINUOUS, pr.PR_SERVE_PLAIN):
        rows += bench_serving(pr, torch, rates, n_requests, mode, tuning, max_seconds)
    cont = {r["rate_per_s"]: r for r in rows if r["mode"] == "continuous"}
    plain = {r["rate_per_s"]: r for r in rows if r["mode"] == "plain"}
    compare = [{"rate_per_s": lam, "mrays_continuous_over_plain": cont[lam]["value"] / plain[lam]["value"],
                "p99_continuous_ms": cont[lam]["p99_ms"], "p99_plain_ms": plain[lam]["p99_ms"],
                "p50_continuous_ms": cont[lam]["p50_ms"], "p50_plain_ms": plain[lam]["p50_ms"]} for lam in rates]
    return {"workload": "serving: Poisson arrivals, teaser / instanced-field (100000 instances) scenes 50/50 from "
                        "pools of 16, resolution 512^2..1920x1080, orbit cameras, 100 GB budget, 64 slots, "
                        "16 Mpx per continuous-batching iteration; continuous mode runs the oldest request "
                        f"alone through pr_trace while at most {SERVE_SOLO_MAX_WAITING} requests wait",
            "tuning": tuning, "points": rows, "continuous_vs_plain": compare}


def cpu_baseline(w, budget_s: float = 15.0) -> dict:
    """The FP64 oracle, as it stands, on a seeded pixel sample of the same frame."""
    import oracle
    threads = os.cpu_count() or 1
    n_pix = w.params.width * w.params.height
    probe = scenes.sample_pixels(w.params.width, w.params.height, min(2000, n_pix), seed=3)
    t0 = time.perf_counter()
    oracle.render(w, pixels=probe, threads=threads)
    dt = time.perf_counter() - t0
    n = int(min(n_pix, max(len(probe), len(probe) * budget_s / max(dt, 1e-3) * 0.8)))
    pix = scenes.sample_pixels(w.params.width, w.params.height, n, seed=4)
    rays, passes = 0, 0
    t0 = time.perf_counter()
    while True:
        ref = oracle.render(w, pixels=pix, threads=threads)
        rays += int(ref["rays"].sum())
        passes += 1
        dt = time.perf_counter() - t0
        if n < n_pix or dt >= 0.65 * budget_s or passes >= 10000:
            break
    return {"value": rays / dt / 1e6, "unit": "Mrays/s", "cores": threads, "kind": "oracle",
            "sample": f"{passes} x {n} of {n_pix} pixels (seeded uniform sample), {rays} rays, {dt:.1f} s, "
                      f"FP64 brute force"}


def run_reference(args):
    """Reference arm: the CPU FP64 oracle, timed on the host cores, on the headline's workload;
    each step renders a bounded seeded sample of it."""
    rank = int(os.environ.get("RANK", "0"))
    if rank != 0:
        return
    import oracle
    threads = os.cpu_count() or 1
    if args.workload == BATCH:
        ws = scenes.batch_requests(0, 64)
        config = {"workload": BATCH_DESC, "config": BATCH, "requests": 64,
                  "pixels": sum(w.params.width * w.params.height for w in ws)}
        frac = 512
        sample_desc = f"seeded 1/{frac} pixel sample of each of the 64 requests per step"
    else:
        ws = [workload_by_name(args.workload)]
        config = workload_config(args.workload, ws[0])
        frac = 32
        sample_desc = f"seeded 1/{frac} pixel sample of the frame per step"
    times, rays = [], 0
    for k in range(args.warmup + args.steps):
        t0 = time.perf_counter()
        r = 0
        for q, w in enumerate(ws):
            n = max(1, w.params.width * w.params.height // frac)
            pix = scenes.sample_pixels(w.params.width, w.params.height, n, seed=100 + 97 * k + q)
            r += int(oracle.render(w, pixels=pix, threads=threads)["rays"].sum())
        dt = time.perf_counter() - t0
        if k >= args.warmup:
            times.append(dt)
            rays += r
    total = sum(times)
    value = rays / total / 1e6
    line = {"impl": "reference", "metric": "Mrays/s", "value": value, "unit": "Mrays/s", "n_gpus": args.gpus,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * total / args.steps,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": config,
            "cpu_baseline": {"value": value, "unit": "Mrays/s", "cores": threads, "kind": "oracle",
                             "sample": sample_desc},
            "e2e": {"value": value, "unit": "Mrays/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


def _strip(block: dict) -> dict:
    return {k: v for k, v in block.items() if not k.startswith("_")}


def run_ours(args):
    import torch
    import torch.distributed as dist
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    if world > 1:
        dist.init_process_group("nccl" if torch.cuda.is_available() else "gloo")
    torch.cuda.set_device(local)
    import paper_2012_10357_b300 as pr
    from paper_2012_10357_b300 import work

    stream = torch.cuda.Stream()
    with torch.cuda.stream(stream):
        flush = torch.empty(L2_FLUSH_BYTES // 4, dtype=torch.float32, device="cuda")
    # measured FP32 FMA throughput (all SMs, 8 independent FMA chains per thread)
    probe_tflops, _ = pr.fma_peak_probe(16384, stream=stream)

    def measure(fn):
        """The timed region, taken once more if the clocks show a slowdown or a leftover lock."""
        sampler = ClockSampler(torch.cuda.current_device())
        res = fn(sampler)
        first = None
        if ClockSampler.rejected(res["clocks"]):
            first = res["clocks"]
            res = fn(ClockSampler(torch.cuda.current_device()))
        if res["clocks"] is not None and first is not None:
            res["clocks"]["remeasured_after"] = first
        return res

    tuning_arg = None
    if args.tuning:
        v = [int(x) for x in args.tuning.split(",")]
        tuning_arg = dict(ctas_per_sm=v[0], tile_w=v[1], tile_h=v[2], queue_chunk=v[3], megakernel=v[4])
    if args.block:
        # one block alone (profiling runs)
        if args.block == "analytic_4096_frames":
            b = bench_analytic_frames(pr, work, torch, stream, flush, reps=args.steps, probe=probe_tflops)
        elif args.block == "field_100k_2160p_tlas":
            b = bench_tlas_variants(pr, work, torch, stream, flush, args.steps, args.warmup, probe_tflops)
        elif args.block == "teaser_1080p_batched":
            # the 1080p teaser as a one-request batch through the batched path (--tuning picks the mode)
            res = bench_batch(pr, work, torch, stream, flush, args.steps, args.warmup, 1, probe_tflops, None, 1,
                              tuning_arg, [scenes.teaser()])
            res["B"].close()
            b = {"workload": "teaser 1080p, one-request batch", "value": res["value"],
                 "ms_per_step": res["total_ms"] / args.steps, "tuning": res["autotune"], "roofline": res["roofline"],
                 "plain": res["plain"], "images_identical_to_plain": res["images_identical_to_plain"]}
        else:
            flags = (pr.PR_BUILD_TLAS_PLOC if args.tlas_builder == "ploc" else 0) | TLAS_FORMATS[args.tlas_format](pr)
            b = bench_scene(pr, work, torch, stream, flush, args.block, args.steps, args.warmup, probe_tflops,
                            args.binary_tlas, build_flags=flags)
            b["_scene"].close()
        print(json.dumps({"block": args.block, **_strip(b)}), flush=True)
        return
    if args.workload == BATCH:
        res = measure(lambda smp: bench_batch(pr, work, torch, stream, flush, args.steps, args.warmup, world,
                                              probe_tflops, smp, args.requests, tuning_arg))
        B = res["B"]
        e2e = None if args.no_e2e else batch_e2e(pr, torch, stream, B, max(3, args.steps), 2, world)
        config = {"workload": BATCH_DESC if B.n == 64 else BATCH_DESC.replace("64", str(B.n), 1),
                  "config": BATCH if B.n == 64 else f"batch{B.n}", "requests": B.n, "pixels": B.total_px,
                  "instances_per_request": [int(len(w.scene.inst_blas)) for w in B.ws],
                  "resolutions": [w.params.width for w in B.ws], "max_depth": 1, "rays_per_pixel_max": 2,
                  "step": "device LBVH builds of the 64 scenes + one batched launch (CUDA graph, autotuned shape)",
                  "output": "rgb float32 images, 12 B/pixel", "l2": "flushed between timed steps (256 MB write); "
                  "the batch's images (1.0 GB) exceed L2", "parallelism": "replicas", "tuning": B.tuned["tuning"]}
        step_ms, build_ms, trace_ms = res["step_ms"], res["build_ms"], res["trace_ms"]
        head = {"value": res["value"], "ms_per_step": res["total_ms"] / args.steps, "config": config,
                "latency_ms": {"p50": float(np.percentile(step_ms, 50)), "p99": float(np.percentile(step_ms, 99)),
                               "per_request": "every request of a batch completes with the batch's launch",
                               "build_p50": float(np.percentile(build_ms, 50)),
                               "trace_p50": float(np.percentile(trace_ms, 50))},
                "rays_per_step": res["rays"] / args.steps, "roofline": res["roofline"], "e2e": e2e,
                "gpu_launches": res["gpu_launches_per_step"] * args.steps, "clocks": res["clocks"],
                "plain": res["plain"],
                "batched_vs_plain": {"mrays": res["value"] / res["plain"]["value"],
                                     "p99_batched_ms": float(np.percentile(step_ms, 99)),
                                     "p99_plain_ms": res["plain"]["latency_ms"]["p99"]},
                "images_identical_to_plain": res["images_identical_to_plain"], "autotune": res["autotune"],
                "batch_device_bytes": res["batch_device_bytes"],
                "device_error_word": max(o.error_word(stream) for o in B.objs)}
        tuning = B.tuned["tuning"]
        ws_for_cpu = B.ws
        B.close()
    else:
        res = measure(lambda smp: bench_scene(pr, work, torch, stream, flush, args.workload, args.steps, args.warmup,
                                              probe_tflops, args.binary_tlas, smp))
        e2e = None if args.no_e2e else scene_e2e(pr, torch, stream, res, max(3, min(args.steps, 100)), args.warmup,
                                                  world)
        total_ms, rays_all = aggregate_over_ranks(res["ms_per_step"] * args.steps, res["rays_per_step"] * args.steps,
                                                  world, "cuda")
        head = {"value": rays_all / (total_ms / 1e3) / 1e6, "ms_per_step": total_ms / args.steps,
                "config": res["config"], "latency_ms": res["latency_ms"], "rays_per_step": res["rays_per_step"],
                "roofline": res["roofline"], "e2e": e2e, "gpu_launches": res["gpu_launches_per_step"] * args.steps,
                "clocks": res.get("clocks"), "device_error_word": res["device_error_word"]}
        tuning = None
        ws_for_cpu = None
        res["_scene"].close()

    extra = {}
    if not args.no_extra and rank == 0:
        field_img = None
        for name, steps in (("teaser_1080p", 500), ("field_100k_2160p", 60)):
            if name != args.workload:
                b = bench_scene(pr, work, torch, stream, flush, name, steps, 3, probe_tflops)
                if name == "field_100k_2160p":
                    field_img = b["_out"].clone()
                b["_scene"].close()
                extra[name] = _strip(b)
        # the same field with its TLAS built by PLOC (same images, fewer node visits)
        b = bench_scene(pr, work, torch, stream, flush, "field_100k_2160p", 60, 3, probe_tflops,
                        build_flags=pr.PR_BUILD_TLAS_PLOC)
        if field_img is not None:
            b["images_identical_to_lbvh"] = bool(torch.equal(b["_out"], field_img))
            del field_img
        b["_scene"].close()
        extra["field_100k_2160p_ploc"] = _strip(b)
        extra["analytic_4096_frames"] = bench_analytic_frames(pr, work, torch, stream, flush, probe=probe_tflops)
        if tuning is None:
            tuning = {"ctas_per_sm": 4, "tile_w": 16, "tile_h": 8, "queue_chunk": 32, "megakernel": 2}
        extra["serving"] = serving_block(pr, torch, args.serve_rates, args.serve_requests, args.serve_max_seconds,
                                         tuning)

    if rank != 0:
        if world > 1:
            dist.barrier()
            dist.destroy_process_group()
        return
    line = {"metric": "Mrays/s", "value": head["value"], "unit": "Mrays/s", "n_gpus": world, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": head["ms_per_step"], "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "f32", "data": "synthetic", **head, **extra}
    if not args.no_cpu_baseline:
        line["cpu_baseline"] = (batch_cpu_baseline(ws_for_cpu) if ws_for_cpu is not None
                                else cpu_baseline(workload_by_name(args.workload), args.cpu_budget))
    print(json.dumps(line), flush=True)
    if world > 1:
        dist.barrier()
        dist.destroy_process_group()


def run_serve_sweep(args):
    """Serving sweep: Poisson rates x {continuous batching, plain per-request launches}."""
    import torch
    import paper_2012_10357_b300 as pr
    torch.cuda.set_device(int(os.environ.get("LOCAL_RANK", "0")))
    tune_path = os.path.join(ROOT, "paper_2012_10357_b300", "tuning_cache.json")
    tuning = None
    if os.path.exists(tune_path):
        cache = json.load(open(tune_path))
        mine = [v for k, v in cache.items() if k.startswith(torch.cuda.get_device_name() + "|batch")]
        tuning = mine[0]["tuning"] if mine else None
    tuning = tuning or {"ctas_per_sm": 4, "tile_w": 16, "tile_h": 8, "queue_chunk": 32, "megakernel": 2}
    block = serving_block(pr, torch, args.serve_rates, args.serve_requests, args.serve_max_seconds, tuning)
    print(json.dumps({"metric": "serving p50/p99 latency and Mrays/s", **block}), flush=True)


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=None,
                    help="timed steps (default: about 0.5-1.5 s of GPU work for the workload; 20 for the reference)")
    ap.add_argument("--warmup", type=int, default=5)
    ap.add_argument("--impl", choices=["ours", "reference"], default="ours")
    ap.add_argument("--workload", choices=[BATCH, *SINGLE], default=BATCH)
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-extra", action="store_true",
                    help="skip the teaser, 4096-frame, 100k-field and serving blocks")
    ap.add_argument("--serve-rates", type=float, nargs="+", default=SERVE_RATES)
    ap.add_argument("--serve-requests", type=int, default=400)
    ap.add_argument("--serve-max-seconds", type=float, default=40.0)
    ap.add_argument("--serve-only", action="store_true", help="only the serving sweep (both modes), one JSON line")
    ap.add_argument("--binary-tlas", action="store_true", help="traverse the binary TLAS instead of the 4-wide one")
    ap.add_argument("--tlas-builder", choices=["lbvh", "ploc"], default="lbvh",
                    help="TLAS builder of a --block scene (PLOC: PR_BUILD_TLAS_PLOC)")
    ap.add_argument("--tlas-format", choices=list(TLAS_FORMATS), default="greedy4",
                    help="wide TLAS of a --block scene: greedy 4-wide (default build), 4-wide by depth parity, "
                         "8-wide quantised, 8-wide float")
    ap.add_argument("--cpu-budget", type=float, default=15.0)
    ap.add_argument("--requests", type=int, default=64, help="requests of the batch workload (64: the headline)")
    ap.add_argument("--block", choices=["analytic_4096_frames", "teaser_1080p", "field_100k_2160p",
                                        "teaser_1080p_batched", "field_100k_2160p_tlas"], default=None,
                    help="run one block alone and print it (profiling)")
    ap.add_argument("--tuning", default=None,
                    help="batch launch shape ctas_per_sm,tile_w,tile_h,queue_chunk,mode instead of the autotuned one")
    args = ap.parse_args()
    if args.warmup < 3:
        args.warmup = 3
    if args.steps is None:
        # long enough for the clock samples (every 50 ms) to fall inside the timed region
        args.steps = 20 if args.impl == "reference" else DEFAULT_STEPS[args.workload]
    if args.impl == "reference":
        run_reference(args)
    elif args.serve_only:
        run_serve_sweep(args)
    else:
        run_ours(args)


if __name__ == "__main__":
    main()
