#!/usr/bin/env python3
"""Benchmark of the procedural ray tracer: Mrays/s and frame latency.

One step = one pass of the whole hot path over the workload: device LBVH
build (BLASes, instance boxes, TLAS) and one full frame (primary, shadow and
mirror rays through two-level traversal, Eq. 1 dispatch, intersection and
closest-hit shaders). Default workload: the teaser-like scene (two pac-men, a
quaternion Julia set, a Mandelbulb, a mirror ground slab) at 1920x1080.

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
# default timed steps per workload: about 0.5-1.5 s of GPU work on a B300
DEFAULT_STEPS = {"analytic_64x64": 2000, "analytic_64x64_x4096": 500, "teaser_1080p": 2000, "field_100k_2160p": 150}


def workload_by_name(name: str):
    if name in ("analytic_64x64", "analytic_64x64_x4096"):
        return scenes.small_analytic()
    if name == "teaser_1080p":
        return scenes.teaser()
    if name == "field_100k_2160p":
        return scenes.field()
    raise SystemExit(f"unknown workload {name}")


def workload_config(name: str, w) -> dict:
    d = {"workload": {"analytic_64x64": "tiny analytic scene, 4 AABB primitives, one BLAS",
                      "analytic_64x64_x4096": "tiny analytic scene, 4096 eye-jittered 64x64 frames per launch",
                      "teaser_1080p": "teaser scene: 2 pac-men + quaternion Julia + Mandelbulb + mirror slab",
                      "field_100k_2160p": "instanced field, 100000 instances of 8 procedural types"}[name],
         "config": name, "width": w.params.width, "height": w.params.height,
         "instances": int(len(w.scene.inst_blas)), "max_depth": w.params.max_depth,
         "rays_per_pixel_max": 1 + 1 + (1 if w.params.max_depth >= 2 else 0),
         "step": "device LBVH build + one frame", "output": "rgb float32 image, 12 B/pixel",
         "l2": "flushed between timed steps (256 MB write)",
         "parallelism": "replicas"}
    return d


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


# DRAM traffic of one timed k_trace launch (dram__bytes_read.sum + dram__bytes_write.sum,
# one ncu capture of this script's own command, L2 flushed before the launch as in the timed
# loop), per workload and traversal mode. A figure holds only for the kernel sources it was
# taken on: it is keyed by their SHA-1 and reported as null once they change.
TRACE_SOURCES = ["paper_2012_10357_b300/csrc/trace.cu", "paper_2012_10357_b300/csrc/tracer.cuh",
                 "paper_2012_10357_b300/csrc/shaders.cuh", "paper_2012_10357_b300/csrc/pr_device.cuh",
                 "include/proceduray.h"]
TRACE_TRAFFIC = {   # {sha1 of TRACE_SOURCES: {workload: bytes per launch}}
    "2f46009b9da347812ca83a8837584c033c9f8967": {"teaser_1080p": 142592 + 306688,
                                                 "field_100k_2160p": 6126592 + 52024832,
                                                 "analytic_64x64_x4096": 403456 + 154923008},
}


def trace_sources_sha1() -> str:
    import hashlib
    h = hashlib.sha1()
    for rel in TRACE_SOURCES:
        with open(os.path.join(ROOT, rel), "rb") as f:
            h.update(f.read())
    return h.hexdigest()


def trace_traffic(workload: str, binary_tlas: bool):
    if binary_tlas:
        return None
    return TRACE_TRAFFIC.get(trace_sources_sha1(), {}).get(workload)


def measured_peaks() -> dict:
    p = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(p):
        with open(p) as f:
            return json.load(f)
    return {}


def _events(torch, n):
    return [torch.cuda.Event(enable_timing=True) for _ in range(n)]


def bench_analytic_frames(pr, work, torch, stream, flush, frames=4096, reps=5) -> dict:
    """The tiny analytic scene as a throughput run: 4096 eye-jittered 64x64 frames in one launch."""
    w = scenes.small_analytic()
    cams = pr.CameraArray(scenes.small_analytic_cameras(0, frames))   # marshalled once
    with torch.cuda.stream(stream):
        scene = pr.Scene(w.scene, stream=stream)
        out = torch.empty((frames, 64, 64, 4), dtype=torch.float32, device="cuda")
        counter = torch.zeros(1, dtype=torch.int64, device="cuda")
    for _ in range(2):
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
    counters = scene.trace_work(None, w.params, out=out, cameras=cams, stream=stream)
    flops = work.frame_flops(counters)
    avg_s = statistics.mean(ms) / 1e3
    props = torch.cuda.get_device_properties(torch.cuda.current_device())
    peak = work.fp32_peak_tflops(props.multi_processor_count, float(measured_peaks().get("sm_max_mhz", 2032.0)))
    scene.close()
    return {"workload": "tiny analytic scene: 4096 eye-jittered 64x64 frames, one pr_trace_frames launch",
            "value": rays / avg_s / 1e6, "unit": "Mrays/s", "ms_per_launch": statistics.mean(ms),
            "rays_per_launch": rays,
            "roofline": {"bound": "alu", "achieved": flops / avg_s / 1e12, "peak": peak, "unit": "TFLOP/s",
                         "frac": flops / avg_s / 1e12 / peak, "flops_per_launch": flops}}


def bench_batched(pr, torch, stream, flush, n_requests=64, reps=3) -> dict:
    """Batch: 64 requests of uneven size, one batched wavefront launch (CUDA
    graph, autotuned launch shape) vs 64 plain per-request launches."""
    ws = scenes.batch_requests(0, n_requests)
    total_px = sum(w.params.width * w.params.height for w in ws)
    with torch.cuda.stream(stream):
        objs = [pr.Scene(w.scene, stream=stream) for w in ws]
        outs_plain = [torch.empty((w.params.height, w.params.width, 4), device="cuda") for w in ws]
        outs_batch = [torch.empty((w.params.height, w.params.width, 4), device="cuda") for w in ws]
        counter = torch.zeros(1, dtype=torch.int64, device="cuda")
    batch = pr.Batch(n_requests, total_px)
    items = [(o, w.camera, w.params, out) for o, w, out in zip(objs, ws, outs_batch)]
    tune_path = os.path.join(ROOT, "paper_2012_10357_b300", "tuning_cache.json")
    key = f"{torch.cuda.get_device_name()}|batch|{n_requests}|{total_px}"
    cache = json.load(open(tune_path)) if os.path.exists(tune_path) else {}
    if key in cache:
        batch.set_tuning(**cache[key]["tuning"])
        tuned = dict(cache[key], from_cache=True)
    else:
        best, best_ms = batch.autotune(items, stream=stream)
        tuned = {"tuning": best, "ms": best_ms, "from_cache": False}
        cache[key] = {"tuning": best, "ms": best_ms}
        with open(tune_path, "w") as f:
            json.dump(cache, f, indent=1)

    def plain_once(record=None):
        for k, (o, w, out) in enumerate(zip(objs, ws, outs_plain)):
            o.trace(w.camera, w.params, out=out, ray_counter=counter, stream=stream)
            if record is not None:
                record[k].record(stream)

    # warm both paths
    plain_once()
    batch.trace(items, stream=stream, graph=True)
    stream.synchronize()
    res = {}
    for mode in ("plain", "batched_graph", "batched_direct"):
        counter.zero_()
        totals, lat = [], []
        for rep in range(reps):
            with torch.cuda.stream(stream):
                flush.fill_(float(rep))
            ev0 = torch.cuda.Event(enable_timing=True)
            done = _events(torch, n_requests if mode == "plain" else 1)
            ev0.record(stream)
            if mode == "plain":
                plain_once(done)
            else:
                batch.trace(items, ray_counter=counter, stream=stream, graph=(mode == "batched_graph"))
                done[0].record(stream)
            stream.synchronize()
            t = [ev0.elapsed_time(e) for e in done]
            totals.append(t[-1])
            lat += t if mode == "plain" else [t[0]] * n_requests
        rays = int(counter.item()) / reps
        res[mode] = {"value": rays / (statistics.mean(totals) / 1e3) / 1e6, "unit": "Mrays/s",
                     "ms_per_batch": statistics.mean(totals), "p50_ms": float(np.percentile(lat, 50)),
                     "p99_ms": float(np.percentile(lat, 99)), "rays_per_batch": rays}
    identical = all(torch.equal(a, b) for a, b in zip(outs_plain, outs_batch))
    out = {"workload": f"batch: {n_requests} requests, resolutions from {{256^2..2048^2}}, "
                       f"1..10000 instances each, {total_px} pixels",
           "plain": res["plain"], "batched_graph": res["batched_graph"], "batched_direct": res["batched_direct"],
           "speedup_graph_vs_plain": res["plain"]["ms_per_batch"] / res["batched_graph"]["ms_per_batch"],
           "images_identical_to_plain": identical, "autotune": tuned,
           "batch_device_bytes": batch.device_bytes()}
    batch.close()
    for o in objs:
        o.close()
    return out


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


def bench_serving(pr, torch, rates, n_requests, mode, tuning=None, max_seconds=60.0, seed=0) -> list:
    """Poisson arrivals at each rate; per-request latency = completion - submission."""
    out_rows = []
    ring = [torch.empty(1920 * 1080 * 4, dtype=torch.float32, device="cuda") for _ in range(128)]
    for lam in rates:
        pool = _RequestPool(seed)
        n = int(min(n_requests, max(20, lam * max_seconds)))
        reqs = [pool.next() for _ in range(n)]
        gaps = np.random.default_rng(seed + 1).exponential(1.0 / lam, n)
        srv = pr.Server(mode=mode, max_active=64, mem_budget_bytes=100 << 30, max_batch_pixels=8 << 20,
                        tuning=tuning)
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
        # where the latency goes: waiting for the scene (build on a miss) and a slot, waiting for
        # the first launch, and from the first launch to completion
        phase = lambda a, b: np.array([s[b] - s[a] for s in st if s["status"] == 0]) * 1e3
        breakdown = {name: {"p50": float(np.percentile(v, 50)), "p99": float(np.percentile(v, 99))}
                     for name, v in (("admit_ms", phase("t_submit", "t_admit")),
                                     ("launch_wait_ms", phase("t_admit", "t_first_launch")),
                                     ("in_flight_ms", phase("t_first_launch", "t_done"))) if len(v)}
        out_rows.append({"rate_per_s": lam, "requests": n, "ok": ok, "mode": "continuous" if mode == 0 else "plain",
                         "p50_ms": float(np.percentile(lat, 50)), "p99_ms": float(np.percentile(lat, 99)),
                         "value": stats["rays"] / span / 1e6, "unit": "Mrays/s", "makespan_s": span,
                         "iterations": stats["iterations"], "cache_hits": stats["cache_hits"],
                         "cache_misses": stats["cache_misses"], "breakdown": breakdown})
    return out_rows


def cpu_baseline(w, budget_s: float = 15.0) -> dict:
    """The FP64 oracle, as it stands, on a seeded pixel sample of the same frame."""
    import oracle
    threads = os.cpu_count() or 1
    n_pix = w.params.width * w.params.height
    probe = scenes.sample_pixels(w.params.width, w.params.height, min(2000, n_pix), seed=3)
    t0 = time.perf_counter()
    ref = oracle.render(w, pixels=probe, threads=threads)
    dt = time.perf_counter() - t0
    n = int(min(n_pix, max(len(probe), len(probe) * budget_s / max(dt, 1e-3) * 0.8)))
    pix = scenes.sample_pixels(w.params.width, w.params.height, n, seed=4)
    # a frame smaller than the budget is rendered whole, repeatedly, for about 10 s
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
    """Reference arm: the CPU FP64 oracle, timed on the host cores."""
    rank = int(os.environ.get("RANK", "0"))
    if rank != 0:
        return
    import oracle
    w = workload_by_name(args.workload)
    threads = os.cpu_count() or 1
    n_pix = w.params.width * w.params.height
    per_step = min(n_pix, max(4096, n_pix // 32))     # ~65k pixels of a 1080p frame per step
    times, rays = [], 0
    for k in range(args.warmup + args.steps):
        pix = scenes.sample_pixels(w.params.width, w.params.height, per_step, seed=100 + k)
        t0 = time.perf_counter()
        ref = oracle.render(w, pixels=pix, threads=threads)
        dt = time.perf_counter() - t0
        if k >= args.warmup:
            times.append(dt)
            rays += int(ref["rays"].sum())
    total = sum(times)
    value = rays / total / 1e6
    line = {"impl": "reference", "metric": "Mrays/s", "value": value, "unit": "Mrays/s", "n_gpus": args.gpus,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * total / args.steps,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": workload_config(args.workload, w),
            "cpu_baseline": {"value": value, "unit": "Mrays/s", "cores": threads, "kind": "oracle",
                             "sample": f"{per_step} seeded pixels of {n_pix} per step"},
            "e2e": {"value": value, "unit": "Mrays/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


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

    w = workload_by_name(args.workload)
    frames = None
    if args.workload == "analytic_64x64_x4096":
        frames = pr.CameraArray(scenes.small_analytic_cameras(0, 4096))    # marshalled once, outside the timed region
    stream = torch.cuda.Stream()
    H, W = w.params.height, w.params.width
    with torch.cuda.stream(stream):
        scene = pr.Scene(w.scene, stream=stream)
        # the image as r, g, b floats per pixel (PR_TRACE_OUTPUT_RGB: the alpha channel, always 1, is not stored)
        out = torch.empty(((len(frames),) if frames else ()) + (H, W, 3), dtype=torch.float32, device="cuda")
        counter = torch.zeros(1, dtype=torch.int64, device="cuda")
        flush = torch.empty(L2_FLUSH_BYTES // 4, dtype=torch.float32, device="cuda")

    def do_trace():
        if frames:
            scene.trace_frames(frames, w.params, out=out, ray_counter=counter, stream=stream)
        else:
            scene.trace(w.camera, w.params, out=out, ray_counter=counter, stream=stream,
                        binary_tlas=args.binary_tlas)

    def step():
        scene.build_bvh(stream)
        do_trace()

    def barrier():
        if world > 1:
            dist.barrier()

    for _ in range(args.warmup):
        step()
    stream.synchronize()
    counter.zero_()
    torch.cuda.synchronize()

    def timed_region():
        counter.zero_()
        torch.cuda.synchronize()
        ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True),
               torch.cuda.Event(enable_timing=True)) for _ in range(args.steps)]
        sampler = ClockSampler(torch.cuda.current_device())
        sampler.start()
        barrier()
        torch.cuda.synchronize()
        sampler.begin()
        with torch.cuda.stream(stream):
            for k in range(args.steps):
                flush.fill_(float(k))                 # evict L2 between timed steps
                ev[k][0].record(stream)
                scene.build_bvh(stream)
                ev[k][1].record(stream)
                do_trace()
                ev[k][2].record(stream)
        stream.synchronize()
        torch.cuda.synchronize()
        sampler.end()
        barrier()
        return ev, sampler.stop()

    ev, clocks = timed_region()
    first_clocks = None
    if ClockSampler.rejected(clocks):
        first_clocks = clocks
        ev, clocks = timed_region()
    if clocks is not None and first_clocks is not None:
        clocks["remeasured_after"] = first_clocks
    step_ms = [a.elapsed_time(c) for a, b, c in ev]
    trace_ms = [b.elapsed_time(c) for a, b, c in ev]
    build_ms = [a.elapsed_time(b) for a, b, c in ev]
    total_ms = sum(step_ms)
    rays = int(counter.item())
    n_build, n_trace = scene.kernel_launches()
    err = scene.error_word(stream)

    # end to end through the public API: host description -> device (pinned staging, one copy),
    # build, frame, image -> pinned host memory, every step
    e2e = None
    if not args.no_e2e:
        n_e2e = max(3, min(args.steps, 100))   # enough frames that the stream's fill and drain are small
        e2e_counter = torch.zeros(1, dtype=torch.int64, device="cuda")
        outs = [out, torch.empty_like(out)]
        hosts = [torch.empty(tuple(out.shape), dtype=torch.float32, pin_memory=True) for _ in range(2)]
        copy_stream = torch.cuda.Stream()
        traced = [torch.cuda.Event(), torch.cuda.Event()]
        copied = [torch.cuda.Event(), torch.cuda.Event()]

        def e2e_frame(k):
            i = k % 2
            if k >= 2:
                copied[i].synchronize()      # frame k-2 has reached the host before its buffers are reused
            scene.upload(w.scene, stream)
            scene.build_bvh(stream)
            if frames:
                scene.trace_frames(frames, w.params, out=outs[i], ray_counter=e2e_counter, stream=stream)
            else:
                scene.trace(w.camera, w.params, out=outs[i], ray_counter=e2e_counter, stream=stream)
            traced[i].record(stream)
            copy_stream.wait_event(traced[i])
            with torch.cuda.stream(copy_stream):
                hosts[i].copy_(outs[i], non_blocking=True)
            copied[i].record(copy_stream)

        # one frame at a time (each step's latency)
        serial_times = []
        for k in range(args.warmup + n_e2e):
            torch.cuda.synchronize()
            if k == args.warmup:
                e2e_counter.zero_()
                torch.cuda.synchronize()
            t0 = time.perf_counter()
            e2e_frame(k)
            copied[k % 2].synchronize()
            if k >= args.warmup:
                serial_times.append(time.perf_counter() - t0)
        serial_rays = int(e2e_counter.item())
        # a stream of frames: the readback of frame k overlaps the upload, build and trace of frame k+1
        for k in range(args.warmup):
            e2e_frame(k)
        torch.cuda.synchronize()
        e2e_counter.zero_()
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        for k in range(n_e2e):
            e2e_frame(k)
        torch.cuda.synchronize()
        pipe_s = time.perf_counter() - t0
        e2e_rays = int(e2e_counter.item())
        desc_bytes = scene.desc_bytes
        # every rank streams its own frames; the job's time is the slowest rank's
        pipe_ms, e2e_rays = aggregate_over_ranks(pipe_s * 1e3, e2e_rays, world, "cuda")
        serial_ms, serial_rays = aggregate_over_ranks(sum(serial_times) * 1e3, serial_rays, world, "cuda")
        pipe_s = pipe_ms / 1e3
        e2e = {"value": e2e_rays / pipe_s / 1e6, "unit": "Mrays/s",
               "h2d_bytes_per_step": int(desc_bytes) + (40 * len(frames) if frames else 0),
               "d2h_bytes_per_step": int(out.numel() * 4),
               "ms_per_step": 1e3 * pipe_s / n_e2e,
               "mode": f"{n_e2e} consecutive frames, each: description to the device, BVH build, frame, "
                       "image to pinned host memory; the image copy of frame k overlaps frame k+1 "
                       "(second stream, double-buffered image)",
               "serial": {"value": serial_rays / (serial_ms / 1e3) / 1e6, "unit": "Mrays/s",
                          "ms_per_step": serial_ms / n_e2e,
                          "mode": "one frame at a time, synchronised after each"}}

    total_all, rays_all = aggregate_over_ranks(total_ms, rays, world, "cuda")

    if rank != 0:
        if world > 1:
            dist.barrier()
            dist.destroy_process_group()
        return

    value = rays_all / (total_all / 1e3) / 1e6

    # roofline of the dominant kernel (the trace megakernel): FP32 ALU bound
    counters = scene.trace_work(w.camera, w.params, stream=stream, cameras=frames, binary_tlas=args.binary_tlas)
    torch.cuda.synchronize()
    flops = work.frame_flops(counters)
    trace_avg_s = statistics.mean(trace_ms) / 1e3
    props = torch.cuda.get_device_properties(torch.cuda.current_device())
    peaks = measured_peaks()
    sm_max = float(peaks.get("sm_max_mhz", 2032.0))
    peak_tflops = work.fp32_peak_tflops(props.multi_processor_count, sm_max)
    achieved_tflops = flops / trace_avg_s / 1e12
    roof = {"bound": "alu", "achieved": achieved_tflops, "peak": peak_tflops, "unit": "TFLOP/s",
            "frac": achieved_tflops / peak_tflops, "traffic": trace_traffic(args.workload, args.binary_tlas),
            "kernel": "k_trace (megakernel)", "flops_per_launch": flops,
            "peak_basis": f"{props.multi_processor_count} SMs x 128 FP32 lanes x 2 x {sm_max:.0f} MHz (sm_max_mhz of measured)",
            "trace_share_of_step": sum(trace_ms) / total_ms,
            "work_counters": {k: v for k, v in counters.items() if v}}
    if clocks:
        roof["peak_at_sampled_clock"] = work.fp32_peak_tflops(props.multi_processor_count, clocks["sm_mhz"])
        roof["frac_at_sampled_clock"] = achieved_tflops / roof["peak_at_sampled_clock"]
    sustained = (peaks.get("clocks_under_load") or {}).get("sm_mhz_median")
    if sustained:
        # the SM clock the driver saw under a seconds-long dense GEMM at the power cap
        roof["peak_at_measured_sustained_clock"] = work.fp32_peak_tflops(props.multi_processor_count, float(sustained))
        roof["frac_at_measured_sustained_clock"] = achieved_tflops / roof["peak_at_measured_sustained_clock"]
    if roof["traffic"]:
        # DRAM bytes of a launch over its mean duration, against the measured copy bandwidth
        roof["traffic_gbs"] = roof["traffic"] / trace_avg_s / 1e9
        if peaks.get("hbm_gbs"):
            roof["traffic_frac_of_hbm"] = roof["traffic_gbs"] / float(peaks["hbm_gbs"])
    # measured FP32 FMA throughput (all SMs, 8 independent FMA chains per thread)
    probe_tflops, _ = pr.fma_peak_probe(16384, stream=stream)
    roof["peak_fma_probe"] = probe_tflops
    roof["frac_of_fma_probe"] = achieved_tflops / probe_tflops if probe_tflops > 0 else None

    extra = {}
    if not args.no_extra:
        extra["analytic_4096_frames"] = bench_analytic_frames(pr, work, torch, stream, flush)
        extra["batched"] = bench_batched(pr, torch, stream, flush)
        tuning = extra["batched"]["autotune"]["tuning"]
        rows = []
        for mode in (pr.PR_SERVE_CONTINUOUS, pr.PR_SERVE_PLAIN):
            rows += bench_serving(pr, torch, args.serve_rates, args.serve_requests, mode, tuning)
        extra["serving"] = {"workload": "serving: Poisson arrivals, teaser / instanced-field (100000 instances) scenes "
                                        "50/50 from pools of 16, resolution 512^2..1920x1080, orbit cameras, "
                                        "100 GB budget, 64 slots, 8 Mpx per continuous-batching iteration",
                            "points": rows}

    line = {
        "metric": "Mrays/s", "value": value, "unit": "Mrays/s", "n_gpus": world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": total_all / args.steps, "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": "f32", "data": "synthetic",
        "config": workload_config(args.workload, w),
        "latency_ms": {"p50": float(np.percentile(step_ms, 50)), "p99": float(np.percentile(step_ms, 99)),
                       "build_p50": float(np.percentile(build_ms, 50)), "trace_p50": float(np.percentile(trace_ms, 50))},
        "rays_per_step": rays / args.steps,
        "roofline": roof,
        "e2e": e2e,
        "gpu_launches": (n_build + n_trace) * args.steps,
        "clocks": clocks,
        "device_error_word": err,
        **extra,
    }
    if not args.no_cpu_baseline:
        line["cpu_baseline"] = cpu_baseline(w, args.cpu_budget)
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
    rows = []
    for mode in (pr.PR_SERVE_CONTINUOUS, pr.PR_SERVE_PLAIN):
        rows += bench_serving(pr, torch, args.serve_rates, args.serve_requests, mode, tuning, args.serve_max_seconds)
    print(json.dumps({"metric": "serving p50/p99 latency and Mrays/s", "points": rows, "tuning": tuning}), flush=True)


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=None,
                    help="timed steps (default: about 0.5-1.5 s of GPU work for the workload; 20 for the reference)")
    ap.add_argument("--warmup", type=int, default=5)
    ap.add_argument("--impl", choices=["ours", "reference"], default="ours")
    ap.add_argument("--workload", choices=["analytic_64x64", "analytic_64x64_x4096", "teaser_1080p", "field_100k_2160p"], default="teaser_1080p")
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-extra", action="store_true", help="skip the 4096-frame throughput, batched and serving blocks")
    ap.add_argument("--serve-rates", type=float, nargs="+", default=[30.0, 1000.0])
    ap.add_argument("--serve-requests", type=int, default=120)
    ap.add_argument("--serve-max-seconds", type=float, default=60.0)
    ap.add_argument("--serve-only", action="store_true", help="only the serving sweep (both modes), one JSON line")
    ap.add_argument("--binary-tlas", action="store_true", help="traverse the binary TLAS instead of the 4-wide one")
    ap.add_argument("--cpu-budget", type=float, default=15.0)
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
