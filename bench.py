"""Benchmark: 1080p frames/s and p50/p99 latency of the forward 3DGS renderer
on a 3M-Gaussian scene, served FP16 (batched launch sets) vs plain FP32.

One step = one fused launch set of V 1080p views (V independent 6DoF
trajectories) of the resident 3M-Gaussian FP16 scene: preprocess, depth sort,
scan, emit, pair sort, tile ranges and blend, outputs in device memory.  The
timed steps go through ``tigas_render_batch_async`` with the next launch set
queued before the previous one is waited on.  ``value`` = frames/s over the
timed steps (CUDA events on the launching stream), ``e2e`` = the same calls
with pinned host output buffers (device->host copies inside the timed region,
on the tickets' copy streams).
Also reported: the plain FP32 single-request path, the request server
(closed-loop clients), per-stage CUDA-event times with the roofline of the
dominant stage, GPU clocks, and the FP64 CPU oracle timed on the host cores.

``--impl reference`` times the FP64 oracle (the only reference for this
method) on the same workload, one bounded sample per step.

Usage: python bench.py [--gpus N] [--steps K] [--warmup W] [--impl tigas|reference]
Under torchrun each rank renders its own replica (weak scaling, no collective
on the data path); rank 0 prints one JSON line.
"""
from __future__ import annotations

import argparse
import json
import math
import os
import statistics
import subprocess
import sys
import threading
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

import synth  # noqa: E402

METRIC = "1080p frames/s & p50/p99 latency, 3M Gaussians: served FP16 vs plain FP32"
WORKLOAD = "3M Gaussians (64 anisotropic blobs, SH degree 3), 1920x1080, 6DoF random-walk trajectories"
N_SM = 148
FP32_LANES_PER_SM = 128


def _peaks() -> dict:
    p = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(p):
        with open(p) as f:
            d = json.load(f)
        d["source"] = "measured"
        return d
    return {"hbm_gbs": 6400.0, "bf16_tflops": 1800.0, "sm_max_mhz": 2032.0, "source": "fallback"}


# ------------------------------------------------------------------ clocks


class ClockSampler:
    """nvidia-smi clocks and throttle reasons sampled during the timed region."""

    FIELDS = ("clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,clocks_event_reasons.hw_slowdown,"
              "clocks_event_reasons.hw_thermal_slowdown,clocks_event_reasons.sw_thermal_slowdown,"
              "clocks_event_reasons.sw_power_cap")

    def __init__(self, index: int):
        self.index = index
        self.proc = None
        self.lines: list[str] = []
        self.t = None

    def start(self):
        try:
            self.proc = subprocess.Popen(["nvidia-smi", "-i", str(self.index), f"--query-gpu={self.FIELDS}",
                                          "--format=csv,noheader,nounits", "-lms", "200"],
                                         stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.t = threading.Thread(target=self._read, daemon=True)
            self.t.start()
        except OSError:
            self.proc = None

    def _read(self):
        for line in self.proc.stdout:
            self.lines.append(line.strip())

    def stop(self) -> dict:
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        time.sleep(0.25)
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except subprocess.TimeoutExpired:
            self.proc.kill()
        sm, smax, power, reasons = [], [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for line in self.lines:
            parts = [x.strip() for x in line.split(",")]
            if len(parts) < 8:
                continue
            try:
                sm.append(float(parts[0]))
                smax.append(float(parts[1]))
                power.append(float(parts[2]))
            except ValueError:
                continue
            for nm, v in zip(names, parts[4:8]):
                if v.lower() == "active":
                    reasons.add(nm)
        if not sm:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["no samples"]}
        return {"sm_mhz": statistics.median(sm), "sm_max_mhz": max(smax), "sm_min_mhz": min(sm),
                "power_w_max": max(power), "samples": len(sm), "reasons": sorted(reasons)}


# ---------------------------------------------------------- CPU baseline


def oracle_frame(scene, pose, width: int, height: int, storage_half: bool = True) -> float:
    """Seconds the FP64 oracle takes for one whole frame (preprocess of every
    Gaussian, then every pixel of every tile composited), on the attributes
    of the given storage (FP16-rounded by default, as the GPU arm stores them)."""
    import oracle
    K = synth.default_intrinsics(width, height)
    t0 = time.perf_counter()
    pr = oracle.preprocess(scene, pose, K, width, height, storage_half=storage_half)
    oracle.render(pr)
    return time.perf_counter() - t0


def cpu_baseline(scene, poses, width, height, budget_s: float = 15.0) -> dict:
    """Whole oracle frames of the headline workload until budget_s has been
    spent (at least one)."""
    t_start = time.perf_counter()
    times = []
    while not times or (time.perf_counter() - t_start < budget_s and len(times) < len(poses)):
        times.append(oracle_frame(scene, poses[len(times)], width, height))
    return {"value": 1.0 / statistics.mean(times), "unit": "frames/s", "cores": os.cpu_count(), "kind": "oracle",
            "sample": (f"{len(times)} whole {width}x{height} frames of the {scene.n}-Gaussian scene (FP16-rounded "
                       f"attributes, FP64 arithmetic, OpenMP over pixel rows), one pose each; "
                       f"{time.perf_counter() - t_start:.1f} s of CPU work")}


# ---------------------------------------------------------------- roofline


# DRAM bytes (read + write) of the dominant kernel per view of a launch set, from one ncu capture of
# the same kernel sources (all six slices of a 4-view 1080p launch set of the 3M-Gaussian scene,
# dram__bytes_read.sum + dram__bytes_write.sum; profiles/blend_ncu_3M_1080p.md), scaled by the
# views a launch set renders.  Reported only while the sources' code (source_digest: comments
# aside) is the captured one: the blend's own file and the files that build its active list (the
# order in which it takes tiles).
KERNEL_TRAFFIC = {
    "blend": {"sources": ["paper_2605_08699_b300/csrc/blend.cu", "paper_2605_08699_b300/csrc/sliced.cu",
                          "paper_2605_08699_b300/csrc/sliced.cuh"],
              "sha1": "7389595234e910b537ae1a1cf5856a9b2c606ea4",
              "bytes_per_view": 366568192 / 4},
}


def source_digest(sources) -> str:
    """SHA-1 of the sources' code: each line without its // comment and
    surrounding blanks, empty lines dropped (comment edits keep the digest)."""
    import hashlib
    import re
    h = hashlib.sha1()
    for src in sources:
        with open(os.path.join(ROOT, src), encoding="utf-8") as f:
            for line in f:
                code = re.sub(r"//.*", "", line).strip()
                if code:
                    h.update(code.encode() + b"\n")
    return h.hexdigest()


def kernel_traffic(kernel: str, views: int):
    t = KERNEL_TRAFFIC.get(kernel)
    if not t:
        return None
    if source_digest(t["sources"]) != t["sha1"]:
        return None   # the kernel changed since the counters were taken
    return int(t["bytes_per_view"] * views)


# What bounds each stage below its roofline, from ncu captures of the same kernels
# (profiles/binning_ncu_3M_1080p.md, profiles/depth_sort_scatter_ncu_3M_1080p.md,
# profiles/preprocess_ncu_3M_1080p.md, profiles/blend_ncu_3M_1080p.md); copied into the stage entries of the bench line.
STAGE_LIMITS = {
    "preprocess": "instructions: 506 thread instructions per (Gaussian, view), 71 % issue active, DRAM 53 % "
                  "of peak; traffic equals the algorithmic bytes",
    "depth_sort": "instructions per key and load latency: 172-192 thread instructions per key per pass, "
                  "44-46 % issue active, long_scoreboard first, DRAM 20-27 % of peak; the threshold and "
                  "histogram kernels each read every key once",
    "scan": "latency: per slice a one-CTA-per-view running-tile table (8 us, barrier first), a count of "
            "46-1655 CTAs (long_scoreboard first) and a one-CTA block-sum scan (about 4 us)",
    "emit": "instructions per pair (45-57 % issue active, not_selected and wait first in the early slices); "
            "the pairs stay in L2 (slice 0: 0.2 MB of DRAM writes for 40 MB of pairs); the late slices "
            "emit from a list of their entries with pairs",
    "pair_sort": "latency and L2: the pair lists live in L2 (DRAM reads are the keys' first touch), later "
                 "slices' scatter passes run at 28-47 % warps active, plus a one-CTA digit-base kernel; the "
                 "last slice's six 64-bit passes about 10 us each",
    "ranges": "latency: a sampled search per tile, long_scoreboard first, 8-13 us per slice",
    "blend": "issue-bound in the first slice (77 % issue active), latency-bound in later ones "
             "(long_scoreboard first) and ended by their longest lists; not DRAM-bound (6-12 % of peak)",
}


def roofline(stage_ms: dict, per_step: dict, peaks: dict, clocks: dict, steps: int,
             timed_stage_ms: dict | None = None) -> tuple[dict, dict]:
    """Achieved rate of every stage (stage_ms: a pass with every stage timed) and
    the roofline entry of the dominant one, whose duration is taken from
    timed_stage_ms (its events recorded inside the timed region) when given.
    Algorithmic work per launch set of the sliced schedule, in bytes (blend: FP32 operations):
      preprocess  12 B per (Gaussian, view) + (A - 12) B per Gaussian + 52 B per kept entry
      depth_sort  24 B per entry and pass run (key and 8-byte compact rectangle with its entry id,
                  read and written), or 32 B with wide rectangles (key, value, rectangle): the
                  first pass over every entry, the later ones over the entries they sort (all, or
                  the near ones of a partial sort)
      scan        12 B per kept entry: the slice count reads the rectangle (8 B) and writes the
                  entry's offset within its block (4 B); the scan of the block sums is negligible
      emit        12 B per kept entry (rect, offset; + 4 B of order with wide rectangles)
                  + 8 B per emitted pair
      pair_sort   passes x 16 B per emitted pair
      ranges      8 B per tile per slice
      blend       FP32 flops: 14 per (pixel, list entry) evaluated until the pixel stops (the
                  per-evaluation figure of the method: offsets, quadratic form, exponent, alpha
                  cut-off and clamp; the ex2 is not counted)"""
    hbm = peaks["hbm_gbs"]
    mhz = clocks.get("sm_mhz") or peaks.get("sm_max_mhz", 2032.0)
    fp32_peak_tflops = N_SM * FP32_LANES_PER_SM * 2 * mhz * 1e6 / 1e12
    w = per_step
    bytes_per = {
        "preprocess": w["entries"] * 12 + w["gaussians"] * (w["attr_bytes"] - 12) + w["kept"] * 52,
        "depth_sort": (w["entries"] + w.get("depth_near", w["entries"]) * max(w["depth_passes"] - 1, 0))
                      * (24 if w.get("compact_rect") else 32),
        "scan": w["kept"] * 12,
        "emit": w["kept"] * (12 if w.get("compact_rect") else 16) + w["pairs"] * 8,
        "pair_sort": w["pairs"] * w["sort_passes"] * 16,
        "ranges": w["tiles"] * w["slices"] * 8,
    }
    stages = {}
    for name, st in stage_ms.items():
        if name == "frame" or st["calls"] == 0 or st["ms"] <= 0.0:
            continue
        ms = st["ms"] / st["calls"]
        if name == "blend":
            fl = w["evals"] * 14.0
            ach = fl / (ms * 1e-3) / 1e12
            stages[name] = {"ms": ms, "bound": "alu", "achieved": ach, "peak": fp32_peak_tflops,
                            "unit": "TFLOP/s", "frac": ach / fp32_peak_tflops, "work": fl}
        else:
            b = bytes_per.get(name, 0)
            ach = b / (ms * 1e-3) / 1e9
            stages[name] = {"ms": ms, "bound": "hbm", "achieved": ach, "peak": hbm, "unit": "GB/s",
                            "frac": ach / hbm, "work": b}
    for name, lim in STAGE_LIMITS.items():
        if name in stages:
            stages[name]["limit"] = lim
    dom = max(stages, key=lambda k: stages[k]["ms"])
    d = dict(stages[dom])
    traffic = kernel_traffic(dom, per_step.get("views", 0))
    timed = (timed_stage_ms or {}).get(dom)
    if timed and timed["calls"] > 0 and timed["ms"] > 0.0:
        ms = timed["ms"] / timed["calls"]
        d["achieved"] = d["work"] / (ms * 1e-3) / (1e12 if d["unit"] == "TFLOP/s" else 1e9)
        d["frac"] = d["achieved"] / d["peak"]
        d["ms"] = ms
    roof = {"kernel": dom, "bound": d["bound"], "achieved": round(d["achieved"], 3), "peak": d["peak"],
            "unit": d["unit"], "frac": round(d["frac"], 4), "traffic": traffic,
            "ms_per_launch_set": round(d["ms"], 4),
            "traffic_note": "DRAM bytes per launch set from an ncu capture of the same kernel source on 4 views, "
                            "scaled to the launch set's views (null when the source changed)",
            "timing": "CUDA events around the kernel's launches inside the timed region, on its stream",
            "peak_source": f"{peaks['source']} ({'hbm_gbs' if d['bound'] == 'hbm' else 'SMs x 128 FP32 lanes x 2 x median SM clock'})",
            "share_of_frame": round(d["ms"] / max(1e-9, sum(s['ms'] for s in stages.values())), 4)}
    return roof, {k: {kk: (round(vv, 4) if isinstance(vv, float) else vv) for kk, vv in v.items()}
                  for k, v in stages.items()}


# ---------------------------------------------------------------- GPU arm


def aggregate_over_ranks(elapsed_ms: float, frames: int, world: int, device=None) -> tuple[float, int]:
    """Whole-job timing: the slowest rank's time and every rank's frames
    (ranks render independent replicas; this is the only collective)."""
    if world <= 1:
        return float(elapsed_ms), int(frames)
    import torch
    t = torch.tensor([float(elapsed_ms)], dtype=torch.float64, device=device)
    n = torch.tensor([int(frames)], dtype=torch.int64, device=device)
    torch.distributed.all_reduce(t, op=torch.distributed.ReduceOp.MAX)
    torch.distributed.all_reduce(n, op=torch.distributed.ReduceOp.SUM)
    return float(t.item()), int(n.item())


def run_gpu(args, rank: int, world: int, local_rank: int) -> dict | None:
    import torch
    import paper_2605_08699_b300 as tg
    torch.cuda.set_device(local_rank)
    dev = torch.device("cuda", local_rank)
    tg.load_library()
    W, H, V = args.width, args.height, args.batch
    scene = synth.config_scene(3, n=args.gaussians)
    K = synth.default_intrinsics(W, H)
    trajs = [synth.config_trajectory(3, i + 1000 * rank) for i in range(V)]
    h16 = tg.scene_from(scene, storage=tg.STORAGE_FP16)
    h32 = tg.scene_from(scene, storage=tg.STORAGE_FP32)
    stream = torch.cuda.Stream(device=dev)
    outs = [torch.empty((H, W, 4), dtype=torch.uint8, device=dev) for _ in range(V)]

    def step(s, handle=h16, o=outs):
        poses = [trajs[v][(s * 7 + v) % len(trajs[v])] for v in range(V)]
        tg.render_batch(handle, poses, [K] * V, [W] * V, [H] * V, o, stream=stream)

    # the timed steps: asynchronous launch sets, the next one queued before the previous one is
    # waited on (double-buffered outputs), so host work between launch sets overlaps the GPU
    outs_b = [torch.empty((H, W, 4), dtype=torch.uint8, device=dev) for _ in range(V)]

    def run_async(first, n):
        prev = None
        for s in range(first, first + n):
            poses = [trajs[v][(s * 7 + v) % len(trajs[v])] for v in range(V)]
            t = tg.render_batch_async(h16, poses, [K] * V, [W] * V, [H] * V, outs if s % 2 == 0 else outs_b,
                                      stream=stream)
            if prev is not None:
                prev.wait()
            prev = t
        if prev is not None:
            prev.wait()

    # the dominant kernel's launches are timed with events inside the timed region; the other
    # stages are timed in a separate untimed pass (each timed stage adds graph nodes)
    tg.profile_stages(["blend"])
    if args.schedule:
        tg.set_schedule(*(int(x) for x in args.schedule.split(",")))
    if not args.no_autotune and not args.schedule:
        # untimed: pick the sliced schedule for this launch-set shape (with the blend events on, as
        # timed), then for the smaller launch sets the other arms form: the server's partial batches
        # of 4 and 2 views, and single views (the plain FP32 arm renders one request at a time, on
        # its own scene).  Each tunes its own launch-set class; the smallest goes last, since a
        # larger one's views-per-set pass may also set a smaller class.
        for m in sorted({V, 4, 2, 1}, reverse=True):
            if m > V:
                continue
            sets = [[trajs[v][(s * 7 + v + 150) % len(trajs[v])] for v in range(m)] for s in range(8)]
            tg.autotune(h32 if m == 1 else h16, sets, [K] * m, [W] * m, [H] * m, outs[:m], iters=4)
    schedule = tg.get_schedule(V)
    schedules = {str(n): tg.get_schedule(n) for n in sorted({1, 2, 4, V})}
    for s in range(args.warmup):
        step(s)
    run_async(0, max(4, args.warmup))   # both in-flight contexts capture their launch sets
    torch.cuda.synchronize()

    # per-step workload (untimed): one launch set of the same kind as a timed step
    st0 = tg.render_batch(h16, [trajs[v][(args.warmup * 7 + v) % len(trajs[v])] for v in range(V)], [K] * V,
                          [W] * V, [H] * V, outs, stream=stream, sort_mode=tg.SORT_SLICED)
    TX, TY = (W + 15) // 16, (H + 15) // 16
    per_step = {"pairs": st0["n_pairs"], "kept": st0["n_visible"], "evals": st0["blend_evals"],
                "fetched": st0["blend_fetched"], "contribs": st0["blend_contribs"], "sort_passes": st0["sort_passes"],
                "depth_passes": st0["depth_sort_passes"], "depth_near": st0["depth_sort_near"],
                # rectangles travel compact (with their entry id, no value stream) when every view
                # has at most 127 x 127 tiles and there are at most 16 views
                "compact_rect": int(V <= 16 and W <= 127 * 16 and H <= 127 * 16),
                "entries": V * scene.n, "gaussians": scene.n, "attr_bytes": 124, "tiles": V * TX * TY, "views": V,
                "slices": schedule["n_slices"]}

    # ---- timed region: device outputs, CUDA events on the launching stream
    tg.profile_read(reset=True)
    clk = ClockSampler(local_rank)
    clk.start()
    time.sleep(0.3)
    launches0 = tg.kernel_launches()
    rerenders0 = tg.exact_rerenders()
    if world > 1:
        torch.distributed.barrier()
    torch.cuda.synchronize()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    step_ms_host = []
    e0.record(stream)
    prev = None
    for s in range(args.steps):
        poses = [trajs[v][((args.warmup + s) * 7 + v) % len(trajs[v])] for v in range(V)]
        t = tg.render_batch_async(h16, poses, [K] * V, [W] * V, [H] * V, outs if s % 2 == 0 else outs_b,
                                  stream=stream)
        if prev is not None:
            prev.wait()
        prev = t
    prev.wait()
    e1.record(stream)
    torch.cuda.synchronize()
    if world > 1:
        torch.distributed.barrier()
    elapsed_ms = e0.elapsed_time(e1)
    launches = tg.kernel_launches() - launches0
    rerenders = tg.exact_rerenders() - rerenders0
    clocks = clk.stop()
    timed_stage_ms = tg.profile_read(reset=True)
    elapsed_ms, frames = aggregate_over_ranks(elapsed_ms, V * args.steps, world, dev)
    value = frames / (elapsed_ms * 1e-3)

    # ---- latency (untimed): one synchronous launch set at a time, submit to frames complete
    for s in range(args.steps):
        t0 = time.perf_counter()
        step(args.warmup + s)
        step_ms_host.append((time.perf_counter() - t0) * 1e3)

    # ---- stage table (untimed): the same launch sets with every stage's events on
    tg.profile_enable(True)
    for s in range(2):
        step(args.warmup + s)
    torch.cuda.synchronize()
    tg.profile_read(reset=True)
    for s in range(args.steps):
        step(args.warmup + s)
    torch.cuda.synchronize()
    stage_ms = tg.profile_read(reset=True)
    tg.profile_enable(False)

    # ---- two launch sets in flight (two host threads, two streams, as the server's two slots)
    concurrent = None
    if args.inflight > 1:
        import threading as _th
        K2 = args.inflight
        streams = [stream] + [torch.cuda.Stream(device=dev) for _ in range(K2 - 1)]
        outs_k = [outs] + [[torch.empty((H, W, 4), dtype=torch.uint8, device=dev) for _ in range(V)]
                           for _ in range(K2 - 1)]

        def worker(k, n_steps, base):
            torch.cuda.set_device(local_rank)
            for s in range(n_steps):
                poses = [trajs[v][((base + s * K2 + k) * 7 + v) % len(trajs[v])] for v in range(V)]
                tg.render_batch(h16, poses, [K] * V, [W] * V, [H] * V, outs_k[k], stream=streams[k])

        for k in range(K2):   # warm-up of every stream's context and graph
            worker(k, 3, 0)
        torch.cuda.synchronize()
        c0, c1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        c0.record(streams[0])
        for k in range(1, K2):
            streams[k].wait_event(c0)
        n_each = max(1, args.steps)
        ths = [_th.Thread(target=worker, args=(k, n_each, 100)) for k in range(K2)]
        for t in ths:
            t.start()
        for t in ths:
            t.join()
        for k in range(1, K2):
            ev = torch.cuda.Event()
            ev.record(streams[k])
            streams[0].wait_event(ev)
        c1.record(streams[0])
        torch.cuda.synchronize()
        cms = c0.elapsed_time(c1)
        concurrent = {"launch_sets_in_flight": K2, "frames": V * n_each * K2, "ms": round(cms, 3),
                      "frames_per_s": round(V * n_each * K2 / (cms * 1e-3), 2),
                      "note": "each host thread renders its own launch sets on its own stream; "
                              "events on stream 0 after it waited for the others"}

        # one host thread, asynchronous launch sets with no caller stream: each
        # outstanding ticket's launch set runs on its own context's stream, so the
        # queued one overlaps the current one (host wall clock, synchronized)
        def run_own(first, n):
            prev = None
            for s in range(first, first + n):
                poses = [trajs[v][(s * 7 + v) % len(trajs[v])] for v in range(V)]
                t = tg.render_batch_async(h16, poses, [K] * V, [W] * V, [H] * V, outs if s % 2 == 0 else outs_b)
                if prev is not None:
                    prev.wait()
                prev = t
            prev.wait()

        run_own(200, 4)
        torch.cuda.synchronize()
        h0 = time.perf_counter()
        run_own(210, args.steps)
        torch.cuda.synchronize()
        own_ms = (time.perf_counter() - h0) * 1e3
        concurrent["own_streams"] = {
            "frames": V * args.steps, "ms": round(own_ms, 3),
            "frames_per_s": round(V * args.steps / (own_ms * 1e-3), 2),
            "note": "tigas_render_batch_async with no caller stream (each ticket's launch set on its "
                    "context's own stream, the next queued, one host thread); host wall clock around "
                    "the synchronized loop"}

    # ---- end to end: pinned host outputs (double-buffered), copies inside the timed region
    houts = [[torch.empty((H, W, 4), dtype=torch.uint8).pin_memory() for _ in range(V)] for _ in range(2)]

    def run_e2e(first, n):
        prev = None
        for s in range(first, first + n):
            poses = [trajs[v][(s * 7 + v) % len(trajs[v])] for v in range(V)]
            t = tg.render_batch_async(h16, poses, [K] * V, [W] * V, [H] * V, houts[s % 2], stream=stream)
            if prev is not None:
                prev.wait()
            prev = t
        prev.wait()

    run_e2e(0, 4)
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    run_e2e(args.warmup, args.steps)
    e2e_s = time.perf_counter() - t0
    e2e_ms, e2e_frames = aggregate_over_ranks(e2e_s * 1e3, V * args.steps, world, dev)
    e2e = {"value": e2e_frames / (e2e_ms * 1e-3), "unit": "frames/s",
           "h2d_bytes_per_step": V * (40 + 32 + 8 + 8), "d2h_bytes_per_step": V * W * H * 4}

    # ---- plain FP32 single-request path, one frame at a time
    lat32 = []
    n32 = args.plain_frames
    out1 = outs[0]
    for i in range(3):
        tg.render_ex(h32, trajs[0][i], K, W, H, out_rgba8=out1, stats=False)
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    for i in range(n32):
        ta = time.perf_counter()
        tg.render_ex(h32, trajs[i % V][(i * 7) % 300], K, W, H, out_rgba8=out1, stats=False)
        lat32.append((time.perf_counter() - ta) * 1e3)
    plain_s = time.perf_counter() - t0
    plain = {"frames_per_s": n32 / plain_s, "latency_ms_p50": float(np.percentile(lat32, 50)),
             "latency_ms_p99": float(np.percentile(lat32, 99)), "frames": n32, "storage": "fp32",
             "path": "tigas_render_ex, one request at a time"}

    configs = None if args.no_configs else run_configs(tg, torch, dev, stream, h16, h32, args)

    # ---- batching workload: 32 views of mixed ABR levels in one launch set
    batching = None
    if not args.no_serving:
        Vb = 32
        lv = [synth.ABR_LEVELS[v % 6] for v in range(Vb)]
        kb = [synth.default_intrinsics(w, h) for w, h in lv]
        tb = [synth.config_trajectory(4, v + 1000 * rank) for v in range(Vb)]
        ob = [torch.empty((h, w, 4), dtype=torch.uint8, device=dev) for w, h in lv]

        def bstep(s):
            tg.render_batch(h16, [tb[v][(s * 5 + v) % 300] for v in range(Vb)], kb, [w for w, _ in lv],
                            [h for _, h in lv], ob, stream=stream)
        for s in range(4):
            bstep(s)
        torch.cuda.synchronize()
        b0, b1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        nb = max(5, args.steps // 2)
        b0.record(stream)
        for s in range(nb):
            bstep(4 + s)
        b1.record(stream)
        torch.cuda.synchronize()
        bms = b0.elapsed_time(b1) / nb
        batching = {"views": Vb, "levels": "6 ABR levels x 1920x1080, uniform mix", "storage": "fp16",
                    "ms_per_launch_set": round(bms, 3), "frames_per_s": round(Vb / bms * 1e3, 1),
                    "megapixels_per_s": round(sum(w * h for w, h in lv) / bms * 1e-3, 1)}

    # ---- frame encoder after the blend: JPEG of the step's frames (device in, device out)
    jpeg = None
    if not args.no_serving:
        jbuf = torch.empty(8 << 20, dtype=torch.uint8, device=dev)
        for q in (90, 65):
            sizes = []
            for o in outs[:2]:
                tg.jpeg_encode(o, q, restart_mcus=2, out=jbuf, stream=stream)
            torch.cuda.synchronize()
            j0, j1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            j0.record(stream)
            for o in outs:
                sizes.append(tg.jpeg_encode(o, q, restart_mcus=2, out=jbuf, stream=stream))
            j1.record(stream)
            torch.cuda.synchronize()
            jms = j0.elapsed_time(j1) / len(outs)
            key = f"quality_{q}"
            jpeg = jpeg or {"resolution": f"{W}x{H}", "restart_mcus": 2,
                            "note": "tigas_jpeg_encode of each rendered frame, device buffers, synchronous calls"}
            jpeg[key] = {"ms_per_frame": round(jms, 4), "frames_per_s": round(1e3 / jms, 1),
                         "kbytes_mean": round(float(np.mean(sizes)) / 1024, 1),
                         "input_gbs": round(W * H * 4 / (jms * 1e-3) / 1e9, 1)}

    # ---- the paper's default colour model: SH degree 0 (same scene, DC terms only)
    sh0 = None
    if not args.no_serving:
        import dataclasses
        h0 = tg.scene_from(dataclasses.replace(scene, sh_degree=0), storage=tg.STORAGE_FP16)
        try:
            def step0(s):
                tg.render_batch(h0, [trajs[v][(s * 7 + v) % len(trajs[v])] for v in range(V)], [K] * V, [W] * V,
                                [H] * V, outs, stream=stream)
            for s in range(4):
                step0(s)
            torch.cuda.synchronize()
            z0, z1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            n0 = max(5, args.steps // 2)
            z0.record(stream)
            for s in range(n0):
                step0(4 + s)
            z1.record(stream)
            torch.cuda.synchronize()
            sh0 = {"frames_per_s": round(V * n0 / (z0.elapsed_time(z1) * 1e-3), 2), "sh_degree": 0,
                   "note": "same scene and views, colour from the degree-0 term only (the paper's default)"}
        finally:
            h0.free()

    # ---- model loading (3DGS PLY of the same scene) and post-session quality evaluation
    models = quality = None
    if not args.no_serving:
        models = run_model_load(tg, scene)
        quality = run_quality(tg, torch, dev, h16, outs, stream, W, H)

    # ---- served FP16: request server, closed-loop clients
    serving = None
    if not args.no_serving:
        serving = run_serving(tg, torch, dev, h16, K, W, H, trajs, args)
    trace = None
    if not args.no_serving and args.trace_seconds > 0:
        trace = run_serving_trace(tg, torch, dev, args)

    res = {"schedule": schedule, "schedules": schedules, "rerenders": rerenders, "concurrent": concurrent, "value": value, "elapsed_ms": elapsed_ms, "frames": frames, "per_step": per_step, "stage_ms": stage_ms,
           "timed_stage_ms": timed_stage_ms,
           "clocks": clocks, "launches": launches, "e2e": e2e, "plain_fp32": plain, "serving": serving, "trace": trace,
           "configs": configs,
           "batching": batching, "sh0": sh0, "jpeg": jpeg, "models": models, "quality": quality,
           "step_ms_host": step_ms_host, "scene": scene}
    h16.free()
    h32.free()
    return res


def run_configs(tg, torch, dev, stream, h16_3m, h32_3m, args) -> dict:
    """Frames/s of every workload configuration besides the headline one, on
    device outputs with CUDA events on the launching stream, after warm-up:
    single requests (tigas_render_ex one at a time, uninstrumented kernels)
    and asynchronous launch sets of 8 views of the same resolution (the next
    one queued before the previous one is waited on)."""
    n = args.config_frames
    ev = [torch.cuda.Event(enable_timing=True) for _ in range(2)]

    def single(h, poses, W, H):
        K = synth.default_intrinsics(W, H)
        o = torch.empty((H, W, 4), dtype=torch.uint8, device=dev)
        for p in poses[:3]:
            tg.render_ex(h, p, K, W, H, out_rgba8=o, stream=stream, stats=False)
        torch.cuda.synchronize()
        ev[0].record(stream)
        for i in range(n):
            tg.render_ex(h, poses[(3 + i) % len(poses)], K, W, H, out_rgba8=o, stream=stream, stats=False)
        ev[1].record(stream)
        torch.cuda.synchronize()
        return round(n / (ev[0].elapsed_time(ev[1]) * 1e-3), 1)

    def batched(h, poses, W, H, V=8):
        K = synth.default_intrinsics(W, H)
        bufs = [[torch.empty((H, W, 4), dtype=torch.uint8, device=dev) for _ in range(V)] for _ in range(2)]
        sets = max(2, n // V)

        def go(first, m):
            prev = None
            for s in range(first, first + m):
                ps = [poses[(s * V + v) % len(poses)] for v in range(V)]
                t = tg.render_batch_async(h, ps, [K] * V, [W] * V, [H] * V, bufs[s % 2], stream=stream)
                if prev is not None:
                    prev.wait()
                prev = t
            prev.wait()
        go(0, 4)   # first appearance, exact render and capture, replays
        torch.cuda.synchronize()
        ev[0].record(stream)
        go(4, sets)
        ev[1].record(stream)
        torch.cuda.synchronize()
        return round(V * sets / (ev[0].elapsed_time(ev[1]) * 1e-3), 1)

    out = {"note": "frames/s per configuration: single = tigas_render_ex one request at a time; batched_8 = "
                   "asynchronous launch sets of 8 views (tigas_render_batch_async); device outputs, CUDA events"}
    s1 = synth.config_scene(1)
    tr1 = synth.config_trajectory(1)
    with tg.scene_from(s1, storage=tg.STORAGE_FP32) as h:
        out["config1_100k_320x240_fp32"] = {"single": single(h, tr1, 320, 240), "batched_8": batched(h, tr1, 320, 240)}
    s2 = synth.config_scene(2)
    tr2 = synth.config_trajectory(2)
    with tg.scene_from(s2, storage=tg.STORAGE_FP32) as h:
        for W, H in ((1280, 720), (1920, 1080)):
            out[f"config2_1M_{W}x{H}_fp32"] = {"single": single(h, tr2, W, H), "batched_8": batched(h, tr2, W, H)}
    tr3 = synth.config_trajectory(3)
    lv = {}
    for W, H in synth.ABR_LEVELS:
        lv[f"{W}x{H}"] = {"fp16": {"single": single(h16_3m, tr3, W, H), "batched_8": batched(h16_3m, tr3, W, H)},
                          "fp32": {"single": single(h32_3m, tr3, W, H), "batched_8": batched(h32_3m, tr3, W, H)}}
    out["config3_3M_abr_levels"] = lv
    return out


def run_model_load(tg, scene) -> dict:
    """Write the scene as a binary 3DGS PLY, then time tigas_scene_load_ply
    (header parse, streamed upload, de-interleave, activate and pack) and a
    registry's first (loading) and second (shared) acquire.  Wall-clock; the
    file is in the page cache, so this is the host-to-HBM path, not the disk."""
    import tempfile
    from synth import ply as sply
    with tempfile.TemporaryDirectory() as d:
        path = os.path.join(d, "scene.ply")
        sply.write_ply(path, scene)
        size = os.path.getsize(path)
        times = []
        for _ in range(3):
            t0 = time.perf_counter()
            h = tg.scene_load_ply(path, tg.STORAGE_FP16)
            times.append(time.perf_counter() - t0)
            h.free()
        with tg.Registry(d, storage=tg.STORAGE_FP16, idle_timeout_s=60.0) as reg:
            t0 = time.perf_counter()
            a = reg.acquire("scene")
            t1 = time.perf_counter()
            b = reg.acquire("scene")
            t2 = time.perf_counter()
            a.free()
            b.free()
    best = min(times)
    return {"gaussians": scene.n, "file_mb": round(size / 2**20, 1), "format": "binary_little_endian, SH degree 3",
            "load_s": round(best, 4), "file_gbs": round(size / best / 1e9, 2),
            "registry_first_acquire_s": round(t1 - t0, 4), "registry_shared_acquire_ms": round((t2 - t1) * 1e3, 4),
            "note": "best of 3 tigas_scene_load_ply, page-cached file, FP16 storage"}


def run_quality(tg, torch, dev, handle, outs, stream, W, H) -> dict:
    """SSIM/PSNR and resample kernels at the frame size, and a replay of a
    Table-1 session log (GT at 1280x720, JPEG at the logged profiles)."""
    from paper_2605_08699_b300 import replay as rp
    low = torch.empty((H // 4, W // 4, 4), dtype=torch.uint8, device=dev)
    tg.render_batch(handle, [synth.BASE_POSE], [synth.default_intrinsics(W // 4, H // 4)], [W // 4], [H // 4], [low],
                    stream=stream)
    up = torch.empty_like(outs[0])
    out = {}
    for name, fn in (("resample", lambda: tg.resample_rgba8(low, W, H, out=up, stream=stream)),
                     ("ssim_psnr", lambda: tg.image_quality(outs[0], up, stream=stream))):
        for _ in range(3):
            fn()
        torch.cuda.synchronize()
        n = 20
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        for _ in range(n):
            fn()
        e1.record(stream)
        torch.cuda.synchronize()
        out[name + "_ms"] = round(e0.elapsed_time(e1) / n, 4)
    q = tg.image_quality(outs[0], up)
    out["ssim_1080p_vs_quarter_res"] = round(q["ssim"], 4)
    out["psnr_1080p_vs_quarter_res"] = round(q["psnr"], 2)
    log = synth.pose_log(n_frames=64)
    recs = [rp.LogRecord(r.i, (r.pose.azimuth, r.pose.elevation, tuple(r.pose.t)),
                         (r.intr.fx, r.intr.fy, r.intr.cx, r.intr.cy), r.width, r.height, r.quality) for r in log]
    rp.replay(handle, recs[:8], (1280, 720))
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    frames = rp.replay(handle, recs, (1280, 720), stride=1)
    dt = time.perf_counter() - t0
    out["replay"] = {"frames": len(frames), "frames_per_s": round(len(frames) / dt, 1),
                     "ssim_mean": round(float(np.mean([f.ssim for f in frames])), 4),
                     "psnr_mean_db_lossy": round(float(np.mean([f.psnr for f in frames if math.isfinite(f.psnr)]
                                                                or [math.inf])), 2),
                     "frames_at_display_size": sum(1 for f in frames if not math.isfinite(f.psnr)),
                     "note": "per frame: render at the logged profile + JPEG, GT render 1280x720, resample, SSIM/PSNR; "
                             "batches of 8, no files written; PSNR mean over frames whose profile is below the "
                             "display size (the others equal their GT)"}
    out["note"] = "ms per call with CUDA events on the launching stream (synchronous calls), 1920x1080 RGBA8 device frames"
    return out


def run_serving(tg, torch, dev, h16, K, W, H, trajs, args) -> dict:
    """Closed loop: C clients each keep one 1080p request in flight; the server
    batches whatever is queued into fused launch sets as slots free up."""
    C = args.clients
    bufs = [torch.empty((H, W, 4), dtype=torch.uint8, device=dev) for _ in range(C)]
    lat, n_done = [], 0
    with tg.Server(max_batch=args.serve_batch, max_inflight=args.serve_inflight) as srv:
        nxt = [0] * C
        for c in range(C):
            srv.submit(h16, trajs[c % len(trajs)][0], K, W, H, bufs[c], client_id=c)
        t_end = time.perf_counter() + args.serve_seconds
        t0 = time.perf_counter()
        warm = 2 * C
        while True:
            for comp in srv.poll(256, timeout_us=200_000):
                c = comp.client_id
                if comp.status == 0:
                    n_done += 1
                    if n_done > warm:
                        lat.append((comp.done_us - comp.submit_us) * 1e-3)
                    if n_done == warm:
                        t0 = time.perf_counter()
                if time.perf_counter() < t_end:
                    nxt[c] += 1
                    srv.submit(h16, trajs[c % len(trajs)][(nxt[c] * 3) % 300], K, W, H, bufs[c], client_id=c)
            if time.perf_counter() >= t_end:
                break
        t1 = time.perf_counter()
        # drain
        while True:
            got = srv.poll(256, timeout_us=500_000)
            if not got:
                break
    measured = len(lat)
    return {"frames_per_s": measured / max(1e-9, t1 - t0), "latency_ms_p50": float(np.percentile(lat, 50)),
            "latency_ms_p99": float(np.percentile(lat, 99)), "frames": measured, "clients": C,
            "max_batch": args.serve_batch, "slots": args.serve_inflight, "storage": "fp16",
            "latency": "submit to frame complete in the client's buffer"}


def _thin(tr, keep: np.ndarray):
    """The trace restricted to the requests where keep is true (thinning a
    Poisson process by an independent coin keeps it Poisson)."""
    return synth.ServingTrace(t=tr.t[keep], client=tr.client[keep], scene=tr.scene[keep],
                              pose_index=tr.pose_index[keep], bw=tr.bw[keep], rates_hz=tr.rates_hz,
                              seconds=tr.seconds, n_scenes=tr.n_scenes)


def run_serving_trace(tg, torch, dev, args) -> dict:
    """Open-loop multi-client trace through the request server, in two arms:
    served FP16 (batched launch sets, overlapping slots) and plain FP32 (one
    request at a time, same server code with max_batch = max_inflight = 1).

    Clients request at fixed Poisson rates; client c uses scene c mod 4 of
    1M/2M/3M/6M Gaussians; each request's resolution comes from the client's
    Latency ABR over its simulated download throughput, so both arms render
    the same requests.  A queued request of a client is superseded by its
    next one (latest pose wins).

    The full trace (64 clients at 60-90 Hz) overloads both arms.  The sweep
    replays the same trace thinned to offered loads of 25, 50, 90 and 150 %
    of the plain arm's measured capacity (its frame rate on the full trace),
    so that each arm is compared where the plain one keeps up as well as
    where it does not.  The served arm's policy needs no tuning for low load:
    it has no batch window, so a free slot takes whatever is queued (up to
    max_batch), which at low load is one request."""
    from paper_2605_08699_b300.abr import assign_levels

    tr_full = synth.serving_trace(n_clients=args.trace_clients, seconds=args.trace_seconds)
    levels = synth.ABR_LEVELS
    lvl_full = assign_levels(tr_full.client, tr_full.bw, levels)
    intr = [synth.default_intrinsics(w, h) for w, h in levels]
    n_pose = int(math.ceil(args.trace_seconds * 90)) + 2
    trajs = [synth.trajectory(synth.BASE_SEED + 600 + c, n_poses=n_pose) for c in range(args.trace_clients)]
    sizes = [int(x) for x in args.trace_scenes.split(",")]
    raw = [synth.make_scene(n, seed=synth.BASE_SEED + 5 + 10 * i) for i, n in enumerate(sizes)]
    W1, H1 = levels[-1]
    bufs = [[torch.empty(W1 * H1 * 4, dtype=torch.uint8, device=dev) for _ in range(3)]
            for _ in range(args.trace_clients)]
    warm = min(1.0, 0.2 * tr_full.seconds)   # of the full trace (reported)

    def replay(tr, lvl, handles, max_batch, max_inflight):
        warm = min(1.0, 0.2 * tr.seconds)
        lat, wait, px, n_ok, n_sup, n_err, n_in = [], [], 0, 0, 0, 0, 0
        lag = []
        rot = [0] * args.trace_clients
        R, i, outstanding = tr.t.size, 0, 0
        with tg.Server(max_batch=max_batch, max_inflight=max_inflight) as srv:
            t0 = time.perf_counter()
            while True:
                now = time.perf_counter() - t0
                while i < R and tr.t[i] <= now:
                    c, l = int(tr.client[i]), int(lvl[i])
                    w, h = levels[l]
                    b = bufs[c][rot[c] % 3]
                    rot[c] += 1
                    srv.submit(handles[int(tr.scene[i])], trajs[c][int(tr.pose_index[i])], intr[l], w, h, b,
                               client_id=c)
                    if tr.t[i] >= warm:
                        lag.append(time.perf_counter() - t0 - tr.t[i])
                    i += 1
                    outstanding += 1
                dt = (tr.t[i] - (time.perf_counter() - t0)) if i < R else 0.2
                for comp in srv.poll(1024, timeout_us=max(0, int(dt * 1e6)) if dt > 2e-4 else 0):
                    outstanding -= 1
                    if comp.submit_us * 1e-6 - t0 < warm:
                        continue
                    n_in += 1
                    if comp.status == 0:
                        n_ok += 1
                        px += comp.width * comp.height
                        lat.append((comp.done_us - comp.submit_us) * 1e-3)
                        wait.append((comp.admit_us - comp.submit_us) * 1e-3)
                    elif comp.status == 4:
                        n_sup += 1
                    else:
                        n_err += 1
                if i >= R and outstanding == 0:
                    break
        T = tr.seconds - warm
        lat_a = np.array(lat) if lat else np.array([float("nan")])
        # superseded requests counted as missed (infinite latency): the p99 over all
        # requests is finite only while at most 1 % of them were superseded
        missed = n_sup / max(1, n_in)
        p99_all = None
        if lat and missed <= 0.01:
            p99_all = float(np.percentile(np.concatenate([lat_a, np.full(n_sup, np.inf)]), 99))
        return {"frames_per_s": n_ok / T, "megapixels_per_s": px / T / 1e6,
                "latency_ms_p50": float(np.percentile(lat_a, 50)), "latency_ms_p99": float(np.percentile(lat_a, 99)),
                "queue_ms_p50": float(np.percentile(wait, 50)) if wait else None,
                "frames": n_ok, "superseded": n_sup, "errors": n_err, "missed_frac": missed,
                "latency_ms_p99_superseded_as_missed": p99_all,
                "submit_lag_ms_p99": float(np.percentile(lag, 99) * 1e3) if lag else None}

    out = {"trace": f"{args.trace_clients} clients, Poisson arrivals at U[60,90] Hz each, {tr_full.seconds:g} s "
                    f"(first {warm:g} s not counted), scenes {args.trace_scenes} Gaussians round-robin, "
                    "resolutions from each client's Latency ABR (ladder f x 1920x1080, 0.2 B/px, "
                    "bandwidth redrawn every second, ln N(ln 22.4 Mbit/s, 0.75) clipped to [5, 100])",
           "requests": int(tr_full.t.size), "offered_per_s": tr_full.t.size / tr_full.seconds,
           "level_mix": {f"{w}x{h}": int(np.sum(lvl_full == k)) for k, (w, h) in enumerate(levels)},
           "latency": "submit to frame complete in the client's buffer (server clock)"}
    h16 = [tg.scene_from(r, storage=tg.STORAGE_FP16) for r in raw]
    h32 = [tg.scene_from(r, storage=tg.STORAGE_FP32) for r in raw]
    try:
        out["served_fp16"] = dict(replay(tr_full, lvl_full, h16, args.serve_batch, args.serve_inflight),
                                  max_batch=args.serve_batch, slots=args.serve_inflight, storage="fp16")
        out["plain_fp32"] = dict(replay(tr_full, lvl_full, h32, 1, 1), max_batch=1, slots=1, storage="fp32")
        cap = out["plain_fp32"]["frames_per_s"]
        sweep = []
        # one shorter trace for every load point and both arms, its levels assigned once
        tr_sw = synth.serving_trace(n_clients=args.trace_clients, seconds=min(args.sweep_seconds, args.trace_seconds))
        lvl_sw = assign_levels(tr_sw.client, tr_sw.bw, levels)
        offered_sw = tr_sw.t.size / tr_sw.seconds
        u = synth.uniforms(synth.BASE_SEED + 700, 1, tr_sw.t.size)
        for frac in (0.25, 0.5, 0.9, 1.5):
            keep = u < min(1.0, frac * cap / offered_sw)
            tr, lvl = _thin(tr_sw, keep), lvl_sw[keep]
            served = replay(tr, lvl, h16, args.serve_batch, args.serve_inflight)
            plain = replay(tr, lvl, h32, 1, 1)
            sustains = plain["missed_frac"] <= 0.01 and plain["errors"] == 0
            sweep.append({
                "load_of_plain_capacity": frac, "offered_per_s": tr.t.size / tr.seconds,
                "served_fp16": served, "plain_fp32": plain,
                "plain_sustains_load": sustains,
                "served_frames_per_s_ge_plain": served["frames_per_s"] >= plain["frames_per_s"] * 0.995,
                "served_p99_le_plain": served["latency_ms_p99"] <= plain["latency_ms_p99"],
                "target_holds": bool(sustains and served["frames_per_s"] >= plain["frames_per_s"] * 0.995
                                     and served["latency_ms_p99"] <= plain["latency_ms_p99"]),
            })
        out["sweep"] = sweep
        out["sweep_note"] = (f"one {tr_sw.seconds:g} s trace of the same generator, thinned to each offered load "
                             "(capacity: the plain arm's frame rate on the full trace); target_holds: the plain arm keeps up (<= 1 % superseded) and served "
                             "FP16 has frames/s >= plain (within 0.5 %) and p99 <= plain")
    finally:
        for h in h16 + h32:
            h.free()
    return out


# --------------------------------------------------------------- reference


def run_reference(args) -> dict:
    """The oracle as the reference arm: each step is one whole frame of the
    headline workload (the 3M-Gaussian scene with FP16-rounded attributes at
    1920x1080, a new pose per step), rendered in FP64 on the host cores."""
    scene = synth.config_scene(3, n=args.gaussians)
    poses = synth.config_trajectory(3, 0)
    W, H = args.width, args.height
    times = []
    for s in range(args.warmup + args.steps):
        t = oracle_frame(scene, poses[(s * 7) % 300], W, H)
        if s >= args.warmup:
            times.append(t)
    value = 1.0 / statistics.mean(times)
    line = {"metric": METRIC, "value": value, "unit": "frames/s", "n_gpus": args.gpus, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": statistics.mean(times) * 1e3, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic", "impl": "reference",
            "config": {"workload": WORKLOAD, "gaussians": scene.n, "width": W, "height": H,
                       "storage": "fp16 (positions fp32), as the GPU arm stores them",
                       "parallelism": "host cores (OpenMP)"},
            "cpu_baseline": {"value": value, "unit": "frames/s", "cores": os.cpu_count(), "kind": "oracle",
                             "sample": f"per step one whole {W}x{H} frame in FP64 (preprocess of every Gaussian, "
                                       "every pixel composited)"},
            "e2e": {"value": value, "unit": "frames/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    return line


# -------------------------------------------------------------------- main


def main(argv=None) -> int:
    ap = argparse.ArgumentParser(description=__doc__.split("\n")[0])
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=20)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", choices=["tigas", "reference"], default="tigas")
    ap.add_argument("--batch", type=int, default=8, help="views per fused launch set")
    ap.add_argument("--gaussians", type=int, default=3_000_000)
    ap.add_argument("--width", type=int, default=1920)
    ap.add_argument("--height", type=int, default=1080)
    ap.add_argument("--clients", type=int, default=16)
    ap.add_argument("--serve-batch", type=int, default=8)
    ap.add_argument("--serve-inflight", type=int, default=2)
    ap.add_argument("--serve-seconds", type=float, default=3.0)
    ap.add_argument("--no-serving", action="store_true")
    ap.add_argument("--no-autotune", action="store_true", help="keep the default schedule")
    ap.add_argument("--inflight", type=int, default=2, help="also time this many launch sets in flight (1: skip)")
    ap.add_argument("--schedule", default="", help="fixed schedule 'slices,first_slice_inv,blend_ctas_per_sm"
                                                   "[,blend_batch[,views_per_set]]' "
                                                   "(no autotuning)")
    ap.add_argument("--trace-seconds", type=float, default=10.0, help="open-loop serving trace length (0: skip)")
    ap.add_argument("--trace-clients", type=int, default=64)
    ap.add_argument("--sweep-seconds", type=float, default=4.0, help="trace length of each offered-load point")
    ap.add_argument("--trace-scenes", default="1000000,2000000,3000000,6000000")
    ap.add_argument("--plain-frames", type=int, default=64, help="frames of the plain FP32 single-request path")
    ap.add_argument("--cpu-seconds", type=float, default=15.0)
    ap.add_argument("--config-frames", type=int, default=32, help="frames per configuration line")
    ap.add_argument("--no-configs", action="store_true", help="skip the per-configuration frame rates")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    args = ap.parse_args(argv)
    args.warmup = max(3, args.warmup)

    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    local_rank = int(os.environ.get("LOCAL_RANK", "0"))

    if args.impl == "reference":
        if rank != 0:
            return 0
        print(json.dumps(run_reference(args)), flush=True)
        return 0

    if world > 1:
        import torch
        torch.distributed.init_process_group("nccl", device_id=torch.device("cuda", local_rank))
    r = run_gpu(args, rank, world, local_rank)
    if rank == 0:
        peaks = _peaks()
        roof, stages = roofline(r["stage_ms"], r["per_step"], peaks, r["clocks"], args.steps, r["timed_stage_ms"])
        cpu = None
        if world == 1 and not args.no_cpu_baseline:
            poses = synth.config_trajectory(3, 0)
            cpu = cpu_baseline(r["scene"], [poses[(k * 37) % 300] for k in range(50)], args.width, args.height,
                               args.cpu_seconds)
        steps_ms = r["step_ms_host"]
        line = {
            "metric": METRIC, "value": round(r["value"], 2), "unit": "frames/s", "n_gpus": world,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": round(r["elapsed_ms"] / args.steps, 4),
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f32",
            "data": "synthetic",
            "config": {"workload": WORKLOAD, "gaussians": args.gaussians, "width": args.width, "height": args.height,
                       "views_per_step": args.batch, "storage": "fp16 (positions fp32)", "sh_degree": 3,
                       "path": "tigas_render_batch (fused launch set per step)",
                       "l2": "inputs larger than L2 (126 MB): 384 MB resident scene, 1.2 GB of per-view splat arrays per step",
                       "parallelism": f"replicas x{world}"},
            "latency_ms": {"p50_step": round(float(np.percentile(steps_ms, 50)), 3),
                           "p99_step": round(float(np.percentile(steps_ms, 99)), 3),
                           "note": "host time of one synchronous launch set of views_per_step frames "
                                   "(tigas_render_batch), measured after the timed region"},
            "schedule": dict(r["schedule"], kind="depth-sliced: nearest-first geometric slices, tiles whose "
                                                  "pixels all stopped are dropped", autotuned=not (args.no_autotune or args.schedule),
                             exact_rerenders_timed=r["rerenders"],
                             by_views=r["schedules"]),
            "served_fp16": r["serving"], "plain_fp32": r["plain_fp32"], "serving_trace": r["trace"],
            "configs": r["configs"],
            "batching_32_mixed": r["batching"], "in_flight": r["concurrent"], "sh_degree_0": r["sh0"],
            "jpeg_encode": r["jpeg"], "model_load": r["models"], "quality_eval": r["quality"],
            "roofline": roof, "stages": stages,
            "stages_timing": "every stage's events on, in an untimed pass of the same launch sets after the timed "
                             "region; the timed region records only the dominant kernel's events", "per_step": {k: int(v) for k, v in r["per_step"].items()},
            "cpu_baseline": cpu, "e2e": r["e2e"], "gpu_launches": int(r["launches"]), "clocks": r["clocks"],
        }
        print(json.dumps(line), flush=True)
    if world > 1:
        import torch
        torch.distributed.destroy_process_group()
    return 0


if __name__ == "__main__":
    sys.exit(main())
