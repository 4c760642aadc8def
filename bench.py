#!/usr/bin/env python
"""Benchmark of the densification path on GB300.

Workload (one step): a batch of B distinct 1920x1080 viewpoints, each with
three staggered 128x1024 LiDAR sweeps (about 124k points each after 5%
dropout, about 373k merged), projected with the nearest-depth z-buffer,
densified with the two-stage joint bilateral filter (r=4 at 1/3 resolution,
r=2 at full resolution, sigma_p 5 px, sigma_c 20) and back-projected to
coloured points. Inputs are seeded synthetic scenes (the paper's capture data
is not available). Metric: dense 1080p frames per second.

  value   device time: inputs resident in HBM, L2 flushed (256 MiB write)
          before every step, CUDA events on the launching stream around the
          step's work, summed over K steps.
  e2e     the same frames through the C ABI with pinned HOST buffers:
          host->device copies of points and RGB, and the coloured points and
          their count written by the GPU into pinned host memory, inside the
          timed region (wall clock).

--impl reference times the FP64 CPU oracle (the method's plain definition)
on the host cores, on a bounded sample of the same workload.

Multi-GPU (torchrun): viewpoints are independent (no exchange between
viewpoints in the paper's system), so each rank runs its own batch of views:
weak scaling, no collective on the data path; rank 0 prints the total.
"""
from __future__ import annotations

import argparse
import json
import os
import subprocess
import sys
import threading
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "1080p dense-depth frames/s (3 merged LiDAR scans, two-stage JBF r=4@1/3 + r=2, coloured points)"
UNIT = "frames/s"
# issue slots of one filter tap in each arithmetic form: the last-resort peak model, used only when
# neither the committed nor a live measurement of the instruction rates is available
TAP_INSTR = {"fp32": 10.0, "fp32_expanded": 6.0, "fp32_expanded_pairs": 3.5, "fp32_sparse": 15.0, "fp16_sparse": 18.5}
ALU_PEAKS = os.path.join(ROOT, "profiles", "alu_peaks.json")
STAGES = ((4, 5.0, 20.0), (2, 5.0, 20.0))
L2_FLUSH_BYTES = 256 << 20


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=20)
    ap.add_argument("--warmup", type=int, default=5)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--batch", type=int, default=8, help="viewpoints per step")
    ap.add_argument("--views", type=int, default=8, help="distinct synthetic views generated")
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--no-clocks", action="store_true", help="skip the clock-sampling window (profiling runs)")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--cpu-frames", type=int, default=32, help="frames in the oracle's timed sample")
    ap.add_argument("--cpu-procs", type=int, default=os.cpu_count() or 1,
                    help="oracle worker processes (one single-threaded oracle per host core)")
    ap.add_argument("--no-serve", action="store_true", help="skip the serving measurement")
    ap.add_argument("--no-fp16", action="store_true", help="skip the FP16-form measurement")
    ap.add_argument("--no-live-peaks", action="store_true",
                    help="skip the live instruction-rate microbenchmark (profiling runs: its kernels stay out of "
                         "the launch list; the committed measurement is used)")
    ap.add_argument("--no-configs", action="store_true",
                    help="skip the 320x240 single-stage (FP32, FP16) and uneven 12-view workloads")
    ap.add_argument("--autotune", type=int, default=1, help="1: pick filter kernels on the first batch")
    ap.add_argument("--kernels", default="",
                    help="STAGE1,STAGE2 filter kernels to use instead of tuning (candidate names as in the "
                         "tuning cache, e.g. tma:kp2:nw4:exp,tma:kp4:nw4:exp_pairs); for profiling runs")
    ap.add_argument("--kernel-timing", type=int, default=2,
                    help="events inside the timed steps: 2 around the full-resolution filter only (the "
                         "per-kernel table then comes from a separate untimed pass), 1 around every kernel")
    ap.add_argument("--serve-seconds", type=float, default=60.0,
                    help="duration of the paper-rate serving run (16 viewpoints x 30 fps)")
    return ap.parse_args()


# ---------------------------------------------------------------------------
# inputs
# ---------------------------------------------------------------------------
def _gen(args):
    import scene
    seed, idx, n = args
    v = scene.make_view(seed, res="1080p", scene_kind="room", n_scans=3, beams=128, az_steps=1024,
                        view_index=idx, n_views=n)
    return v


def _gen_mixed(args):
    import scene
    seed, res, idx, n = args
    return scene.make_batch_view(seed, res, idx, n)


def make_mixed_views(n, seed0):
    """Serving viewpoints: mixed 1080p / 720p / 540p, 1-3 sweeps of 64-128 x 512-2048."""
    import concurrent.futures as cf
    import multiprocessing as mp
    res = ["1080p", "720p", "540p"]
    jobs = [(seed0, res[i % 3], i, n) for i in range(n)]
    with cf.ProcessPoolExecutor(max(1, min(n, (os.cpu_count() or 2) - 1, 12)),
                                mp_context=mp.get_context("spawn")) as ex:
        return list(ex.map(_gen_mixed, jobs))


def serve_measure(views, dev, seconds, autotune=1):
    """Frames/s and p50/p99 latency of the serving loop at the paper's load (16 viewpoints x 30 fps,
    Poisson-jittered, ``seconds`` long) and at two saturating loads, in three modes: single-frame
    launches in FP32, continuous batching in FP32 and continuous batching in FP16 (so that the
    effect of batching and the effect of precision are measured apart). Each context owns its
    streams (two batches in flight overlap on the GPU). The loop is a host Python busy-poll, so
    the latencies include its turn time."""
    from paper_2601_01210_gb300 import Densifier
    from paper_2601_01210_gb300.frames import FrameBuffers
    from paper_2601_01210_gb300.serve import ServeLoop, poisson_arrivals
    ring = [[FrameBuffers(v.camera, v.rgb, [(s.xyz, s.lidar_to_world) for s in v.scans], device=dev)
             for _ in range(3)] for v in views]
    frames = [[b.frame for b in r] for r in ring]
    modes = {
        "single_frame_fp32": dict(max_batch=1, batches_in_flight=1, precision=0),
        "batched_fp32": dict(max_batch=16, batches_in_flight=2, precision=0),
        "batched_fp16": dict(max_batch=16, batches_in_flight=2, precision=1),
    }
    # the paper's rate, a load above the single-frame form's capacity, and one above every form's
    # capacity (its frames/s is the form's serving capacity; its latencies are queueing)
    loads = {"paper_rate_30fps": (30.0, seconds), "saturating_1000fps": (1000.0, 2.0),
             "capacity_4000fps": (4000.0, 2.0)}
    out = {}
    for mname, extra in modes.items():
        params = dict(num_stages=2, stages=STAGES, max_inflight=32, launch_policy=0, autotune=autotune,
                      hbm_budget_bytes=4 << 30, **extra)
        with Densifier(params, device=dev.index) as d:
            # warm-up: the first batch tunes the filters and captures every slot's graph; then a
            # saturating burst sends batches of every size through both slots
            ServeLoop(d, frames).run(poisson_arrivals(len(views), 1000.0, 0.2, seed=9), 0.2)
            for lname, (fps, dur) in loads.items():
                arr = poisson_arrivals(len(views), fps, dur, seed=11)
                st = ServeLoop(d, frames).run(arr, dur, drain_s=10.0)
                out[f"{mname}/{lname}"] = dict(st.summary(), batches=d.describe()["batches"])
    return out


def fp16_measure(a, bufs, params, dev, stream, flush_buf, taps2):
    """The same batches in the FP16 form (FP16 guide and weights in the
    full-resolution stage, FP32 sums): device frames/s and the stage-2 kernel."""
    import torch
    from paper_2601_01210_gb300 import Densifier
    p = dict(params, precision=1)
    B = len(bufs)
    with Densifier(p, device=dev.index, stream=stream.cuda_stream) as d:
        def step(k, ev):
            ts = [d.submit(b.frame) for b in bufs]
            flush_buf.fill_(k)
            if ev:
                ev[0].record(stream)
            d.flush(-1)
            if ev:
                ev[1].record(stream)
            for t in ts:
                d.poll(t, -1)

        for k in range(max(3, a.warmup)):
            step(k, None)
        torch.cuda.synchronize()
        d.reset_kernel_times()
        evs = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(a.steps)]
        for k in range(a.steps):
            step(k, evs[k])
        torch.cuda.synchronize()
        ms = sum(s.elapsed_time(e) for s, e in evs)
        kt = d.kernel_times()
        choice = d.describe()
    s2 = kt.get("jbf_stage2", (0.0, 1))
    avg = s2[0] / max(1, s2[1])
    return {"value": B * a.steps / (ms / 1000.0), "unit": UNIT, "ms_per_step": ms / a.steps,
            "jbf_stage2_avg_us": avg, "jbf_stage2_gtap_s": taps2 / (avg * 1e-6) / 1e9 if avg > 0 else None,
            "kernels": {k: round(v[0] / max(1, v[1]), 3) for k, v in kt.items()}, "filter_kernels": choice}


# ---------------------------------------------------------------------------
# the other workloads: 320x240 single stage (FP32 and FP16) and the uneven 12-view batch
# ---------------------------------------------------------------------------
QVGA_STAGES = ((4, 3.0, 20.0),)          # 9x9 window, sigma_p 3 px, sigma_c 20
UNEVEN_RES = ["1080p"] * 4 + ["720p"] * 4 + ["540p"] * 4


def _gen_qvga(seed):
    import scene
    return scene.make_workload("qvga_1scan", seed)


def _gen_uneven(args):
    import scene
    seed, i = args
    return scene.make_batch_view(seed, UNEVEN_RES[i], i, len(UNEVEN_RES))


def make_config_views(n_qvga=16, seed_qvga=1000, seed_uneven=1003):
    """Distinct views of the 320x240 workload and the 12 uneven views (spawn pool, before CUDA)."""
    import concurrent.futures as cf
    import multiprocessing as mp
    with cf.ProcessPoolExecutor(max(1, min(12, (os.cpu_count() or 2) - 1)), mp_context=mp.get_context("spawn")) as ex:
        qvga = list(ex.map(_gen_qvga, [seed_qvga + i for i in range(n_qvga)]))
        uneven = list(ex.map(_gen_uneven, [(seed_uneven, i) for i in range(len(UNEVEN_RES))]))
    return {"qvga": qvga, "uneven": uneven}


EXTRA_CONFIGS = {
    # one viewpoint at 320x240, one 32x256 sweep, single-stage 9x9 window (FP32, and FP16 guide and weights)
    "qvga_1scan_single_stage_fp32": dict(views="qvga", stages=QVGA_STAGES, precision=0, batch=32),
    "qvga_1scan_single_stage_fp16": dict(views="qvga", stages=QVGA_STAGES, precision=1, batch=32),
    # 12 uneven views (4 x 1080p, 4 x 720p, 4 x 540p) in one batched, graph-captured launch sequence, FP16, autotuned
    "uneven_12view_two_stage_fp16": dict(views="uneven", stages=STAGES, precision=1, batch=12),
    # the 1080p three-scan views with the single-stage alternative: one 15x15 window at full resolution
    "1080p_3scan_single_stage_15x15_fp32": dict(views="main", stages=((7, 5.0, 20.0),), precision=0, batch=4),
    # the headline workload with the preprocessing of Sec. 4.1 (afterimage removal against a previous frame
    # in which a block of the image changed; occluded-point removal) and the contour removal of Sec. 5
    "1080p_3scan_two_stage_prepost_fp32": dict(views="main", stages=STAGES, precision=0, batch=8, moved=True,
                                               prepost=dict(occlusion_radius=5, occlusion_margin=0.3,
                                                            motion_threshold=40.0, motion_close_radius=2,
                                                            contour_threshold=0.05)),
}


def moved_frame(view, seed=0):
    """A previous RGB frame of the view in which a block of the image differed (something moved there)."""
    import numpy as np
    rng = np.random.default_rng(seed)
    prev = view.rgb.copy()
    H, W = prev.shape[:2]
    y0, x0 = H // 3, W // 3
    prev[y0:y0 + H // 4, x0:x0 + W // 4] = rng.integers(0, 256, 3, dtype=np.uint8)
    return prev


def config_measure(name, cfg, views, a, dev, stream, flush_buf, tap_peak, hbm):
    """Device frames/s of one workload (same method as the headline: inputs resident, L2 flushed before
    every step, CUDA events around the launch), per-kernel times from a separate pass, the path roofline,
    and the probe outputs (depth, validity) of each distinct view for the CPU leg's error report."""
    import torch
    from paper_2601_01210_gb300 import Densifier
    from paper_2601_01210_gb300.frames import FrameBuffers
    stages, B, ns = cfg["stages"], cfg["batch"], len(cfg["stages"])
    prev = [moved_frame(v, i) for i, v in enumerate(views)] if cfg.get("moved") else [None] * len(views)

    def fb(i, **kw):
        v = views[i]
        return FrameBuffers(v.camera, v.rgb, [(s.xyz, s.lidar_to_world) for s in v.scans], device=dev,
                            num_stages=ns, prev_rgb=prev[i], **kw)

    bufs = [fb(i % len(views)) for i in range(B)]
    # max_batch above the step's frames: the batch leaves at the flush, between the step's events
    params = dict(num_stages=ns, stages=stages, precision=cfg["precision"], max_batch=min(64, 2 * B),
                  max_inflight=max(B, 16),
                  launch_policy=1, timing=2, autotune=a.autotune, batches_in_flight=1,
                  hbm_budget_bytes=max(2 << 30, B * 48 << 20), **cfg.get("prepost", {}))

    def run(d, frames, k, ev=None):
        ts = [d.submit(f.frame) for f in frames]
        flush_buf.fill_(k)
        if ev:
            ev[0].record(stream)
        d.flush(-1)
        if ev:
            ev[1].record(stream)
        for t in ts:
            d.poll(t, -1)

    with Densifier(params, device=dev.index, stream=stream.cuda_stream) as d:
        for k in range(max(3, a.warmup)):
            run(d, bufs, k)
        torch.cuda.synchronize()
        d.reset_kernel_times()
        evs = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(a.steps)]
        for k in range(a.steps):
            run(d, bufs, k, evs[k])
        torch.cuda.synchronize()
        step_ms = [s_.elapsed_time(e_) for s_, e_ in evs]
        choice = d.describe()
        launches = d.kernel_launches()
        probe = [fb(i, debug=True) for i in range(min(len(views), 16))]
        run(d, probe, 0)
        torch.cuda.synchronize()
    with Densifier(dict(params, timing=1), device=dev.index, stream=stream.cuda_stream) as d3:
        for k in range(3 + 10):
            if k == 3:
                torch.cuda.synchronize()
                d3.reset_kernel_times()
            run(d3, bufs, k)
        torch.cuda.synchronize()
        kt = d3.kernel_times()
    ktable = {k: {"avg_us": round(v[0] / max(1, v[1]), 3), "launches": v[1]} for k, v in kt.items()}
    # algorithmic work of one step: the batch cycles through the probed views
    works = [step_work(b, v, single_radius=stages[0][0] if ns == 1 else None, prepost=cfg.get("prepost"))
             for b, v in zip(probe, views)]
    work = {k: sum(works[i % len(works)][k] for i in range(B)) for k in works[0]}
    forms = [st["chosen"].get("form", "fp32") for st in choice["stages"]]
    roof = {k: work[k] / hbm * 1e6 for k in ("prep_compose_clear", "motion_mask", "motion_dilate", "motion_erode",
                                              "project_zbuf", "occlusion", "pool3", "tile_mark1", "contour",
                                              "bp_count", "bp_write") if k in work}
    roof["jbf_stage1"] = work["taps1"] / tap_peak(forms[0])[0] * 1e6
    if ns == 2:
        roof["jbf_stage2"] = work["taps2"] / tap_peak(forms[1])[0] * 1e6
    kroof = {k: {"roof_us": round(r, 2), "measured_us": ktable[k]["avg_us"],
                 "frac": round(r / ktable[k]["avg_us"], 3) if ktable[k]["avg_us"] else None}
             for k, r in roof.items() if k in ktable}
    ms = sum(step_ms) / len(step_ms)
    ideal = sum(v["roof_us"] for v in kroof.values())
    sizes = sorted({f"{v.camera.width}x{v.camera.height}" for v in views})
    out = {
        "config": dict({"workload": name, "frames_per_step": B, "distinct_views": len(views), "resolutions": sizes,
                        "stages": [list(st) for st in stages], "precision": "fp16" if cfg["precision"] else "fp32",
                        "l2": "flushed (256 MiB write) before every step", "launch": "batched CUDA graph"},
                       **({"prepost": cfg["prepost"], "previous_frame": "a block of the image changed"}
                          if cfg.get("prepost") else {})),
        "value": B / (ms / 1000.0), "unit": UNIT, "ms_per_step": ms,
        "latency_ms_per_step": {"p50": sorted(step_ms)[len(step_ms) // 2], "max": max(step_ms)},
        "gpu_launches": launches,
        "kernels": ktable,
        "path_roofline": {"ideal_us_per_step": round(ideal, 2), "measured_us_per_step": round(1000 * ms, 2),
                          "frac": round(ideal / (1000 * ms), 3), "kernels": kroof},
        "filter_kernels": choice,
    }
    outputs = [{"depth": b.depth.cpu().numpy(), "valid": b.valid.cpu().numpy()} for b in probe]
    return out, outputs


def config_cpu_leg(name, cfg, views, outputs, procs):
    """The oracle on the config's distinct views: its rate on the host cores and, per view, the GPU depth
    against it (valid masks compared exactly; max and p99 absolute error, max relative error)."""
    import concurrent.futures as cf
    import multiprocessing as mp

    import numpy as np
    n = len(outputs)
    t0 = time.perf_counter()
    extra = dict(cfg.get("prepost", {}))
    jobs = [(views[i], cfg["stages"], dict(extra, prev_rgb=moved_frame(views[i], i)) if cfg.get("moved") else extra)
            for i in range(n)]
    with cf.ProcessPoolExecutor(max(1, min(procs, n)), mp_context=mp.get_context("spawn")) as ex:
        refs = list(ex.map(_oracle_config_frame, jobs))
    dt = time.perf_counter() - t0
    per_view = []
    for v, g, (depth, valid) in zip(views, outputs, refs):
        m = valid.astype(bool) & g["valid"].astype(bool)   # depth where both are valid (masks reported apart)
        err = np.abs(g["depth"].astype(np.float64) - depth)[m] if m.any() else np.zeros(1)
        rel = err / depth[m] if m.any() else np.zeros(1)
        bound = np.maximum(1e-3, 1e-3 * depth[m]) if cfg["precision"] else 1e-4 * depth[m]
        per_view.append({"view": f"{v.camera.width}x{v.camera.height}", "valid_mask_exact": bool(
            np.array_equal(g["valid"], valid)), "mask_differences_px": int((g["valid"] != valid).sum()),
            "max_abs_m": float(err.max()), "p99_abs_m": float(np.percentile(err, 99)),
            "max_rel": float(rel.max()), "pixels_over_bar": int((err > bound).sum()) if m.any() else 0})
    return {"value": n / dt, "unit": UNIT, "cores": min(procs, n), "kind": "oracle",
            "sample": f"{n} distinct views of the workload, FP64, one single-threaded oracle process per view "
                      f"(start-up included), {dt:.1f} s",
            "error_vs_oracle": {"bar": "valid masks exact; depth within 1e-4 relative (FP32) or 1 mm absolute / "
                                       "1e-3 relative (FP16)", "per_view": per_view,
                                "all_masks_exact": all(p["valid_mask_exact"] for p in per_view),
                                **({"masks_note": "contour decisions are taken on the FP32 filtered map; pixels "
                                                  "whose relative step is within rounding of the threshold may "
                                                  "decide differently from the FP64 oracle"}
                                   if extra.get("contour_threshold") else {}),
                                "pixels_over_bar": sum(p["pixels_over_bar"] for p in per_view),
                                "max_abs_m": max(p["max_abs_m"] for p in per_view),
                                "max_rel": max(p["max_rel"] for p in per_view)}}


def _oracle_config_frame(args):
    import oracle
    v, stages, extra = args
    oracle.build()
    o = oracle.densify_view(v, num_stages=len(stages), stages=stages, emit_points=False, **extra)
    return o["depth"], o["valid"]


def make_views(n, seed0, rank=0):
    """Distinct 1080p three-scan viewpoints, generated in a spawn pool."""
    import concurrent.futures as cf
    import multiprocessing as mp
    jobs = [(s, i % 7, 7) for i, s in enumerate(rank_seeds(rank, n, seed0))]
    workers = max(1, min(n, (os.cpu_count() or 2) - 1, 12))
    if workers == 1:
        return [_gen(j) for j in jobs]
    with cf.ProcessPoolExecutor(workers, mp_context=mp.get_context("spawn")) as ex:
        return list(ex.map(_gen, jobs))


# ---------------------------------------------------------------------------
# replicas: viewpoints are independent, each rank densifies its own views
# ---------------------------------------------------------------------------
def rank_seeds(rank, n_views, base=1001):
    """Seeds of the distinct views rank ``rank`` generates (disjoint across ranks)."""
    return [base + 1000 * rank + i for i in range(n_views)]


def job_throughput(step_ms_local, frames_per_step, world, reduce_max):
    """Whole-job frames/s: all ranks' frames over the slowest rank's summed step time.
    ``reduce_max`` maps a local float to the max over ranks (identity at N=1)."""
    total_ms = reduce_max(float(sum(step_ms_local)))
    steps = len(step_ms_local)
    return world * frames_per_step * steps / (total_ms / 1000.0), total_ms


# ---------------------------------------------------------------------------
# clocks
# ---------------------------------------------------------------------------
class ClockSampler:
    Q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
         "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
         "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, index):
        self.index = index
        self.proc = None
        self.lines = []
        self.err = ""

    def start(self):
        try:
            self.proc = subprocess.Popen(["nvidia-smi", f"--id={self.index}", f"--query-gpu={self.Q}",
                                          "--format=csv,noheader,nounits", "-lms", "200"],
                                         stdout=subprocess.PIPE, stderr=subprocess.PIPE, text=True)
            self.t = threading.Thread(target=self._read, daemon=True)
            self.t.start()
        except Exception:
            self.proc = None

    def _read(self):
        for line in self.proc.stdout:
            self.lines.append(line.strip())

    def stop(self):
        if not self.proc:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except Exception:
            self.proc.kill()
        self.t.join(timeout=2)
        try:
            self.err = (self.proc.stderr.read() or "").strip()[:200]
        except Exception:
            pass
        sm, mx, reasons = [], None, set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for l in self.lines:
            p = [x.strip() for x in l.split(",")]
            if len(p) < 9:
                continue
            try:
                sm.append(float(p[1]))
                mx = float(p[2])
            except ValueError:
                continue
            for n, val in zip(names, p[5:9]):
                if val.lower() == "active":
                    reasons.add(n)
        sm.sort()
        out = {"sm_mhz": sm[len(sm) // 2] if sm else None, "sm_max_mhz": mx, "reasons": sorted(reasons),
               "samples": len(sm)}
        if not sm:
            out["error"] = self.err or (self.lines[0][:200] if self.lines else "no output")
        return out


# ---------------------------------------------------------------------------
# reference arm: the FP64 oracle on the host cores
# ---------------------------------------------------------------------------
_ORACLE_VIEWS = None


def _oracle_init(views):
    global _ORACLE_VIEWS
    import oracle
    oracle.build()
    _ORACLE_VIEWS = views


def _oracle_frame(i):
    import oracle
    oracle.densify_view(_ORACLE_VIEWS[i % len(_ORACLE_VIEWS)], num_stages=2, stages=STAGES)
    return i


def oracle_pool(views, procs):
    """Worker processes (spawned: the caller may already hold a CUDA context), each running the
    single-threaded FP64 oracle on whole frames; the views travel once, without ground truth."""
    import dataclasses
    import multiprocessing as mp
    slim = [dataclasses.replace(v, gt_depth=None) for v in views]
    pool = mp.get_context("spawn").Pool(procs, initializer=_oracle_init, initargs=(slim,))
    pool.map(_oracle_frame, range(procs))   # start-up and first touch, untimed
    return pool


def cpu_oracle_rate(views, frames, procs):
    """Frames/s of the oracle over a sample of ``frames`` frames: one process per core."""
    import oracle
    oracle.build()
    with oracle_pool(views, procs) as pool:
        t0 = time.perf_counter()
        pool.map(_oracle_frame, range(frames), chunksize=1)
        dt = time.perf_counter() - t0
    return frames / dt, dt


def reference_arm(a, rank, world):
    if rank != 0:
        return
    views = make_views(max(1, min(a.views, a.cpu_frames)), 1001, 0)
    import oracle
    oracle.build()
    procs = a.cpu_procs
    per = procs * max(1, a.cpu_frames // max(1, a.steps * procs))   # frames per step, a multiple of the workers
    with oracle_pool(views, procs) as pool:
        for _ in range(min(a.warmup, 1)):
            pool.map(_oracle_frame, range(procs))
        t0 = time.perf_counter()
        n = 0
        for s in range(a.steps):
            pool.map(_oracle_frame, range(s * per, (s + 1) * per), chunksize=1)
            n += per
        dt = time.perf_counter() - t0
    rate = n / dt
    sample = (f"{n} frames of the 1080p three-scan workload, {per} per step, FP64, one single-threaded "
              f"oracle process per core ({procs})")
    print(json.dumps({
        "impl": "reference", "metric": METRIC, "value": rate, "unit": UNIT, "n_gpus": a.gpus, "steps": a.steps,
        "warmup": a.warmup, "ms_per_step": 1000.0 * dt / a.steps, "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": "f64", "data": "synthetic",
        "config": {"workload": "1080p_3scan_two_stage", "frames_per_step": per, "resolution": "1920x1080",
                   "scans": 3, "sweep": "128x1024", "stages": "r4@1/3 + r2", "parallelism": "host cores"},
        "cpu_baseline": {"value": rate, "unit": UNIT, "cores": procs, "kind": "oracle", "sample": sample},
        "e2e": {"value": rate, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }), flush=True)


# ---------------------------------------------------------------------------
# our arm
# ---------------------------------------------------------------------------
def profiled_traffic(kernel, chosen=None):
    """DRAM bytes per launch recorded in profiles/traffic.json for ``kernel``, or None if
    the kernel's sources changed since that capture or the run chose another variant."""
    import hashlib
    try:
        recs = json.load(open(os.path.join(ROOT, "profiles", "traffic.json")))[kernel]
    except Exception:
        return None
    for rec in recs if isinstance(recs, list) else [recs]:
        if chosen is not None and any(chosen.get(k) != v for k, v in rec.get("variant", {}).items()):
            continue
        ok = True
        for path, digest in rec["sources"].items():
            try:
                ok &= hashlib.sha256(open(os.path.join(ROOT, path), "rb").read()).hexdigest()[:16] == digest
            except OSError:
                ok = False
        if ok:
            return rec["dram_bytes_per_launch"]
    return None


def valid_taps_stage2(coarse_valid, W, H, pool=3, r=2):
    """(output pixel, observed tap) pairs of the full-resolution filter."""
    import numpy as np
    from scipy.ndimage import correlate
    b2 = np.kron(coarse_valid.astype(np.float64), np.ones((pool, pool)))[:H, :W]
    return int(correlate(b2, np.ones((2 * r + 1, 2 * r + 1)), mode="constant").sum())


def valid_taps_stage1(cnt_pos, r=4):
    import numpy as np
    from scipy.ndimage import correlate
    return int(correlate(cnt_pos.astype(np.float64), np.ones((2 * r + 1, 2 * r + 1)), mode="constant").sum())


def step_work(b, view, pool=3, single_radius=None, prepost=None):
    """Algorithmic work of every kernel of the path for one frame (probe buffers with debug outputs):
    bytes each HBM-bound kernel must move at least, observed taps of the filters. single_radius:
    the single-stage form at that radius (no pooling; the mark kernel reads the z-buffer). prepost:
    the preprocessing and post-filter parameters, whose kernels' bytes are added."""
    import numpy as np
    W, H = b.W, b.H
    extra = {}
    if prepost:
        if prepost.get("motion_threshold"):
            extra["motion_mask"] = 7 * W * H          # RGB and previous RGB in, mask out
            extra["motion_dilate"] = 2 * W * H        # mask in, mask out
            extra["motion_erode"] = 2 * W * H
        if prepost.get("occlusion_radius"):
            extra["occlusion"] = 8 * W * H            # merged z-buffer in, kept z-buffer out
        if prepost.get("contour_threshold"):
            extra["contour"] = 10 * W * H             # filtered depth and validity in, outputs out
    if single_radius is not None:
        z = b.zbuf.cpu().numpy().view(np.uint32)
        obs = z != 0x7F800000
        npts = sum(s.xyz.shape[0] for s in view.scans)
        return {
            "prep_compose_clear": 4 * W * H,
            "project_zbuf": 12 * npts + 4 * int(obs.sum()),
            "tile_mark1": 4 * W * H,
            "bp_count": W * H,
            "bp_write": 8 * W * H + 16 * b.n_points(),
            "taps1": valid_taps_stage1(obs, single_radius),
            **extra,
        }
    Wc, Hc = -(-W // pool), -(-H // pool)
    z = b.zbuf.cpu().numpy().view(np.uint32)
    obs = z != 0x7F800000
    zp = np.zeros((Hc * pool, Wc * pool), bool)
    zp[:H, :W] = obs
    cnt_pos = zp.reshape(Hc, pool, Wc, pool).any(axis=(1, 3))
    npts = sum(s.xyz.shape[0] for s in view.scans)
    nout = b.n_points()
    return {
        "prep_compose_clear": 4 * W * H,                      # z-buffer clear
        "project_zbuf": 12 * npts + 4 * int(obs.sum()),       # point reads + one depth word per observed pixel
        "pool3": 7 * W * H + 20 * Wc * Hc,                    # z-buffer + RGB in, guide + sums out
        "tile_mark1": 4 * Wc * Hc,                            # one observation word per pooled pixel
        "bp_count": W * H,                                    # validity bytes
        "bp_write": 8 * W * H + 16 * nout,                    # validity, depth, colour in; points out
        "taps1": valid_taps_stage1(cnt_pos),
        "taps2": valid_taps_stage2(b.coarse_valid.cpu().numpy(), W, H),
        **extra,
    }


def host_link_bounds(link, h2d_bytes, d2h_bytes, frames, world=1):
    """End-to-end rates the host link allows for a step of ``frames`` frames at the measured copy
    rates: both directions at once (full duplex; the batch slots' copies in and out overlap),
    and one direction at a time (serial)."""
    t_in = h2d_bytes / (link["h2d_GBps"] * 1e9)
    t_out = d2h_bytes / (link["d2h_GBps"] * 1e9)
    both = link.get("both_GBps")
    extra = {}
    if both:   # both directions at once at the measured combined rate
        extra["duplex_frames_per_s"] = round(frames / max(t_in, t_out, (h2d_bytes + d2h_bytes) / (both * 1e9)) * world, 1)
    return dict(link, bound_frames_per_s=round(frames / max(t_in, t_out) * world, 1),
                serial_frames_per_s=round(frames / (t_in + t_out) * world, 1), **extra,
                note="copy-engine rates, 256 MiB pinned <-> device, each direction alone and both at once; "
                     "bound: both directions at once at their separate rates (the larger of bytes in / h2d rate "
                     "and bytes out / d2h rate per step); duplex: the same, also held to the measured combined "
                     "rate of both directions at once; serial: one direction after the other")


def host_link_gbps(dev, mb=256, reps=5):
    """Pinned host <-> device copy rates (GB/s), CUDA events: each direction alone, and both at once
    (two streams; the sum of the two directions' bytes over the common time)."""
    import torch
    h = torch.empty(mb << 20, dtype=torch.uint8, pin_memory=True)
    d = torch.empty(mb << 20, dtype=torch.uint8, device=dev)
    h2 = torch.empty(mb << 20, dtype=torch.uint8, pin_memory=True)
    d2 = torch.empty(mb << 20, dtype=torch.uint8, device=dev)
    out = {}
    for name, fn in (("h2d_GBps", lambda: d.copy_(h, non_blocking=True)),
                     ("d2h_GBps", lambda: h.copy_(d, non_blocking=True))):
        fn()
        torch.cuda.synchronize()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record()
        for _ in range(reps):
            fn()
        e1.record()
        torch.cuda.synchronize()
        out[name] = round(reps * (mb << 20) / (e0.elapsed_time(e1) / 1e3) / 1e9, 1)
    s1, s2 = torch.cuda.Stream(dev), torch.cuda.Stream(dev)
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    with torch.cuda.stream(s1):
        for _ in range(reps):
            d.copy_(h, non_blocking=True)
    with torch.cuda.stream(s2):
        for _ in range(reps):
            h2.copy_(d2, non_blocking=True)
    torch.cuda.synchronize()
    out["both_GBps"] = round(2 * reps * (mb << 20) / (time.perf_counter() - t0) / 1e9, 1)
    return out


def ours_arm(a, rank, world, local_rank):
    import numpy as np
    import torch
    from paper_2601_01210_gb300 import Densifier, build
    from paper_2601_01210_gb300.densify import DENSIFY_MEM_HOST
    from paper_2601_01210_gb300.frames import FrameBuffers

    views = make_views(a.views, 1001, rank)   # before any CUDA call (spawn pool)
    if "DENSIFY_TUNE_CACHE" not in os.environ or a.kernels:   # later contexts reuse the first one's choices
        import tempfile
        os.environ["DENSIFY_TUNE_CACHE"] = os.path.join(tempfile.mkdtemp(prefix="densify_tune_"), "tune.txt")
    if a.kernels:   # the tuner takes cached choices without timing: key = stage kind, radius, precision, pixel class
        px = a.batch * 1920 * 1080
        names = a.kernels.split(",")
        with open(os.environ["DENSIFY_TUNE_CACHE"], "w") as f:
            for (kind, st), name in zip(((1, STAGES[0]), (2, STAGES[1])), names):
                f.write(f"kind={kind},r={st[0]},half=0,px=2^{px.bit_length() - 1} {name}\n")
        a.autotune = 1
    mixed_views = make_mixed_views(16, 4004) if (not a.no_serve and rank == 0) else None
    config_views = make_config_views() if (not a.no_configs and rank == 0) else None
    build.build()
    torch.cuda.set_device(local_rank)
    dev = torch.device("cuda", local_rank)
    stream = torch.cuda.Stream(dev)           # library and events share this stream
    torch.cuda.set_stream(stream)
    B = a.batch
    def fb(i, **kw):
        v = views[i % len(views)]
        return FrameBuffers(v.camera, v.rgb, [(s.xyz, s.lidar_to_world) for s in v.scans], device=dev, **kw)

    bufs = [fb(i) for i in range(B)]
    params = dict(num_stages=2, stages=STAGES, max_batch=min(64, 2 * B), max_inflight=max(B, 16), launch_policy=1,
                  timing=a.kernel_timing, autotune=a.autotune,
                  batches_in_flight=1, hbm_budget_bytes=max(2 << 30, B * 48 << 20))
    flush_buf = torch.empty(L2_FLUSH_BYTES // 4, dtype=torch.int32, device=dev)
    with Densifier(params, device=local_rank, stream=stream.cuda_stream) as d:
        def step(k, timed):
            """Queue B frames (no launch yet), evict L2, then launch the batch between two events.
            The L2 flush keeps the GPU busy while the host records the events and launches, so the
            events bracket device work only."""
            ts = [d.submit(b.frame) for b in bufs]
            flush_buf.fill_(k)
            if timed:
                ev[k][0].record(stream)
            d.flush(-1)
            if timed:
                ev[k][1].record(stream)
            for t in ts:
                d.poll(t, -1)

        ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(a.steps)]
        for k in range(max(3, a.warmup)):
            step(k, False)
        torch.cuda.synchronize()
        # algorithmic work of the dominant kernel: observed taps of the full-resolution filter,
        # counted from each distinct view's first-stage mask (outside the timed region)
        probe = [fb(i, debug=True) for i in range(len(views))]
        for t in [d.submit(b.frame) for b in probe]:
            d.poll(t, -1)
        torch.cuda.synchronize()
        taps_view = [valid_taps_stage2(b.coarse_valid.cpu().numpy(), b.W, b.H) for b in probe]
        taps2 = sum(taps_view[i % len(views)] for i in range(B))
        work_view = [step_work(b, views[i]) for i, b in enumerate(probe)]
        work = {k: sum(work_view[i % len(views)][k] for i in range(B)) for k in work_view[0]}
        del probe
        d.reset_kernel_times()
        if world > 1:
            torch.distributed.barrier()
        # clocks: sample nvidia-smi over a window of the same workload that contains the timed steps
        props = torch.cuda.get_device_properties(dev)
        uuid = getattr(props, "uuid", None)
        clocks = ClockSampler(f"GPU-{uuid}" if uuid else local_rank)
        if not a.no_clocks:
            clocks.start()
        t_end = time.perf_counter() + (0.0 if a.no_clocks else 1.5)
        while time.perf_counter() < t_end:
            step(0, False)
        torch.cuda.synchronize()
        d.reset_kernel_times()
        if world > 1:
            torch.distributed.barrier()
        torch.cuda.synchronize()
        for k in range(a.steps):
            step(k, True)
        torch.cuda.synchronize()
        if world > 1:
            torch.distributed.barrier()
        times = d.kernel_times()
        gpu_launches = d.kernel_launches()   # CUDA kernels of the timed steps
        t_end = time.perf_counter() + (0.0 if a.no_clocks else 0.5)
        while time.perf_counter() < t_end:
            step(0, False)
        torch.cuda.synchronize()
        ck = clocks.stop() if not a.no_clocks else {"skipped": "--no-clocks"}
        step_ms = [s.elapsed_time(e) for s, e in ev]

        def reduce_max(x):
            if world == 1:
                return x
            t = torch.tensor([x], dtype=torch.float64, device=dev)
            torch.distributed.all_reduce(t, op=torch.distributed.ReduceOp.MAX)
            return float(t.item())

        value, total_ms = job_throughput(step_ms, B, world, reduce_max)
        kernel_choice = d.describe()

    # per-kernel table: a separate pass with an event after every kernel (those events add gaps
    # between kernels, so they stay out of the timed steps)
    ktable_times = times
    if a.kernel_timing != 1:
        with Densifier(dict(params, timing=1), device=local_rank, stream=stream.cuda_stream) as d3:
            for k in range(3 + 10):
                if k == 3:
                    torch.cuda.synchronize()
                    d3.reset_kernel_times()
                ts = [d3.submit(b.frame) for b in bufs]
                flush_buf.fill_(k)
                d3.flush(-1)
                for t in ts:
                    d3.poll(t, -1)
            torch.cuda.synchronize()
            ktable_times = d3.kernel_times()

    # e2e: pinned host buffers through the C ABI (points and RGB in, coloured points out), two batch
    # slots on the context's own streams so that one batch's copies overlap the next batch's kernels
    e2e = None
    if not a.no_e2e:
        # three batches in flight (three sets of page-locked buffers): while one batch's points travel to
        # the host, the next one's inputs travel to the device and a third one computes
        NB = 3
        hb = [[fb(i, memory=DENSIFY_MEM_HOST, depth_out=False) for i in range(B)] for _ in range(NB)]
        pe = dict(params, timing=0, batches_in_flight=NB, max_batch=B, max_inflight=(NB + 1) * B,
                  hbm_budget_bytes=max(2 << 30, NB * B * 64 << 20))
        with Densifier(pe, device=local_rank) as d2:
            def e2e_steps(n):
                pending = []
                for k in range(n):
                    pending.append([d2.submit(b.frame) for b in hb[k % NB]])   # the B-th submit launches it
                    if len(pending) == NB:   # collect the oldest batch before its buffers are reused
                        for t in pending.pop(0):
                            d2.poll(t, -1)
                for ts in pending:
                    for t in ts:
                        d2.poll(t, -1)

            e2e_steps(3)
            if world > 1:
                torch.distributed.barrier()
            t0 = time.perf_counter()
            e2e_steps(a.steps)
            dt = time.perf_counter() - t0
            dt = reduce_max(dt) if world > 1 else dt
        h2d = sum(sum(x.numel() * 4 for x, _ in b.scans) + b.rgb.numel() for b in hb[0])
        d2h = sum(8 + b.n_points() * 16 for b in hb[0])
        link = host_link_gbps(dev)
        e2e = {"value": B * a.steps / dt * world, "unit": UNIT, "h2d_bytes_per_step": int(h2d),
               "d2h_bytes_per_step": int(d2h),
               "what": "pinned host points + RGB in, coloured points out (written by the GPU into pinned memory)",
               "host_link": host_link_bounds(link, h2d, d2h, B, world)}
    serving = None
    if not a.no_serve and rank == 0:
        serving = serve_measure(mixed_views, dev, a.serve_seconds, a.autotune)
    fp16 = None
    if not a.no_fp16:
        fp16 = fp16_measure(a, bufs, params, dev, stream, flush_buf, taps2)
    if rank != 0:
        return
    peaks = {}
    try:
        peaks = json.load(open(os.path.join(ROOT, "MEASURED_PEAKS.json")))
    except Exception:
        pass
    sm_max = peaks.get("sm_max_mhz", 2070.0)
    sms = torch.cuda.get_device_properties(dev).multi_processor_count
    form1 = kernel_choice["stages"][0]["chosen"].get("form", "fp32_expanded")
    form2 = kernel_choice["stages"][-1]["chosen"].get("form", "fp32_expanded")
    # ALU peak of the filters: the measured instruction rates (profiles/alu_peaks.json, the microbenchmark
    # of the filter forms' arithmetic on this GPU model) give each form's tap peak as the least of the
    # issue, FMA-pipe and ex2 bounds; a live run of the same microbenchmark is reported beside it
    alu_file = alu_live = None
    try:
        alu_file = json.load(open(ALU_PEAKS))
    except Exception:
        pass
    try:
        if a.no_live_peaks:
            alu_live = {"skipped": "--no-live-peaks"}
        else:
            from paper_2601_01210_gb300 import alu_peaks
            alu_live = alu_peaks.measure(local_rank)
    except Exception as ex:   # the bench still reports against the committed measurement
        alu_live = {"error": str(ex)[:200]}
    alu_src = alu_file if alu_file else (alu_live if "tap_peaks" in (alu_live or {}) else None)

    def tap_peak(form):
        """(taps/s, basis) of a filter form."""
        if alu_src and form in alu_src["tap_peaks"]:
            t = alu_src["tap_peaks"][form]
            return t["taps_per_s"], (f"{'profiles/alu_peaks.json' if alu_file else 'live microbenchmark'}: "
                                     f"{t['taps_per_sm_clk']:.2f} taps per SM clock ({t['binds']} bound of "
                                     f"{t['bounds_taps_per_sm_clk']}) x {alu_src['sms']} SMs x "
                                     f"{alu_src['sm_mhz_median'] or alu_src['sm_max_mhz']:.0f} MHz, measured")
        ti = TAP_INSTR.get(form, 6.0)
        return sms * 128 / ti * sm_max * 1e6, f"{sms} SMs x 128 lanes / {ti:g} instructions per tap x {sm_max:.0f} MHz (model)"

    peak2, basis2 = tap_peak(form2)
    peak_gtap = peak2 / 1e9
    s2 = times.get("jbf_stage2", (0.0, 1))
    avg_us = s2[0] / max(1, s2[1])
    achieved = taps2 / (avg_us * 1e-6) / 1e9 if avg_us > 0 else 0.0
    ktable = {k: {"total_us": round(v[0], 2), "launches": v[1], "avg_us": round(v[0] / max(1, v[1]), 3)}
              for k, v in ktable_times.items()}
    # each kernel's roofline time for the step's work (HBM-bound kernels at the measured copy rate,
    # the filters at the ALU peak of their form), against its measured time; their sum is the path's roof
    hbm = peaks.get("hbm_gbs", 6758.5) * 1e9
    alu = lambda form: tap_peak(form)[0]   # taps per second
    roof_us = {k: work[k] / hbm * 1e6 for k in ("prep_compose_clear", "project_zbuf", "pool3", "tile_mark1",
                                                "bp_count", "bp_write")}
    roof_us["jbf_stage1"] = work["taps1"] / alu(form1) * 1e6
    roof_us["jbf_stage2"] = work["taps2"] / alu(form2) * 1e6
    kroof = {k: {"roof_us": round(r, 2), "measured_us": ktable[k]["avg_us"],
                 "frac": round(r / ktable[k]["avg_us"], 3) if ktable.get(k, {}).get("avg_us") else None}
             for k, r in roof_us.items() if k in ktable}
    ideal = sum(v["roof_us"] for v in kroof.values())
    path_roof = {"ideal_us_per_step": round(ideal, 2), "measured_us_per_step": round(1000.0 * total_ms / a.steps, 2),
                 "frac": round(ideal / (1000.0 * total_ms / a.steps), 3),
                 "basis": "sum over the path's kernels of algorithmic work / peak (HBM: measured copy rate; "
                          "filters: measured tap peak of their form)", "kernels": kroof}
    configs, config_outputs = {}, {}
    cviews = lambda cfg: views if cfg["views"] == "main" else config_views[cfg["views"]]
    if config_views:
        for cname, cfg in EXTRA_CONFIGS.items():
            configs[cname], config_outputs[cname] = config_measure(
                cname, cfg, cviews(cfg), a, dev, stream, flush_buf, tap_peak, hbm)
    cpu = None
    if not a.no_cpu_baseline:
        for cname, cfg in EXTRA_CONFIGS.items():   # each workload's oracle rate and error report
            if cname in configs:
                configs[cname]["cpu_baseline"] = config_cpu_leg(cname, cfg, cviews(cfg), config_outputs[cname],
                                                                a.cpu_procs)
        rate, dt = cpu_oracle_rate(views, a.cpu_frames, a.cpu_procs)
        cpu = {"value": rate, "unit": UNIT, "cores": a.cpu_procs, "kind": "oracle",
               "sample": f"{a.cpu_frames} frames of the same workload, FP64, one single-threaded oracle process "
                         f"per core ({a.cpu_procs}), {dt:.1f} s"}
        # the FP32 projection contract against a pure FP64 projection of the first view (untimed)
        import oracle
        v0 = views[0]
        cpu["projection_fp32_vs_fp64"] = oracle.projection_precision_report(
            v0.camera, [(s.xyz, s.lidar_to_world) for s in v0.scans])
    sorted_ms = sorted(step_ms)
    out = {
        "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": a.steps, "warmup": a.warmup,
        "ms_per_step": total_ms / a.steps, "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
        "dtype": "f32", "data": "synthetic (seeded room scenes, 3 LiDAR sweeps per view)",
        "config": {"workload": "1080p_3scan_two_stage", "frames_per_step": B, "distinct_views": len(views),
                   "clock_window": "nvidia-smi every 200 ms over >= 2 s of the same steps, timed steps inside",
                   "resolution": "1920x1080", "scans": 3, "sweep": "128x1024", "stages": "r4@1/3 + r2",
                   "sigma_p": 5.0, "sigma_c": 20.0, "precision": "fp32", "parallelism": f"replicas x{world}",
                   "l2": "flushed (256 MiB write) before every step", "launch": "batched CUDA graph"},
        "latency_ms_per_step": {"p50": sorted_ms[len(sorted_ms) // 2],
                                "p99": sorted_ms[min(len(sorted_ms) - 1, int(0.99 * len(sorted_ms)))]},
        "roofline": {"kernel": "jbf_stage2", "bound": "alu", "achieved": achieved, "peak": peak_gtap,
                     "unit": "Gtap/s", "frac": achieved / peak_gtap if peak_gtap else None,
                     "traffic": profiled_traffic("jbf_stage2", kernel_choice["stages"][-1]["chosen"]),
                     "traffic_unit": "bytes per launch (ncu capture of the same kernel variant)",
                     "peak_basis": f"{form2}: {basis2}",
                     "peak_live": (alu_live or {}).get("tap_peaks", {}).get(form2, alu_live),
                     "taps_per_launch": taps2, "avg_launch_us": avg_us},
        "kernels": ktable,
        "path_roofline": path_roof,
        "kernels_how": ("per-kernel CUDA events in a separate pass of 10 steps; the timed steps carry events "
                        "around the full-resolution filter only" if a.kernel_timing != 1 else
                        "per-kernel CUDA events inside the timed steps"),
        "filter_kernels": kernel_choice,
        "clocks": ck,
        "gpu_launches": gpu_launches,
        "e2e": e2e,
        "cpu_baseline": cpu,
        "fp16": fp16 and {"precision": "full-resolution stage: FP16 guide and weights, FP32 sums", **fp16},
        "configs": configs or None,
        "serving": serving and {"viewpoints": "16 (1080p/720p/540p mixed, 1-3 sweeps each)",
                                "paper_rate_seconds": a.serve_seconds,
                                "note": "frames/s and latency from arrival to completion seen by the loop (a host "
                                        "Python busy-poll: its turn time is part of every latency); batches: "
                                        "launched so far by the context and the most in flight at once",
                                **serving},
    }
    print(json.dumps(out), flush=True)


def main():
    a = parse()
    rank = int(os.environ.get("RANK", 0))
    world = int(os.environ.get("WORLD_SIZE", 1))
    local_rank = int(os.environ.get("LOCAL_RANK", 0))
    if a.impl == "reference":
        reference_arm(a, rank, world)
        return
    if world > 1:
        import torch
        import torch.distributed as dist
        # a multi-rank run times the headline workload and its end-to-end form only: the serving loop, the
        # other workloads and the FP16 form are single-GPU measurements that would hold every rank's GPU
        a.no_serve = a.no_configs = a.no_fp16 = True
        # views are generated before the first CUDA call (spawn pool), then the group starts
        dist.init_process_group("nccl" if torch.cuda.is_available() else "gloo")
    ours_arm(a, rank, world, local_rank)
    if world > 1:
        import torch.distributed as dist
        dist.destroy_process_group()


if __name__ == "__main__":
    main()
