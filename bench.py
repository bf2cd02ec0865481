#!/usr/bin/env python3
"""Benchmark of the HRC hot path on GB300.

A step is one HRC frame (Algorithm 1: trace T_0..T_2, merge up T_3..T_N,
merge down R_{N-1}..R_0, four-quadrant fluence sum) over the 1024 x 1024,
three-channel volumetric workload, fp32, with the inputs resident in HBM.
The L2 is flushed (a 256 MB write) before every timed step, outside the
timed events.

  python bench.py [--gpus N] [--steps K] [--warmup W] [--impl reference]

Prints one JSON line (rank 0).  ``--impl reference`` times the FP64 CPU
oracle on the same workload instead (the method has no other reference
implementation).
"""
from __future__ import annotations

import argparse
import hashlib
import json
import os
import statistics
import subprocess
import sys
import threading
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

WORKLOADS = {
    "volumetric1024": "1024x1024, C=3, sigma_t = 5 fBm (4 octaves) + 30 emitter disks + 100 walls "
                      "(sigma_t 200, 1-3 px), seed 2",
    "fog512": "512x512, C=3, fog 0.02 + 20 emitter disks + 40 rotated rectangles (sigma_t 50), seed 1",
    "fog2048": "2048x2048, C=3, as fog512 scaled, seed 5",
    "disks64": "64x64, C=1, vacuum, 3 emitter disks, 2 opaque boxes, seed 0",
}
PAPER_MS = {"volumetric1024": 7.67, "fog512": 1.85, "fog2048": 33.9}   # Table 1, RTX 3080 Laptop
METRIC = "HRC ms/frame & HBM GB/s (% peak) at 1024²; fwd+bwd ms; batched scenes/s"


def peaks():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            p = json.load(f)
        return float(p["hbm_gbs"]), "measured"
    except Exception:
        return 6800.0, "fallback"


def source_hash():
    h = hashlib.sha256()
    d = os.path.join(ROOT, "paper_2505_02041_gb300", "csrc")
    for f in sorted(os.listdir(d)):
        if f.endswith((".cu", ".cuh", ".h")):
            with open(os.path.join(d, f), "rb") as fh:
                h.update(fh.read())
    return h.hexdigest()[:16]


def bench_cross_blur(h, fwd, fwd_bwd, timed, gF, gE, gS, hbm_peak, thr=0.5, steps=10):
    """The frame with the Eq. 21 cross blur on (graph-launched forward and
    forward+backward), and the blur kernels' own per-launch times against
    their algorithmic bytes ((2C + 1) fp32 planes per pixel each)."""
    from paper_2505_02041_gb300 import _lib
    h.set_cross_blur(True, thr)
    for _ in range(3):
        fwd_bwd()
    f_ms = timed(fwd, steps)
    fb_ms = timed(fwd_bwd, steps)
    _lib.hrc_set_timing(h.ctx, True)
    kf, kb = {}, {}
    timed(fwd, steps, kf)
    timed(lambda: _lib.hrc_fluence_backward(h.ctx, gF, gE, gS), steps, kb)
    _lib.hrc_set_timing(h.ctx, False)
    h.set_cross_blur(False)
    out = {"threshold": thr, "forward_ms": statistics.mean(f_ms), "fwd_bwd_ms": statistics.mean(fb_ms)}
    for name, d in (("cross_blur", kf.get("cross_blur")), ("adj_cross_blur", kb.get("adj_cross_blur"))):
        if d:
            us = d[0] / d[2] * 1e3
            by = d[1] / d[2]
            out[name] = {"us": us, "bytes": by, "GBps": by / (us * 1e-6) / 1e9,
                         "frac_of_peak": by / (us * 1e-6) / 1e9 / hbm_peak}
    return out


def bench_bounces(h, e, s, timed, hbm_peak, K=6, rho=0.5, steps=5):
    """Multi-bounce lighting with K bounces (the count of the paper's Fig. 14)
    and a uniform albedo: graph-launched forward and forward+backward, and
    the source-update kernel's per-launch time against its algorithmic bytes
    ((4C + 1) fp32 planes per pixel)."""
    import torch
    from paper_2505_02041_gb300 import _lib
    C, H, W = e.shape
    h.reserve_bounces(K)
    a = torch.full_like(e, rho)
    F = torch.empty_like(e)
    gF = torch.ones_like(e)
    ge, gsg, ga = torch.empty_like(e), torch.empty_like(s), torch.empty_like(e)
    fwd = lambda: _lib.hrc_fluence_bounces(h.ctx, e, s, a, K, F)
    fwd_bwd = lambda: (fwd(), _lib.hrc_fluence_bounces_backward(h.ctx, gF, ge, gsg, ga))
    for _ in range(3):
        fwd_bwd()
    f_ms = timed(fwd, steps)
    fb_ms = timed(fwd_bwd, steps)
    fwd()
    launches = h.launch_count()
    _lib.hrc_set_timing(h.ctx, True)
    kf = {}
    timed(fwd, steps, kf)
    _lib.hrc_set_timing(h.ctx, False)
    out = {"bounces": K, "albedo": rho, "forward_ms": statistics.mean(f_ms), "fwd_bwd_ms": statistics.mean(fb_ms),
           "forward_ms_per_bounce": statistics.mean(f_ms) / (K + 1), "launches_forward": launches}
    d = kf.get("bounce_source")
    if d:
        us = d[0] / d[2] * 1e3
        by = d[1] / d[2]
        out["bounce_source"] = {"us": us, "bytes": by, "GBps": by / (us * 1e-6) / 1e9,
                                "frac_of_peak": by / (us * 1e-6) / 1e9 / hbm_peak}
    return out


def bench_environment(h, fwd, fwd_bwd, timed, steps=10):
    """The frame under an environment map (footnote 1 of Sec. 4.2; a smooth
    sky-like map of 256 directions): graph-launched forward and
    forward+backward."""
    import math
    import torch
    C = h.C
    th = torch.tensor([2 * math.pi * (m + 0.5) / 256 for m in range(256)], device="cuda")
    env = torch.stack([1.0 + 0.8 * torch.sin(th + 0.3 * k) for k in range(C)]).float().contiguous()
    h.set_environment(env)
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    h.set_environment(env)                 # the table build (synchronous), timed on the host
    table_ms = (time.perf_counter() - t0) * 1e3
    for _ in range(3):
        fwd_bwd()
    out = {"map_directions": 256, "forward_ms": statistics.mean(timed(fwd, steps)),
           "fwd_bwd_ms": statistics.mean(timed(fwd_bwd, steps)), "table_build_ms": table_ms}
    h.set_environment(None)
    return out


def bench_channels(h, e, s, timed, steps=10):
    """Per-channel extinction (sigma_t[C][H][W]: the workload's extinction
    scaled by 1, 0.5 and 2 per channel): graph-launched forward and
    forward+backward through the per-channel contexts."""
    import torch
    from paper_2505_02041_gb300 import _lib
    C = h.C
    S = torch.stack([s * f for f in (1.0, 0.5, 2.0, 1.5)[:C]]).contiguous()
    F = torch.empty_like(e)
    gF = torch.ones_like(e)
    ge, gs = torch.empty_like(e), torch.empty_like(S)
    cfg = h.launch_config
    h.set_channel_extinction(True)
    tuned = h.autotune()          # tunes the single-channel contexts (their best configuration differs)
    fwd = lambda: _lib.hrc_fluence(h.ctx, e, S, F)
    fwd_bwd = lambda: (fwd(), _lib.hrc_fluence_backward(h.ctx, gF, ge, gs))
    for _ in range(3):
        fwd_bwd()
    f_ms = timed(fwd, steps)
    fb_ms = timed(fwd_bwd, steps)
    fwd()
    out = {"forward_ms": statistics.mean(f_ms), "fwd_bwd_ms": statistics.mean(fb_ms),
           "launches_forward": h.launch_count(), "autotune_best_ms": tuned, "launch_config": h.launch_config}
    h.set_channel_extinction(False)
    h.set_launch_config(**cfg)
    return out


def traffic_key(kind, cfg):
    """The kernel variant whose DRAM bytes stand for `kind`: the merge down
    has a per-thread-load kernel (mdown 0) and a bulk-copy-staged one
    (mdown 1), each with its own line."""
    if kind == "merge_down" and cfg.get("mdown", 0) == 1:
        return "merge_down_bulk"
    return kind


def ncu_traffic(kind, workload):
    """Per-launch DRAM bytes of `kind` from the committed ncu summary, if it
    was taken on the current kernel sources."""
    path = os.path.join(ROOT, "profiles", "traffic.txt")
    if not os.path.exists(path):
        return None
    src = source_hash()
    with open(path) as f:
        for line in f:
            parts = line.split()
            if len(parts) >= 4 and parts[0] == kind and parts[1] == workload and parts[3] == src:
                return float(parts[2])
    return None


class Clocks:
    """nvidia-smi sampler running during the timed region."""
    Q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
         "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
         "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, index):
        self.index = index
        self.proc = None
        self.lines = []

    def start(self):
        try:
            self.proc = subprocess.Popen(["nvidia-smi", f"--id={self.index}", f"--query-gpu={self.Q}",
                                          "--format=csv,noheader,nounits", "-lms", "20"],
                                         stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.t = threading.Thread(target=self._read, daemon=True)
            self.t.start()
        except Exception:
            self.proc = None

    def _read(self):
        for line in self.proc.stdout:
            self.lines.append(line.strip())

    def stop(self):
        if self.proc is None:
            return None
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except Exception:
            self.proc.kill()
        sm, smax, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for ln in self.lines:
            f = [x.strip() for x in ln.split(",")]
            if len(f) < 9:
                continue
            try:
                sm.append(float(f[1]))
                smax.append(float(f[2]))
            except ValueError:
                continue
            for nm, val in zip(names, f[5:9]):
                if val.lower() == "active":
                    reasons.add(nm)
        if not sm:
            return None
        return {"sm_mhz": statistics.median(sm), "sm_max_mhz": max(smax), "reasons": sorted(reasons),
                "samples": len(sm)}


def paper_schedule_bytes(W, H, C, precision):
    """Bytes of one forward frame when every T level and two R levels are
    stored (Sec. 4.3.2) and every materialised array is written once and
    read once per consuming phase: per quadrant frame (U along the gathering
    axis, V across, N = ceil(log2 U), |T_n| = U V (1 + 2^-n) entries)
    V_T (sum_{n<=N} |T_n| + sum_{2<=n<N} |T_n| + sum_{n<N} |T_n|) + 2 N U V V_R,
    plus the inputs read and the fluence written once."""
    bl = 4.0 if precision == "fp32" else 2.0
    vt, vr = C * bl + 4.0, C * bl
    total = 0.0
    for U, V in ((W, H), (W, H), (H, W), (H, W)):
        N = max(0, (U - 1).bit_length())
        t = lambda n: U * V * (1.0 + 2.0 ** -n)
        total += vt * (sum(t(n) for n in range(N + 1)) + sum(t(n) for n in range(2, N)) +
                       sum(t(n) for n in range(N))) + 2 * N * U * V * vr
    return total + W * H * (1 + C) * 4.0 + W * H * C * 4.0


def aggregate_max(values, world, device=None):
    """Element-wise max over ranks of per-rank totals (identity on one rank):
    the job's time is its slowest rank's."""
    if world == 1:
        return [float(v) for v in values]
    import torch
    import torch.distributed as dist
    t = torch.tensor([float(v) for v in values], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return [float(v) for v in t.tolist()]


def per_frame(total_ms, steps, world):
    """Whole-job ms per frame: every rank runs `steps` frames of its own
    (independent replicas, weak scaling), all ranks in the max time."""
    return total_ms / (steps * world)


def dist_setup(n_gpus):
    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return rank, world, local


def run_reference(args):
    """FP64 CPU oracle, as it stands, on the host cores (rank 0 only)."""
    rank, world, _ = dist_setup(args.gpus)
    if rank != 0:
        return
    import numpy as np  # noqa: F401
    import oracle
    from paper_2505_02041_gb300 import scenes
    e, s = scenes.scene_by_name(args.workload)
    for _ in range(args.warmup):
        oracle.fluence(e, s)
    times = []
    for _ in range(args.steps):
        t0 = time.perf_counter()
        oracle.fluence(e, s)
        times.append((time.perf_counter() - t0) * 1e3)
    ms = statistics.mean(times)
    C, H, W = e.shape
    line = {
        "impl": "reference", "metric": METRIC, "value": ms, "unit": "ms/frame", "n_gpus": args.gpus,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": ms, "higher_is_better": False,
        "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
        "config": {"workload": f"{args.workload}: {WORKLOADS[args.workload]}", "precision": "fp64 CPU oracle"},
        "cpu_baseline": {"value": ms, "unit": "ms/frame", "cores": oracle.num_threads(), "kind": "oracle",
                         "cpu_model": cpu_model(), "cpu_count": os.cpu_count(),
                         "sample": f"{args.steps} full {W}x{H} C={C} frames (OpenMP over rows)"},
        "e2e": {"value": ms, "unit": "ms/frame", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line), flush=True)


def cpu_model():
    """The host CPU's model name (x86 'model name', or the Arm implementer /
    part numbers), for the CPU-baseline record."""
    try:
        with open("/proc/cpuinfo") as f:
            info = f.read()
    except OSError:
        return os.uname().machine
    fields = {}
    for line in info.splitlines():
        if ":" in line:
            k, v = (x.strip() for x in line.split(":", 1))
            fields.setdefault(k, v)
    if "model name" in fields:
        return fields["model name"]
    parts = {"0xd4f": "Neoverse V2", "0xd40": "Neoverse V1", "0xd0c": "Neoverse N1"}
    part = fields.get("CPU part", "")
    return f"{os.uname().machine} {parts.get(part, 'CPU part ' + part)}".strip()


def cpu_baseline(workload, budget_s=20.0):
    import oracle
    from paper_2505_02041_gb300 import scenes
    e, s = scenes.scene_by_name(workload)
    C, H, W = e.shape
    times = []
    t_start = time.perf_counter()
    while True:
        t0 = time.perf_counter()
        oracle.fluence(e, s)
        times.append((time.perf_counter() - t0) * 1e3)
        if time.perf_counter() - t_start > budget_s * 0.5 or len(times) >= 5:
            break
    return {"value": statistics.mean(times), "unit": "ms/frame", "cores": oracle.num_threads(), "kind": "oracle",
            "cpu_model": cpu_model(), "cpu_count": os.cpu_count(),
            "sample": f"{len(times)} full {W}x{H} C={C} frames of the same workload (FP64, OpenMP over rows)"}


def run_ours(args):
    import numpy as np
    import torch
    from paper_2505_02041_gb300 import HRC, _lib, scenes

    rank, world, local = dist_setup(args.gpus)
    torch.cuda.set_device(local)
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl")
    dev = torch.device("cuda", local)
    e_np, s_np = scenes.scene_by_name(args.workload)
    C, H, W = e_np.shape
    e = torch.from_numpy(e_np).to(dev)
    s = torch.from_numpy(s_np).to(dev)
    F = torch.empty((C, H, W), dtype=torch.float32, device=dev)
    h = HRC(W, H, C, 0, args.precision)
    tuned_ms = h.autotune() if not args.profile_once else None
    if args.schedule >= 0:
        _lib.hrc_set_schedule(h.ctx, args.schedule)
    if args.profile_once:
        # For profilers: one forward and one backward with direct (not
        # graph-replayed) launches inside the NVTX range "hrc_profile" (ncu
        # --nvtx --nvtx-include "hrc_profile/"), in a fixed launch
        # configuration: the autotuner's usual pick at 1024^2 (its timings are
        # meaningless under a profiler, which serialises every launch).
        # --profile-blur adds the Eq. 21 cross blur to both passes,
        # --profile-bounces K runs a K-bounce forward + backward instead.
        h.set_launch_config(*args.profile_config)
        gF1 = torch.ones((C, H, W), dtype=torch.float32, device=dev)
        if args.profile_blur:
            h.set_cross_blur(True)
        K = args.profile_bounces
        if K > 0:
            h.reserve_bounces(K)
            alb = torch.full_like(e, 0.5)

        def passes():
            if K > 0:
                h.forward_bounces(e, s, alb, K, F)
                h.backward_bounces(gF1)
            else:
                h.forward(e, s, F)
                h.backward(gF1)

        passes()
        torch.cuda.synchronize(dev)
        _lib.hrc_set_timing(h.ctx, True)
        torch.cuda.nvtx.range_push("hrc_profile")
        passes()
        torch.cuda.synchronize(dev)
        torch.cuda.nvtx.range_pop()
        _lib.hrc_set_timing(h.ctx, False)
        print(json.dumps({"profile_once": args.workload, "launches_fwd_bwd": h.launch_count()}))
        return
    stream = torch.cuda.current_stream(dev)
    flush = torch.empty(256 << 20, dtype=torch.uint8, device=dev)
    gF = torch.ones((C, H, W), dtype=torch.float32, device=dev)
    gE = torch.empty_like(e)
    gS = torch.empty_like(s)

    def barrier():
        torch.cuda.synchronize(dev)
        if world > 1:
            torch.distributed.barrier()
        torch.cuda.synchronize(dev)

    def fwd():
        h.forward(e, s, F)

    def fwd_bwd():
        h.forward(e, s, F)
        _lib.hrc_fluence_backward(h.ctx, gF, gE, gS)

    def timed(step, n, per_kind=None):
        """n steps, L2 flushed before each, CUDA events on the launching
        stream around each step; returns per-step ms."""
        out = []
        for _ in range(n):
            flush.zero_()
            a = torch.cuda.Event(enable_timing=True)
            b = torch.cuda.Event(enable_timing=True)
            a.record(stream)
            step()
            b.record(stream)
            b.synchronize()
            out.append(a.elapsed_time(b))
            if per_kind is not None:
                for kind, level, ms, by in _lib.hrc_get_timing(h.ctx):
                    d = per_kind.setdefault(kind, [0.0, 0.0, 0])
                    d[0] += ms
                    d[1] += by
                    d[2] += 1
        return out

    for _ in range(max(args.warmup, 3)):
        fwd_bwd()
    fwd()
    fwd_launches = h.launch_count()
    fwd_bwd()
    bwd_launches = h.launch_count()

    # timed region 1: forward frames, graph-launched (the headline value)
    clocks = Clocks(local)
    barrier()
    clocks.start()
    step_ms = timed(fwd, args.steps)
    barrier()
    # timed region 2: forward + backward
    fb_ms = timed(fwd_bwd, args.steps)
    barrier()
    # timed region 2b: forward + backward that recomputes every level
    _lib.hrc_set_backward_recompute(h.ctx, 1)
    fwd_bwd()
    fwd_bwd()
    rc_launches = h.launch_count()
    barrier()
    fbr_ms = timed(fwd_bwd, args.steps)
    barrier()
    _lib.hrc_set_backward_recompute(h.ctx, 0)
    fwd_bwd()
    # timed region 3: the same frames with per-launch CUDA events (kernel
    # durations for the roofline; launches are not graph-replayed here)
    _lib.hrc_set_timing(h.ctx, True)
    per_kind = {}
    prof_ms = timed(fwd, args.steps, per_kind)
    bwd_kind = {}
    h.forward(e, s, F)
    for _ in range(args.steps):
        flush.zero_()
        _lib.hrc_fluence_backward(h.ctx, gF, gE, gS)
        for kind, level, ms, by in _lib.hrc_get_timing(h.ctx):
            d = bwd_kind.setdefault(kind, [0.0, 0.0, 0])
            d[0] += ms
            d[1] += by
            d[2] += 1
    _lib.hrc_set_timing(h.ctx, False)
    barrier()
    clk = clocks.stop()
    total_ms, fb_total, fbr_total = aggregate_max([sum(step_ms), sum(fb_ms), sum(fbr_ms)], world, dev)
    ms_per_frame = per_frame(total_ms, args.steps, world)
    fb_mean = per_frame(fb_total, args.steps, world)
    fbr_mean = per_frame(fbr_total, args.steps, world)

    # end to end: host buffers through the C ABI, copies included
    e_h = torch.from_numpy(e_np).pin_memory()
    s_h = torch.from_numpy(s_np).pin_memory()
    F_h = torch.empty((C, H, W), dtype=torch.float32).pin_memory()
    for _ in range(2):
        h.forward_host(e_h, s_h, F_h)
    barrier()
    t0 = time.perf_counter()
    for _ in range(args.steps):
        h.forward_host(e_h, s_h, F_h)
    e2e_ms = (time.perf_counter() - t0) * 1e3 / args.steps

    if rank != 0:
        if world > 1:
            torch.distributed.destroy_process_group()
        return

    hbm_peak, peak_kind = peaks()
    kind, (kms, kbytes, kcount) = max(per_kind.items(), key=lambda kv: kv[1][0])
    achieved = (kbytes / kcount) / ((kms / kcount) * 1e-3) / 1e9
    phases = {k: {"ms_per_frame": v[0] / args.steps, "launches_per_frame": v[2] / args.steps,
                  "GBps": v[1] / (v[0] * 1e-3) / 1e9 if v[0] > 0 else None}
              for k, v in sorted(per_kind.items())}
    frame_bytes = sum(v[1] for v in per_kind.values()) / args.steps
    bwd_bytes = sum(v[1] for v in bwd_kind.values()) / args.steps
    fb_bytes = frame_bytes + bwd_bytes
    paper_bytes = paper_schedule_bytes(W, H, C, args.precision)
    sum_bytes = per_kind.get("fluence_sum", [0.0, 0.0, 0])[1] / args.steps
    fbr_bytes = fb_bytes + frame_bytes - sum_bytes   # the recompute repeats the forward but the sum
    line = {
        "metric": METRIC, "value": ms_per_frame, "unit": "ms/frame", "n_gpus": world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": total_ms / args.steps, "higher_is_better": False,
        "scaling": "weak",
        "vs_baseline": (ms_per_frame / PAPER_MS[args.workload]) if args.workload in PAPER_MS else None,
        "dtype": "f32" if args.precision == "fp32" else args.precision,
        "data": "synthetic",
        "config": {"workload": f"{args.workload}: {WORKLOADS[args.workload]}", "precision": args.precision,
                   "parallelism": "replicas" if world > 1 else "single GPU",
                   "l2": "flushed (256 MB write) before every timed step, outside the timed events",
                   "launch": "one CUDA graph per pass (captured at warm-up); configuration chosen by hrc_autotune",
                   "autotune_best_ms": tuned_ms,
                   "launch_config": h.launch_config,
                   "baseline_context": "paper Table 1 on an RTX 3080 Laptop with fp16 storage"},
        "roofline": {"bound": "hbm", "kernel": kind, "achieved": achieved, "peak": hbm_peak, "unit": "GB/s",
                     "frac": achieved / hbm_peak, "peak_kind": peak_kind,
                     "traffic": ncu_traffic(traffic_key(kind, h.launch_config), args.workload),
                     "timing": "per-launch CUDA events on the launching stream (timed region 3)"},
        "frame": {"algorithmic_bytes": frame_bytes, "GBps": frame_bytes / (ms_per_frame * 1e-3) / 1e9,
                  "frac_of_peak": frame_bytes / (ms_per_frame * 1e-3) / 1e9 / hbm_peak,
                  "ms_with_per_launch_events": statistics.mean(prof_ms),
                  "paper_schedule_bytes": paper_bytes,
                  "paper_schedule_frac": paper_bytes / (ms_per_frame * 1e-3) / 1e9 / hbm_peak,
                  "note": "algorithmic_bytes: this implementation's schedule (live entries only, R_0 and the "
                          "fluence sum fused); paper_schedule_bytes: every level materialised and re-read "
                          "once per consuming phase (Sec. 4.3.2), whose time at the measured peak is the "
                          "roofline the frame is also compared with"},
        "phases": phases,
        "fwd_bwd": {"ms": fb_mean, "algorithmic_bytes": fb_bytes,
                    "GBps": fb_bytes / (fb_mean * 1e-3) / 1e9,
                    "frac_of_peak": fb_bytes / (fb_mean * 1e-3) / 1e9 / hbm_peak,
                    "backward_phases": {k: {"ms_per_frame": v[0] / args.steps, "launches_per_frame": v[2] / args.steps,
                                            "GBps": v[1] / (v[0] * 1e-3) / 1e9 if v[0] > 0 else None}
                                        for k, v in sorted(bwd_kind.items())},
                    "backward": "reads the levels the forward left in the context"},
        "fwd_bwd_recompute": {"ms": fbr_mean, "algorithmic_bytes": fbr_bytes,
                              "GBps": fbr_bytes / (fbr_mean * 1e-3) / 1e9,
                              "frac_of_peak": fbr_bytes / (fbr_mean * 1e-3) / 1e9 / hbm_peak,
                              "backward": "recomputes every level from the inputs first (hrc_set_backward_recompute)"},
        "e2e": {"value": e2e_ms, "unit": "ms/frame", "h2d_bytes_per_step": (C + 1) * H * W * 4,
                "d2h_bytes_per_step": C * H * W * 4},
        "gpu_launches": fwd_launches * args.steps,
        "launches_per_step": {"forward": fwd_launches, "backward": bwd_launches,
                              "backward_recompute": rc_launches,
                              "note": "gpu_launches counts the forward frames timed for value"},
        "clocks": clk,
    }
    line["cross_blur"] = bench_cross_blur(h, fwd, fwd_bwd, timed, gF, gE, gS, hbm_peak)
    line["multi_bounce"] = bench_bounces(h, e, s, timed, hbm_peak)
    line["environment"] = bench_environment(h, fwd, fwd_bwd, timed)
    line["per_channel_extinction"] = bench_channels(h, e, s, timed)
    if args.precisions and world == 1:
        import oracle
        Fr = oracle.fluence(e_np, s_np)
        rows = {}
        for prec in ("fp32", "fp16", "bf16"):
            hp = HRC(W, H, C, 0, prec)
            hp.autotune()
            Fp = torch.empty((C, H, W), dtype=torch.float32, device=dev)
            for _ in range(3):
                hp.forward(e, s, Fp)
            ms = timed(lambda: hp.forward(e, s, Fp), args.steps)
            Fn = Fp.cpu().numpy().astype(np.float64)
            lit = np.abs(Fr) >= 1e-3 * np.max(np.abs(Fr))   # pixels with non-negligible fluence
            rows[prec] = {"ms_per_frame": statistics.mean(ms),
                          "err_max": float(np.max(np.abs(Fn - Fr)) / np.max(np.abs(Fr))),
                          "rel_l2": float(np.linalg.norm(Fn - Fr) / np.linalg.norm(Fr)),
                          "pixel_rel_max": float(np.max(np.abs(Fn - Fr)[lit] / np.abs(Fr)[lit])),
                          "pixel_rel_mean": float(np.mean(np.abs(Fn - Fr)[lit] / np.abs(Fr)[lit]))}
            hp.close()
        line["precisions"] = rows
    if args.batched and world == 1:
        del h, e, s, F, gF, gE, gS, flush
        torch.cuda.empty_cache()
        line["batched"] = bench_batched(args, dev)
    if world == 1 and not args.no_cpu_baseline:
        line["cpu_baseline"] = cpu_baseline(args.workload)
    print(json.dumps(line), flush=True)
    if world > 1:
        torch.distributed.destroy_process_group()


def bench_batched(args, dev):
    """64 scenes of sizes drawn from {128, 256, 512, 1024, 2048}^2 (seed 4),
    C = 3, fog / disks / rectangles as the 512^2 workload (seeds 400+i),
    bf16 interval storage: forward and forward+backward of the whole batch,
    each pass one graph-replayed launch sequence: the tile steps of all
    scenes as ordinary launches around one persistent launch of the merge
    cascade."""
    import torch
    from paper_2505_02041_gb300 import BatchedHRC, scenes
    sizes = scenes.batched_sizes(64, 4)
    es, ss = [], []
    for i, X in enumerate(sizes):
        e, s = scenes.scene_disks_rects_fog(X, X, 3, 400 + i)
        es.append(torch.from_numpy(e))
        ss.append(torch.from_numpy(s))
    try:
        b = BatchedHRC([(X, X) for X in sizes], 3, 0, "bf16")
    except Exception as ex:   # the batch needs about 200 GB of device memory
        return {"unavailable": f"batched context: {ex}"}
    e, s = b.pack(es, ss)
    del es, ss
    F = torch.empty_like(e)
    gF = torch.ones_like(e)
    ge = torch.empty_like(e)
    gs = torch.empty_like(s)
    tune = b.autotune(e, s, reps=2)
    best = min(tune, key=tune.get)
    b.forward(e, s, F)
    b.backward(gF, ge, gs)
    b.sync()
    n = max(3, min(args.steps, 5))
    stream = torch.cuda.current_stream(dev)

    def run(step):
        ts = []
        for _ in range(n):
            a = torch.cuda.Event(enable_timing=True)
            z = torch.cuda.Event(enable_timing=True)
            a.record(stream)
            step()
            z.record(stream)
            z.synchronize()
            ts.append(a.elapsed_time(z))
        return statistics.mean(ts)

    from paper_2505_02041_gb300 import _lib
    fwd_ms = run(lambda: b.forward(e, s, F))
    n_fwd = _lib.hrc_last_launch_count(b.ctx)
    fb_ms = run(lambda: (b.forward(e, s, F), b.backward(gF, ge, gs)))
    n_bwd = _lib.hrc_last_launch_count(b.ctx)
    b.sync()
    from collections import Counter
    out = {"scenes": len(sizes), "sizes": dict(Counter(sizes)), "channels": 3, "precision": "bf16",
           "forward_ms": fwd_ms, "forward_scenes_per_s": len(sizes) / (fwd_ms * 1e-3),
           "fwd_bwd_ms": fb_ms, "fwd_bwd_scenes_per_s": len(sizes) / (fb_ms * 1e-3),
           "launches_per_pass": {"forward": n_fwd, "backward": n_bwd},
           "schedule": ("persistent: trace / adjoint trace of all scenes as tile launches, the merge cascade "
                        "of all scenes in one persistent launch" if best[0] == 0 else
                        "per-scene launch chains on 8 parallel graph branches"),
           "autotune_ms": {f"sched{k[0]}_bpsm{k[1]}_order{k[2]}": v for k, v in tune.items()},
           "timed_batches": n}
    b.close()
    return out


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=20)
    ap.add_argument("--warmup", type=int, default=5)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--workload", default="volumetric1024", choices=sorted(WORKLOADS))
    ap.add_argument("--precision", default="fp32", choices=["fp32", "fp16", "bf16"])
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-precisions", dest="precisions", action="store_false",
                    help="skip the fp16 / bf16 error-and-time sweep against the FP64 oracle")
    ap.add_argument("--schedule", type=int, default=-1, help="launch schedule (default: the library's)")
    ap.add_argument("--no-batched", dest="batched", action="store_false",
                    help="skip the 64-scene batched persistent-launch measurement")
    ap.add_argument("--profile-config", type=int, nargs=5, default=[0, 1, 128, 1, 0],
                    metavar=("SCHEDULE", "GROUPS", "THREADS", "VMAJOR", "MDOWN"),
                    help="launch configuration of --profile-once (default: the autotuner's usual pick at 1024^2)")
    ap.add_argument("--profile-blur", action="store_true", help="--profile-once with the cross blur on")
    ap.add_argument("--profile-bounces", type=int, default=0,
                    help="--profile-once: a forward + backward of this many bounces (albedo 0.5)")
    ap.add_argument("--profile-once", action="store_true",
                    help="run one forward + backward inside the NVTX range hrc_profile with direct "
                         "launches in --profile-config (a target for ncu), print no bench line")
    args = ap.parse_args()
    if args.impl == "reference":
        run_reference(args)
    else:
        run_ours(args)


if __name__ == "__main__":
    main()
