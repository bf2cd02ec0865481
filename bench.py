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
    timed(fwd, steps, h, kf)
    timed(lambda: _lib.hrc_fluence_backward(h.ctx, gF, gE, gS), steps, h, kb)
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
    timed(fwd, steps, h, kf)
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


def bench_autograd(h, e, s, steps=10, warmup=3):
    """Gradient steps of an inverse-rendering loop through the autograd
    function `fluence` (forward hrc_fluence, backward hrc_fluence_backward):
    loss = mean((F(e) - F_target)^2), F_target the workload's own fluence,
    Adam on the emission from half its value.  `steady`: the plain loop,
    whose fresh output and gradient tensors come back from the caching
    allocator at recurring addresses; `moving`: every step differentiates
    through copies of its inputs that stay alive for 16 steps, so every step
    presents new addresses.  Each with graph replay on (the default) and off:
    ms per step (CUDA events on the stream, the optimiser step included) and
    the graphs the context captured per timed step."""
    import torch
    from paper_2505_02041_gb300 import _lib, fluence
    with torch.no_grad():
        target = h.forward(e, s).clone()
    stream = torch.cuda.current_stream(e.device)
    out = {}
    for mode in ("steady", "moving"):
        for graphs in (True, False):
            _lib.hrc_set_graphs(h.ctx, graphs)
            p = torch.nn.Parameter(0.5 * e.clone())
            opt = torch.optim.Adam([p], lr=0.01)
            keep = []

            def step():
                ein, sin = p, s
                if mode == "moving":
                    ein, sin = p.clone(), s.clone()
                    keep.append((ein, sin))
                    if len(keep) > 16:
                        keep.pop(0)
                loss = torch.mean((fluence(h, ein, sin) - target) ** 2)
                opt.zero_grad(set_to_none=True)
                loss.backward()
                opt.step()

            for _ in range(warmup):
                step()
            torch.cuda.synchronize(e.device)
            c0 = _lib.hrc_graph_captures(h.ctx)
            ts = []
            for _ in range(steps):
                a = torch.cuda.Event(enable_timing=True)
                z = torch.cuda.Event(enable_timing=True)
                a.record(stream)
                step()
                z.record(stream)
                z.synchronize()
                ts.append(a.elapsed_time(z))
            out[f"{mode}_graphs_{'on' if graphs else 'off'}"] = {
                "ms_per_step": statistics.mean(ts),
                "graph_captures_per_step": (_lib.hrc_graph_captures(h.ctx) - c0) / steps}
            del keep, opt, p
    _lib.hrc_set_graphs(h.ctx, True)
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


def survey_backward_bytes(W, H, C, precision, recompute):
    """Bytes of one backward pass over the same stored-level schedule
    (Sec. 4.3.2 with the adjoint of every step; the SURVEY byte model), per
    quadrant frame with |T_n| = U V (1 + 2^-n), V_T = C b_L + 4, V_R = C b_L,
    gradients fp32 (V_gT = 4 (C + 1), V_gR = 4 C):
      forward recompute (recompute=True only): T_0..T_N written, T_2..T_{N-1}
        read by the merge up, R_1..R_{N-1} written;
      adjoint of the sum: dL/dF read once (per image);
      adjoint merge down, n = N-1 .. 0: dL/dR_n and R_{n+1} read, |T_n| T
        entries read, dL/dR_{n+1} and |T_n| dL/dT entries written (each
        counted once: the lower end of 'a write plus at most one
        read-modify-write');
      adjoint merge up, n = N .. 3: dL/dT_n and T_{n-1} read, dL/dT_{n-1}
        read-modified-written;
      trace adjoint: dL/dT_0..dL/dT_2 and the inputs read, dL/de and dL/dsigma
        written (per image)."""
    bl = 4.0 if precision == "fp32" else 2.0
    vt, vr = C * bl + 4.0, C * bl
    vgt, vgr = 4.0 * (C + 1), 4.0 * C
    total = 0.0
    for U, V in ((W, H), (W, H), (H, W), (H, W)):
        N = max(0, (U - 1).bit_length())
        X2 = U * V
        t = lambda n: X2 * (1.0 + 2.0 ** -n)
        if recompute:
            total += vt * sum(t(n) for n in range(N + 1)) + vt * sum(t(n) for n in range(2, N)) + (N - 1) * X2 * vr
        for n in range(N - 1, -1, -1):
            total += X2 * vgr + (X2 * vr if n + 1 < N else 0.0) + t(n) * vt
            total += (X2 * vgr if n + 1 < N else 0.0) + t(n) * vgt
        for n in range(N, 2, -1):
            total += t(n) * vgt + t(n - 1) * vt + 2 * t(n - 1) * vgt
        total += sum(t(n) for n in range(min(N, 2) + 1)) * vgt
    img = W * H
    return total + img * C * 4.0 + img * (1 + C) * 4.0 + img * (1 + C) * 4.0


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


class Timer:
    """Steps timed with CUDA events on the launching stream, the L2 flushed
    (a 256 MB write) before each step, outside the events."""

    def __init__(self, dev):
        import torch
        self.torch = torch
        self.dev = dev
        self.flush = torch.empty(256 << 20, dtype=torch.uint8, device=dev)

    def __call__(self, step, n, h=None, per=None):
        torch = self.torch
        stream = torch.cuda.current_stream(self.dev)
        out = []
        for _ in range(n):
            self.flush.zero_()
            a = torch.cuda.Event(enable_timing=True)
            b = torch.cuda.Event(enable_timing=True)
            a.record(stream)
            step()
            b.record(stream)
            b.synchronize()
            out.append(a.elapsed_time(b))
            if per is not None:
                accumulate(per, h)
        return out


def accumulate(per, h):
    """Add the timing records of h's last call to per[kind] = [ms, bytes,
    records, launches]."""
    from paper_2505_02041_gb300 import _lib
    for kind, level, ms, by, nl in _lib.hrc_get_timing(h.ctx):
        d = per.setdefault(kind, [0.0, 0.0, 0, 0])
        d[0] += ms
        d[1] += by
        d[2] += 1
        d[3] += nl


def phase_table(per, steps, hbm_peak):
    return {k: {"ms_per_frame": v[0] / steps, "launches_per_frame": v[3] / steps, "bytes_per_frame": v[1] / steps,
                "GBps": v[1] / (v[0] * 1e-3) / 1e9 if v[0] > 0 else None,
                "frac_of_peak": v[1] / (v[0] * 1e-3) / 1e9 / hbm_peak if v[0] > 0 else None}
            for k, v in sorted(per.items())}


def measure_context(h, e, s, timed, steps, hbm_peak):
    """One context on one workload: graph-replayed forward and forward +
    backward (both backward strategies), then the same frames with the
    kernels timed by phase inside the replayed graphs (timing mode 3: one
    event before the first and one after the last launch of each phase, no
    event between launches) and launch by launch with direct launches
    (timing mode 1, each record including that launch's host-side launch
    latency)."""
    import torch
    from paper_2505_02041_gb300 import _lib
    F = torch.empty_like(e)
    gF = torch.ones_like(e)
    gE = torch.empty_like(e)
    gS = torch.empty_like(s)
    fwd = lambda: h.forward(e, s, F)

    def fwd_bwd():
        h.forward(e, s, F)
        _lib.hrc_fluence_backward(h.ctx, gF, gE, gS)

    for _ in range(3):
        fwd_bwd()
    fwd()
    n_fwd = h.launch_count()
    fwd_bwd()
    n_bwd = h.launch_count()
    out = {"forward_ms": timed(fwd, steps), "fwd_bwd_ms": timed(fwd_bwd, steps),
           "launches": {"forward": n_fwd, "backward": n_bwd}}
    _lib.hrc_set_backward_recompute(h.ctx, 1)
    fwd_bwd()
    fwd_bwd()
    out["launches"]["backward_recompute"] = h.launch_count()
    out["fwd_bwd_recompute_ms"] = timed(fwd_bwd, steps)
    _lib.hrc_set_backward_recompute(h.ctx, 0)
    for mode, name in ((3, "graph"), (1, "direct")):
        _lib.hrc_set_timing(h.ctx, mode)
        fw, bw = {}, {}
        fwd()
        timed(fwd, steps, h, fw)
        h.forward(e, s, F)
        timed(lambda: _lib.hrc_fluence_backward(h.ctx, gF, gE, gS), steps, h, bw)
        _lib.hrc_set_timing(h.ctx, 0)
        out["phases_" + name] = (fw, bw)
    h.sync()
    out["gbufs"] = (F, gF, gE, gS)
    return out


def roofline_of(phases_graph, phases_direct, steps, hbm_peak, workload, launch_config):
    """The dominant phase (largest share of the forward, timed inside the
    graph) against the measured copy peak, beside its launch-by-launch
    direct timing."""
    kind, (kms, kbytes, krec, klaunch) = max(phases_graph.items(), key=lambda kv: kv[1][0])
    achieved = kbytes / (kms * 1e-3) / 1e9
    d = phases_direct.get(kind)
    direct = None
    if d and d[0] > 0:
        ad = (d[1] / d[2]) / ((d[0] / d[2]) * 1e-3) / 1e9
        direct = {"achieved": ad, "frac": ad / hbm_peak, "us_per_launch": d[0] / d[2] * 1e3,
                  "timing": "each launch launched directly, bracketed by CUDA events (host launch latency included)"}
    return {"bound": "hbm", "kernel": kind, "achieved": achieved, "peak": hbm_peak, "unit": "GB/s",
            "frac": achieved / hbm_peak, "launches_per_frame": klaunch / steps,
            "bytes_per_launch": kbytes / max(klaunch, 1), "us_per_launch": kms / max(klaunch, 1) * 1e3,
            "traffic": ncu_traffic(traffic_key(kind, launch_config), workload),
            "timing": "the phase's launches as the replayed graph runs them, one CUDA event before the first and "
                      "one after the last (timing mode 3, on the launching stream, timed region 3); per launch = "
                      "phase time / launches, inter-launch gaps included",
            "per_launch_direct": direct}


def summarize(m, W, H, C, precision, steps, hbm_peak, world=1):
    """Per-frame figures of measure_context's record."""
    fw3, bw3 = m["phases_graph"]
    fwd_ms = per_frame(sum(m["forward_ms"]), steps, world)
    fb_ms = per_frame(sum(m["fwd_bwd_ms"]), steps, world)
    fbr_ms = per_frame(sum(m["fwd_bwd_recompute_ms"]), steps, world)
    frame_bytes = sum(v[1] for v in fw3.values()) / steps
    bwd_bytes = sum(v[1] for v in bw3.values()) / steps
    sum_bytes = fw3.get("fluence_sum", [0.0, 0.0, 0, 0])[1] / steps
    fb_bytes = frame_bytes + bwd_bytes
    fbr_bytes = fb_bytes + frame_bytes - sum_bytes
    paper = paper_schedule_bytes(W, H, C, precision)
    sb = survey_backward_bytes(W, H, C, precision, False)
    sbr = survey_backward_bytes(W, H, C, precision, True)
    gbps = lambda b, ms: b / (ms * 1e-3) / 1e9
    return {
        "forward_ms": fwd_ms, "fwd_bwd_ms": fb_ms, "fwd_bwd_recompute_ms": fbr_ms,
        "frame": {"algorithmic_bytes": frame_bytes, "GBps": gbps(frame_bytes, fwd_ms),
                  "frac_of_peak": gbps(frame_bytes, fwd_ms) / hbm_peak,
                  "paper_schedule_bytes": paper, "paper_schedule_frac": gbps(paper, fwd_ms) / hbm_peak},
        "fwd_bwd": {"ms": fb_ms, "algorithmic_bytes": fb_bytes, "GBps": gbps(fb_bytes, fb_ms),
                    "frac_of_peak": gbps(fb_bytes, fb_ms) / hbm_peak,
                    "survey_schedule_bytes": paper + sb, "survey_schedule_frac": gbps(paper + sb, fb_ms) / hbm_peak,
                    "backward": "reads the levels the forward left in the context"},
        "fwd_bwd_recompute": {"ms": fbr_ms, "algorithmic_bytes": fbr_bytes, "GBps": gbps(fbr_bytes, fbr_ms),
                              "frac_of_peak": gbps(fbr_bytes, fbr_ms) / hbm_peak,
                              "survey_schedule_bytes": paper + sbr,
                              "survey_schedule_frac": gbps(paper + sbr, fbr_ms) / hbm_peak,
                              "backward": "recomputes every level from the inputs first"},
    }


def bench_size(name, precision, timed, steps, hbm_peak):
    """Another workload size (512^2 or 2048^2) in its own autotuned context."""
    import torch
    from paper_2505_02041_gb300 import HRC, scenes
    e_np, s_np = scenes.scene_by_name(name)
    C, H, W = e_np.shape
    dev = torch.device("cuda", torch.cuda.current_device())
    e = torch.from_numpy(e_np).to(dev)
    s = torch.from_numpy(s_np).to(dev)
    h = HRC(W, H, C, 0, precision)
    tuned = h.autotune()
    m = measure_context(h, e, s, timed, steps, hbm_peak)
    out = {"workload": f"{name}: {WORKLOADS[name]}", "launch_config": h.launch_config, "autotune_best_ms": tuned,
           "launches": m["launches"]}
    out.update(summarize(m, W, H, C, precision, steps, hbm_peak))
    out["roofline"] = roofline_of(m["phases_graph"][0], m["phases_direct"][0], steps, hbm_peak, name, h.launch_config)
    out["phases"] = phase_table(m["phases_graph"][0], steps, hbm_peak)
    out["backward_phases"] = phase_table(m["phases_graph"][1], steps, hbm_peak)
    if name in PAPER_MS:
        out["paper_table1_ms"] = PAPER_MS[name]
    h.close()
    return out


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
    timed = Timer(dev)
    hbm_peak, peak_kind = peaks()

    def barrier():
        torch.cuda.synchronize(dev)
        if world > 1:
            torch.distributed.barrier()
        torch.cuda.synchronize(dev)

    for _ in range(max(args.warmup, 3)):
        h.forward(e, s, F)
    # timed regions 1 (forward frames, graph-replayed: the headline value),
    # 2 (forward + backward, both strategies) and 3 (the same frames with
    # phase and launch timing), nvidia-smi sampling the clocks throughout
    clocks = Clocks(local)
    barrier()
    clocks.start()
    m = measure_context(h, e, s, timed, args.steps, hbm_peak)
    barrier()
    clk = clocks.stop()
    F, gF, gE, gS = m["gbufs"]
    total_ms, fb_total, fbr_total = aggregate_max([sum(m["forward_ms"]), sum(m["fwd_bwd_ms"]),
                                                   sum(m["fwd_bwd_recompute_ms"])], world, dev)
    ms_per_frame = per_frame(total_ms, args.steps, world)

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

    fw3, bw3 = m["phases_graph"]
    fw1, bw1 = m["phases_direct"]
    summ = summarize(m, W, H, C, args.precision, args.steps, hbm_peak, world)
    summ["fwd_bwd"]["ms"] = per_frame(fb_total, args.steps, world)
    summ["fwd_bwd_recompute"]["ms"] = per_frame(fbr_total, args.steps, world)
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
        "roofline": roofline_of(fw3, fw1, args.steps, hbm_peak, args.workload, h.launch_config),
        "frame": dict(summ["frame"],
                      note="algorithmic_bytes: this implementation's schedule (live entries only, R_0 and the "
                           "fluence sum fused); paper_schedule_bytes: every level materialised and re-read once per "
                           "consuming phase (Sec. 4.3.2), whose time at the measured peak is the roofline the frame "
                           "is also compared with"),
        "phases": phase_table(fw3, args.steps, hbm_peak),
        "phases_direct": phase_table(fw1, args.steps, hbm_peak),
        "fwd_bwd": dict(summ["fwd_bwd"], backward_phases=phase_table(bw3, args.steps, hbm_peak)),
        "fwd_bwd_recompute": summ["fwd_bwd_recompute"],
        "e2e": {"value": e2e_ms, "unit": "ms/frame", "h2d_bytes_per_step": (C + 1) * H * W * 4,
                "d2h_bytes_per_step": C * H * W * 4},
        "gpu_launches": m["launches"]["forward"] * args.steps,
        "launches_per_step": dict(m["launches"], note="gpu_launches counts the forward frames timed for value"),
        "clocks": clk,
    }
    if world == 1 and args.sizes:
        line["sizes"] = {nm: bench_size(nm, args.precision, timed, 10, hbm_peak) for nm in ("fog512", "fog2048")}
    fwd = lambda: h.forward(e, s, F)

    def fwd_bwd():
        h.forward(e, s, F)
        _lib.hrc_fluence_backward(h.ctx, gF, gE, gS)

    line["cross_blur"] = bench_cross_blur(h, fwd, fwd_bwd, timed, gF, gE, gS, hbm_peak)
    line["multi_bounce"] = bench_bounces(h, e, s, timed, hbm_peak)
    line["environment"] = bench_environment(h, fwd, fwd_bwd, timed)
    line["per_channel_extinction"] = bench_channels(h, e, s, timed)
    line["autograd"] = bench_autograd(h, e, s)
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
            ms = statistics.mean(timed(lambda: hp.forward(e, s, Fp), args.steps))
            _lib.hrc_set_timing(hp.ctx, 3)
            per = {}
            hp.forward(e, s, Fp)
            timed(lambda: hp.forward(e, s, Fp), 5, hp, per)
            _lib.hrc_set_timing(hp.ctx, 0)
            by = sum(v[1] for v in per.values()) / 5
            Fn = Fp.cpu().numpy().astype(np.float64)
            lit = np.abs(Fr) >= 1e-3 * np.max(np.abs(Fr))   # pixels with non-negligible fluence
            rows[prec] = {"ms_per_frame": ms, "algorithmic_bytes": by, "GBps": by / (ms * 1e-3) / 1e9,
                          "frac_of_peak": by / (ms * 1e-3) / 1e9 / hbm_peak,
                          "paper_schedule_bytes": paper_schedule_bytes(W, H, C, prec),
                          "launch_config": hp.launch_config,
                          "phases": phase_table(per, 5, hbm_peak),
                          "err_max": float(np.max(np.abs(Fn - Fr)) / np.max(np.abs(Fr))),
                          "rel_l2": float(np.linalg.norm(Fn - Fr) / np.linalg.norm(Fr)),
                          "pixel_rel_max": float(np.max(np.abs(Fn - Fr)[lit] / np.abs(Fr)[lit])),
                          "pixel_rel_mean": float(np.mean(np.abs(Fn - Fr)[lit] / np.abs(Fr)[lit]))}
            hp.close()
        rows["speedup_vs_fp32"] = {p: rows["fp32"]["ms_per_frame"] / rows[p]["ms_per_frame"] for p in ("fp16", "bf16")}
        line["precisions"] = rows
    if args.batched and world == 1:
        h.close()
        del h, e, s, F, gF, gE, gS, m
        torch.cuda.empty_cache()
        # 64 scenes of sizes drawn from {128, ..., 2048}^2 (the 2048^2 ones
        # hold ~80 % of the work), and 256 small scenes from {64, 128, 256}^2
        line["batched"] = bench_batched(args, dev, scenes.batched_sizes(64, 4), 400)
        line["batched_small"] = bench_batched(args, dev, scenes.batched_sizes(256, 5, (64, 128, 256)), 1000)
    if world == 1 and not args.no_cpu_baseline:
        line["cpu_baseline"] = cpu_baseline(args.workload)
    print(json.dumps(line), flush=True)
    if world > 1:
        torch.distributed.destroy_process_group()


def bench_batched(args, dev, sizes, seed0):
    """A batch of square scenes of the given sizes, C = 3, fog / disks /
    rectangles as the 512^2 workload (seeds seed0 + i), bf16 interval
    storage: forward and forward+backward of the whole batch, each pass one
    graph-replayed launch sequence.  Beside it, the same scenes as a loop of
    single-scene hrc_fluence (+ hrc_fluence_backward) calls in the same
    precision: one autotuned context per size, each scene's inputs copied
    into that context's fixed buffers (so that its graph is replayed) and
    its outputs copied out, every copy inside the timed region."""
    import torch
    from paper_2505_02041_gb300 import BatchedHRC, HRC, _lib, scenes
    es, ss = [], []
    for i, X in enumerate(sizes):
        e, s = scenes.scene_disks_rects_fog(X, X, 3, seed0 + i)
        es.append(torch.from_numpy(e))
        ss.append(torch.from_numpy(s))
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

    # the loop of single-scene calls
    ed = [t.to(dev) for t in es]
    sd = [t.to(dev) for t in ss]
    Fd = [torch.empty_like(t) for t in ed]
    ged = [torch.empty_like(t) for t in ed]
    gsd = [torch.empty_like(t) for t in sd]
    ctxs, bufs = {}, {}
    for X in sorted(set(sizes)):
        hx = HRC(X, X, 3, 0, "bf16")
        hx.autotune()
        ctxs[X] = hx
        bufs[X] = [torch.empty((3, X, X), device=dev), torch.empty((X, X), device=dev),
                   torch.empty((3, X, X), device=dev), torch.ones((3, X, X), device=dev),
                   torch.empty((3, X, X), device=dev), torch.empty((X, X), device=dev)]

    def loop(backward):
        for i, X in enumerate(sizes):
            eb, sb, Fb, gFb, geb, gsb = bufs[X]
            eb.copy_(ed[i])
            sb.copy_(sd[i])
            ctxs[X].forward(eb, sb, Fb)
            Fd[i].copy_(Fb)
            if backward:
                _lib.hrc_fluence_backward(ctxs[X].ctx, gFb, geb, gsb)
                ged[i].copy_(geb)
                gsd[i].copy_(gsb)

    loop(True)
    loop(True)
    torch.cuda.synchronize(dev)
    loop_fwd_ms = run(lambda: loop(False))
    loop_fb_ms = run(lambda: loop(True))
    for hx in ctxs.values():
        hx.close()
    del ctxs, bufs, ed, sd, Fd, ged, gsd
    torch.cuda.empty_cache()

    try:
        b = BatchedHRC([(X, X) for X in sizes], 3, 0, "bf16")
    except Exception as ex:   # the batch needs about 200 GB of device memory
        return {"unavailable": f"batched context: {ex}", "loop_forward_ms": loop_fwd_ms, "loop_fwd_bwd_ms": loop_fb_ms}
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
    fwd_ms = run(lambda: b.forward(e, s, F))
    n_fwd = _lib.hrc_last_launch_count(b.ctx)
    fb_ms = run(lambda: (b.forward(e, s, F), b.backward(gF, ge, gs)))
    n_bwd = _lib.hrc_last_launch_count(b.ctx)
    b.sync()
    from collections import Counter
    out = {"scenes": len(sizes), "sizes": dict(Counter(sizes)), "channels": 3, "precision": "bf16",
           "forward_ms": fwd_ms, "forward_scenes_per_s": len(sizes) / (fwd_ms * 1e-3),
           "fwd_bwd_ms": fb_ms, "fwd_bwd_scenes_per_s": len(sizes) / (fb_ms * 1e-3),
           "loop_forward_ms": loop_fwd_ms, "loop_fwd_bwd_ms": loop_fb_ms,
           "speedup_vs_loop": {"forward": loop_fwd_ms / fwd_ms, "fwd_bwd": loop_fb_ms / fb_ms},
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
    ap.add_argument("--no-sizes", dest="sizes", action="store_false",
                    help="skip the 512^2 and 2048^2 workloads")
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
