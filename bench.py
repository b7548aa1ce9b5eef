"""Benchmark: Mpix/s of the 5x5 DDF on 1920x1080 RGB, FP32 certified path
(+ FP64 recheck of near-ties) against the plain FP64 GPU path.

    python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]

One step filters one 1080p frame through the whole hot path (load, pair
terms, aggregation, DDF scores, selection, FP64 recheck, store).  Inputs are
24 distinct synthetic frames (149 MB, more than the 129 MB L2) resident in HBM
and used in rotation.  Rank 0 prints one JSON line.  Under torchrun every rank
filters its own frames (independent replicas, weak scaling); the slowest
rank's time sets the whole-job throughput.

``--impl reference`` times the CPU oracle (the plain FP64/binary128 C
implementation in oracle/) on the host cores, on a pixel sample of the same
workload, and prints the same line with "impl": "reference".
"""
from __future__ import annotations

import argparse
import ctypes
import hashlib
import json
import os
import statistics
import subprocess
import sys
import tempfile
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

M, N, WIN, FILTER, P, DIST, Q = 1080, 1920, 5, "ddf", 0.25, "exact", 4
NOISE, RECTS, FRAMES = 0.10, 12, 24
WORKLOAD = ("DDF 5x5 (p=0.25, exact arccos) on 1920x1080 RGB uint8: sinusoid field + 12 flat rectangles, "
            "10% impulsive noise")
METRIC = "Mpix/s, 5x5 DDF on 1080p RGB: FP32+FP64-tie path vs plain FP64 GPU path"
UNIT = "Mpix/s"
CONFIG = {"workload": WORKLOAD, "M": M, "N": N, "win": WIN, "filter": FILTER, "p": P, "dist": DIST,
          "noise": NOISE, "rectangles": RECTS, "frames_in_rotation": FRAMES,
          "l2": "inputs larger than L2: 24 distinct frames (149 MB) in rotation"}



def set_workload(m, n, noise, nframes, workload, metric, config):
    global M, N, NOISE, FRAMES, WORKLOAD, METRIC, CONFIG
    M, N, NOISE, FRAMES, WORKLOAD, METRIC, CONFIG = m, n, noise, nframes, workload, metric, config


def use_4k_workload():
    """The precision stress case (3840 x 2160, 20% impulsive noise): same
    filter and path, frames rebound for every function of this module."""
    global M, N, NOISE, FRAMES, WORKLOAD, METRIC, CONFIG
    M, N, NOISE, FRAMES = 2160, 3840, 0.20, 6
    WORKLOAD = ("DDF 5x5 (p=0.25, exact arccos) on 3840x2160 RGB uint8: sinusoid field + 12 flat rectangles, "
                "20% impulsive noise")
    METRIC = "Mpix/s, 5x5 DDF on 4K RGB, 20% noise: FP32+FP64-tie path vs plain FP64 GPU path"
    CONFIG = {"workload": WORKLOAD, "M": M, "N": N, "win": WIN, "filter": FILTER, "p": P, "dist": DIST,
              "noise": NOISE, "rectangles": RECTS, "frames_in_rotation": FRAMES,
              "l2": "inputs larger than L2: 6 distinct frames (149 MB) in rotation"}


# Algorithmic work per output pixel (the roofline's numerator), fixed before
# any tuning from the operation counts of the method itself, not from the
# kernels' source: see opcount().
ANGLE_TERM_OPS = {"exact": 25, "minimax": 25, "rgb": 9}
DIST_TERM_OPS = {2: 7, 1: 6, "inf": 6}


def opcount(win: int, filt: str, dist: str = "exact", order=2) -> int:
    """FP32-pipe operations per output pixel of one filter configuration.

    Derivation (window side w, n = w^2 members, U = ((2w-1)^2 - 1) / 2
    unordered pair offsets a pixel meets across the windows that contain it,
    12 for 3x3 and 40 for 5x5):
      * pair terms, each computed once and reused by every window holding the
        pair: U x (angle + distance).  The angle of Eq. (2) (or Method 1's
        polynomial): 3 multiply-adds for <x,y>, 6 for |x cross y|^2, 2 SFU
        operations, 8 polynomial multiply-adds, 1 select, rounded to 25.
        Method 2's chromaticity distance (Eq. (7)): 8 multiply-adds + 1 SFU = 9.
        The Minkowski distance of Eq. (1): order 2, 6 multiply-adds + 1 SFU
        = 7; orders 1 and infinity, 3 differences + 3 combines = 6.
      * aggregation: n (n - 1) adds (each of the n members sums n terms);
      * selection: n - 1 compares;
      * DDF combine: 2 n logarithms (one per aggregate).
    BVDF = U x angle + n(n-1) + (n-1); DDF adds U x distance and 2n; VMF =
    U x distance + n(n-1) + (n-1).  DDF 5x5 exact: 40 x 32 + 600 + 24 + 50 =
    1954.  The count does not depend on the kernels, so it does not move when
    they change; a kernel that needs fewer operations shows as a higher
    fraction of the peak.
    """
    U, n = ((2 * win - 1) ** 2 - 1) // 2, win * win
    agg, sel = n * (n - 1), n - 1
    if filt == "vmf":
        return U * DIST_TERM_OPS[order] + agg + sel
    if filt == "bvdf":
        return U * ANGLE_TERM_OPS[dist] + agg + sel
    return U * (ANGLE_TERM_OPS[dist] + DIST_TERM_OPS[order]) + agg + sel + 2 * n


def opcount_acwddf(win: int, dist: str = "exact") -> int:
    """The ACWDDF of Eq. (9): the DDF's count, plus n centre distances (order
    2), three centre-weighted levels of n multiply-adds and n - 1 compares each,
    and the switching sum over three levels (one angle, one distance and two
    operations each)."""
    n = win * win
    return (opcount(win, "ddf", dist) + n * DIST_TERM_OPS[2] + 3 * (n + n - 1)
            + 3 * (ANGLE_TERM_OPS[dist] + DIST_TERM_OPS[2] + 2))


SMS, FP32_LANES_PER_SM = 152, 128

# DRAM bytes per launch of the FP32 tile kernel, from one ncu capture, keyed
# by a hash of the kernel sources it was taken on (null once they change).
TRAFFIC_BY_SOURCE = {"96fbf97cada8ac60": 6258688}   # profiles/tile_kernel_fp32_ddf5_1080p.md


# DRAM bytes per launch of the backward gather on the differentiable workload
# (profiles/backward_gather_autograd_32x512x512.md), keyed like the above by a
# hash of vdf_backward.cu only.
BACKWARD_TRAFFIC_BY_SOURCE = {"44b820dcd4629e61": 166681856}   # 109,069,824 read + 57,612,032 written


def backward_source_hash() -> str:
    with open(os.path.join(ROOT, "paper_1009_0958_gb300", "csrc", "vdf_backward.cu"), "rb") as fh:
        return hashlib.sha256(fh.read()).hexdigest()[:16]


def kernel_source_hash() -> str:
    h = hashlib.sha256()
    for f in ("vdf_tile.cuh", "vdf_internal.cuh", "vdf_fp32.cu", "vdf_fp32_inst.cuh", "vdf_dispatch.h"):
        with open(os.path.join(ROOT, "paper_1009_0958_gb300", "csrc", f), "rb") as fh:
            h.update(fh.read())
    return h.hexdigest()[:16]


def frames(count: int, seed0: int = 100):
    from paper_1009_0958_gb300 import synth
    return [synth.make_image(M, N, seed0 + i, NOISE, rectangles=RECTS)[1] for i in range(count)]


def dist_env():
    ws = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return ws, rank, local


def frame_seed(rank: int) -> int:
    """Replicas filter different frames: rank r uses seeds 100 + 1000 r + i."""
    return 100 + 1000 * rank


def reduce_max(value: float, world: int, device=None) -> float:
    """Max over ranks (the slowest replica sets the whole-job time)."""
    if world == 1:
        return value
    import torch
    import torch.distributed as dist
    t = torch.tensor([value], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def whole_job_rate(pixels_per_rank: int, world: int, max_ms: float) -> float:
    """Mpix/s of all ranks together over the slowest rank's time."""
    return world * pixels_per_rank / (max_ms * 1e-3) / 1e6


def measured_peaks():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as fh:
            return json.load(fh)
    except OSError:
        return {}


class ClockSampler:
    """nvidia-smi clock / throttle samples taken while the timed region runs."""

    Q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,clocks_event_reasons.hw_slowdown,"
         "clocks_event_reasons.hw_thermal_slowdown,clocks_event_reasons.sw_thermal_slowdown,"
         "clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index: int, interval_ms: int = 20):
        self.gpu = gpu_index
        self.interval = interval_ms
        self.proc = None
        self.path = None

    def __enter__(self):
        fd, self.path = tempfile.mkstemp(suffix=".csv")
        os.close(fd)
        try:
            self.fh = open(self.path, "w")
            self.proc = subprocess.Popen(["nvidia-smi", "-i", str(self.gpu), f"--query-gpu={self.Q}",
                                          "--format=csv,noheader,nounits", "-lms", str(self.interval)],
                                         stdout=self.fh, stderr=subprocess.DEVNULL)
        except (OSError, FileNotFoundError):
            self.proc = None
        return self

    def __exit__(self, *exc):
        if self.proc is not None:
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except subprocess.TimeoutExpired:
                self.proc.kill()
            self.fh.close()

    def summary(self):
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"], "samples": 0}
        rows = []
        with open(self.path) as fh:
            for line in fh:
                parts = [p.strip() for p in line.split(",")]
                if len(parts) >= 9:
                    rows.append(parts)
        os.unlink(self.path)
        if not rows:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["no samples"], "samples": 0}
        # samples taken while the GPU was busy: power well above idle, or the
        # SM clock at least half of its maximum
        sm = [float(r[1]) for r in rows if r[1].replace(".", "").isdigit()]
        mx = [float(r[2]) for r in rows if r[2].replace(".", "").isdigit()]
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        reasons = sorted({names[k] for r in rows for k in range(4) if r[5 + k].lower() == "active"})
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": max(mx) if mx else None,
                "reasons": reasons, "samples": len(rows)}


def cpu_oracle_rate(seconds_target: float = 12.0, sample_pixels: int | None = None):
    """Time the oracle on a pixel sample of one frame on all host cores."""
    import oracle
    oracle.build()
    img = frames(1)[0]
    cores = oracle.max_threads()
    rng = np.random.default_rng(0)
    # calibrate: ~0.5 s probe, then size the sample for the target time
    probe = rng.integers(0, M * N, 4000 * max(1, cores))
    t0 = time.perf_counter()
    oracle.filter_u8(img, WIN, FILTER, P, DIST, Q, pixels=probe)
    rate = len(probe) / (time.perf_counter() - t0)
    n = sample_pixels or int(min(M * N, max(10000, rate * seconds_target)))
    pix = rng.integers(0, M * N, n)
    t0 = time.perf_counter()
    oracle.filter_u8(img, WIN, FILTER, P, DIST, Q, pixels=pix)
    dt = time.perf_counter() - t0
    return {"value": n / dt / 1e6, "unit": UNIT, "cores": cores, "kind": "oracle",
            "sample": f"{n} random pixels of one {N}x{M} frame ({dt:.1f} s of CPU work, all cores)"}


def run_reference(args):
    ws, rank, _ = dist_env()
    if rank != 0:
        return
    import oracle
    oracle.build()
    img = frames(1)[0]
    cores = oracle.max_threads()
    rng = np.random.default_rng(1)
    # size each step so that warm-up + timed steps take about a minute
    probe = rng.integers(0, M * N, 2000 * max(1, cores))
    t0 = time.perf_counter()
    oracle.filter_u8(img, WIN, FILTER, P, DIST, Q, pixels=probe)
    rate = len(probe) / (time.perf_counter() - t0)
    per_step = int(min(65536, max(64, rate * 60.0 / (args.steps + args.warmup))))
    for _ in range(args.warmup):
        oracle.filter_u8(img, WIN, FILTER, P, DIST, Q, pixels=rng.integers(0, M * N, per_step))
    t0 = time.perf_counter()
    for _ in range(args.steps):
        oracle.filter_u8(img, WIN, FILTER, P, DIST, Q, pixels=rng.integers(0, M * N, per_step))
    dt = time.perf_counter() - t0
    value = per_step * args.steps / dt / 1e6
    line = {"metric": METRIC, "value": value, "unit": UNIT, "n_gpus": args.gpus, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": dt / args.steps * 1e3, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic", "config": CONFIG,
            "impl": "reference",
            "cpu_baseline": {"value": value, "unit": UNIT, "cores": cores, "kind": "oracle",
                             "sample": f"{per_step} random pixels of one {N}x{M} frame per step"},
            "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


def batch_images(count: int, seed: int):
    """The uneven-batch workload: sides log-uniform in [64, 2048] (aspect
    0.5-2), each image cropped from one of four 2048x2048 sinusoid fields,
    with 3 flat rectangles and 10% impulses of its own."""
    from paper_1009_0958_gb300 import synth
    bases = [synth.sinusoid_field(2048, 2048, seed + b) for b in range(4)]
    rng = np.random.default_rng(seed)
    out = []
    for k, (M, N) in enumerate(synth.batch_shapes(count, seed)):
        M, N = min(M, 2048), min(N, 2048)
        r0, c0 = int(rng.integers(0, 2048 - M + 1)), int(rng.integers(0, 2048 - N + 1))
        img = bases[k % 4][r0:r0 + M, c0:c0 + N]
        img = synth.add_rectangles(img, seed + 10 * k + 1, 3)
        out.append(synth.impulsive_noise(img, NOISE, seed + 10 * k + 2))
    return out


def run_vmf_workload(args):
    """The vector median filter of Eq. (1) (5x5) on the 1080p frames, at
    Minkowski orders 2 (the paper's), 1 and infinity: the FP32 path (with its
    FP64 recheck; none is needed at orders 1 and infinity, whose aggregates are
    exact integers) against the plain FP64 path, one call per frame."""
    import torch

    from paper_1009_0958_gb300 import build as vbuild
    from paper_1009_0958_gb300 import vdf
    vbuild.build()
    dev = torch.device("cuda", 0)
    ins = [torch.from_numpy(f).to(dev) for f in frames(FRAMES)]
    outs = [torch.empty_like(x) for x in ins]
    idxs = [torch.empty((M, N), dtype=torch.int8, device=dev) for _ in ins]
    wst = vdf.alloc_workspace(M, N, "fp32", dev)
    stream = torch.cuda.current_stream(dev)
    shape, _ = vdf.autotune(ins[0], WIN, "vmf", P, reps=5)
    K = args.steps

    def timed(order, prec, steps):
        for s in range(args.warmup):
            vdf.filter(ins[s % FRAMES], WIN, "vmf", precision=prec, out=outs[s % FRAMES], index=idxs[s % FRAMES],
                       workspace=wst, order=order)
        torch.cuda.synchronize(dev)
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        for s in range(steps):
            vdf.filter(ins[s % FRAMES], WIN, "vmf", precision=prec, out=outs[s % FRAMES], index=idxs[s % FRAMES],
                       workspace=wst, order=order)
        e1.record(stream)
        torch.cuda.synchronize(dev)
        return e0.elapsed_time(e1) / steps

    orders = {}
    with ClockSampler(0) as clk:
        for order in (2, 1, "inf"):
            ms = timed(order, "fp32", K)
            rechecked = vdf.workspace_stats(wst)[0]
            ms64 = timed(order, "fp64", max(3, min(K, 20)))
            orders[str(order)] = {"value": M * N / (ms * 1e-3) / 1e6, "ms_per_step": ms,
                                  "fp64_value": M * N / (ms64 * 1e-3) / 1e6, "speedup_vs_fp64": ms64 / ms,
                                  "rechecked_last_frame": rechecked}
    head = orders["2"]
    ops = opcount(WIN, "vmf")
    achieved = ops * M * N / (head["ms_per_step"] * 1e-3) / 1e12
    peak = SMS * FP32_LANES_PER_SM * 2.070e9 / 1e12
    roofline = {"bound": "alu", "achieved": achieved, "peak": peak, "unit": "T FP32-pipe ops/s",
                "frac": achieved / peak, "traffic": None,
                "kernel": "vdf::tile_kernel<R=2,VMF,order 2,FP32> (the whole call: counter reset, tile kernel, "
                          "recheck)", "ops_per_pixel": ops, "ops_basis": "opcount(5, 'vmf'): algorithmic count",
                "peak_basis": "152 SMs x 128 FP32 lanes x 2070 MHz max SM clock"}
    line = {"metric": "Mpix/s, 5x5 VMF (Eq. (1), Minkowski order 2) on 1080p RGB: FP32+FP64-tie path",
            "value": head["value"], "unit": UNIT, "n_gpus": 1, "steps": K, "warmup": args.warmup,
            "ms_per_step": head["ms_per_step"], "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
            "dtype": "f32+f64", "data": "synthetic",
            "config": {"workload": "VMF 5x5 on the 1920x1080 frames of the DDF workload (sinusoid field + 12 "
                                   "rectangles, 10% impulses), 24 frames (149 MB) in rotation", "M": M, "N": N,
                       "win": WIN, "tuned_shape": vdf.tile_shapes()[shape]},
            "orders": orders, "fp64_path": {"value": head["fp64_value"], "unit": UNIT},
            "speedup_vs_fp64": head["speedup_vs_fp64"], "gpu_launches": 2 * K, "roofline": roofline,
            "clocks": clk.summary()}
    print(json.dumps(line), flush=True)


def run_acwddf_workload(args):
    """The ACWDDF of Eq. (9) (Section 3.2, lambda = 2, T = 10.8) on the 1080p
    frames: 3x3 (the paper's window) in the three distance modes, and 5x5
    exact; the FP32 certified path (whole-pixel FP64 recheck where a decision
    is open) against the plain FP64 path, one call per frame."""
    import torch

    from paper_1009_0958_gb300 import build as vbuild
    from paper_1009_0958_gb300 import vdf
    vbuild.build()
    dev = torch.device("cuda", 0)
    ins = [torch.from_numpy(f).to(dev) for f in frames(FRAMES)]
    outs = [torch.empty_like(x) for x in ins]
    idxs = [torch.empty((M, N), dtype=torch.int8, device=dev) for _ in ins]
    wst = vdf.alloc_workspace(M, N, "fp32", dev)
    stream = torch.cuda.current_stream(dev)
    K = args.steps
    tuned = {}
    for win, dist in ((3, "exact"), (3, "minimax"), (3, "rgb"), (5, "exact")):
        shape, _ = vdf.autotune_acwddf(ins[0], win, dist, 4, 2, 10.8, reps=3, workspace=wst)
        tuned[f"{win}x{win} {dist}"] = vdf.tile_shapes()[shape]

    def timed(win, dist, prec, steps):
        def call(s):
            vdf.filter_acwddf(ins[s % FRAMES], win, dist, 4, 2, 10.8, precision=prec, out=outs[s % FRAMES],
                              index=idxs[s % FRAMES], workspace=wst)
        for s in range(args.warmup):
            call(s)
        torch.cuda.synchronize(dev)
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        for s in range(steps):
            call(s)
        e1.record(stream)
        torch.cuda.synchronize(dev)
        return e0.elapsed_time(e1) / steps

    cases = {}
    with ClockSampler(0) as clk:
        for win, dist in ((3, "exact"), (3, "minimax"), (3, "rgb"), (5, "exact")):
            ms = timed(win, dist, "fp32", K)
            rechecked = vdf.workspace_stats(wst)[0]
            ms64 = timed(win, dist, "fp64", max(3, min(K, 10)))
            cases[f"{win}x{win} {dist}"] = {"value": M * N / (ms * 1e-3) / 1e6, "ms_per_step": ms,
                                            "fp64_value": M * N / (ms64 * 1e-3) / 1e6,
                                            "speedup_vs_fp64": ms64 / ms, "rechecked_last_frame": rechecked}
    head = cases["3x3 exact"]
    ops = opcount_acwddf(3)
    achieved = ops * M * N / (head["ms_per_step"] * 1e-3) / 1e12
    peak = SMS * FP32_LANES_PER_SM * 2.070e9 / 1e12
    roofline = {"bound": "alu", "achieved": achieved, "peak": peak, "unit": "T FP32-pipe ops/s",
                "frac": achieved / peak, "traffic": None,
                "kernel": "vdf::tile_kernel<R=1,DDF,EXACT,FP32,ACW> (the whole call: counter reset, tile kernel, "
                          "recheck); ops: opcount_acwddf(3), the DDF, the CWVMF levels and the switch",
                "ops_per_pixel": ops, "peak_basis": "152 SMs x 128 FP32 lanes x 2070 MHz max SM clock"}
    line = {"metric": "Mpix/s, 3x3 ACWDDF (Eq. (9), lambda 2, T 10.8) on 1080p RGB: FP32+FP64-tie path",
            "value": head["value"], "unit": UNIT, "n_gpus": 1, "steps": K, "warmup": args.warmup,
            "ms_per_step": head["ms_per_step"], "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
            "dtype": "f32+f64", "data": "synthetic",
            "config": {"workload": "ACWDDF on the 1920x1080 frames of the DDF workload (sinusoid field + 12 "
                                   "rectangles, 10% impulses), 24 frames (149 MB) in rotation", "M": M, "N": N,
                       "lambda": 2, "T": 10.8, "tuned_shapes": tuned},
            "cases": cases, "fp64_path": {"value": head["fp64_value"], "unit": UNIT},
            "speedup_vs_fp64": head["speedup_vs_fp64"], "gpu_launches": 2 * K, "roofline": roofline,
            "clocks": clk.summary()}
    print(json.dumps(line), flush=True)


def run_batch_workload(args, emit: bool = True):
    """256 uneven images, mixed 3x3/5x5 BVDF/DDF, one persistent launch per
    batch replayed from a CUDA graph, tile shapes from the autotuner.  Returns
    the JSON line (printed when ``emit``)."""
    import torch

    from paper_1009_0958_gb300 import build as vbuild
    from paper_1009_0958_gb300 import vdf
    vbuild.build()
    dev = torch.device("cuda", 0)
    imgs = batch_images(256, 4242)
    rng = np.random.default_rng(7)
    cfgs = [(int(rng.choice([3, 5])), str(rng.choice(["bvdf", "ddf"]))) for _ in imgs]
    probe = torch.from_numpy(frames(1)[0]).to(dev)
    tuned = {}
    for win in (3, 5):
        for f in ("bvdf", "ddf"):
            tuned[f"{f}{win}x{win}"] = vdf.autotune(probe, win, f, P, reps=5)
    items = [dict(img=torch.from_numpy(x).to(dev), win=w, filter=f, p=P) for x, (w, f) in zip(imgs, cfgs)]
    plan = vdf.Plan(items)
    pixels = sum(int(x.shape[0]) * int(x.shape[1]) for x in imgs)
    stream = torch.cuda.current_stream(dev)
    for _ in range(args.warmup):
        plan.graph_launch()
    torch.cuda.synchronize(dev)
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    K = args.steps
    with ClockSampler(0) as clk:
        e0.record(stream)
        for _ in range(K):
            plan.graph_launch()
        e1.record(stream)
        torch.cuda.synchronize(dev)
    ms = e0.elapsed_time(e1) / K
    rechecked, overflow = plan.stats()
    ties = vdf.read_stats(plan.workspace)["structural_ties"]
    groups = len(set(cfgs))
    # the persistent work-queue form of the same plan, timed beside it
    plan_p = vdf.Plan(items, persistent=True)
    for _ in range(args.warmup):
        plan_p.graph_launch()
    Kp = max(3, min(K, 100))
    torch.cuda.synchronize(dev)
    e0.record(stream)
    for _ in range(Kp):
        plan_p.graph_launch()
    e1.record(stream)
    torch.cuda.synchronize(dev)
    ms_p = e0.elapsed_time(e1) / Kp
    plan_p.close()
    ops = sum(opcount(w, f) * int(x.shape[0]) * int(x.shape[1]) for x, (w, f) in zip(imgs, cfgs))
    achieved = ops / (ms * 1e-3) / 1e12
    peak = SMS * FP32_LANES_PER_SM * 2.070e9 / 1e12
    roofline = {"bound": "alu", "achieved": achieved, "peak": peak, "unit": "T FP32-pipe ops/s",
                "frac": achieved / peak, "traffic": None,
                "kernel": "vdf::batch_item_kernel (the step's time, which also holds the batch recheck kernel)",
                "ops_per_step": ops, "ops_basis": "sum over the images of opcount(win, filter) x pixels",
                "peak_basis": "152 SMs x 128 FP32 lanes x 2070 MHz max SM clock"}
    line = {"metric": "Mpix/s, batch of 256 uneven RGB images, mixed 3x3/5x5 BVDF/DDF, FP32+FP64-tie path",
            "value": pixels / (ms * 1e-3) / 1e6, "unit": UNIT, "n_gpus": 1, "steps": K, "warmup": args.warmup,
            "ms_per_step": ms, "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
            "dtype": "f32+f64", "data": "synthetic",
            "config": {"workload": "256 images, sides log-uniform [64, 2048], aspect 0.5-2, 10% impulses, "
                                   "win/filter uniform over {3,5} x {BVDF, DDF}, p = 0.25, exact arccos",
                       "pixels": pixels, "launch": "one tile kernel per configuration present (one CTA per "
                                                   "work item) + one recheck kernel per step, replayed from a "
                                                   "CUDA graph", "tuned_shapes": tuned},
            "persistent_form": {"value": pixels / (ms_p * 1e-3) / 1e6, "unit": UNIT, "ms_per_step": ms_p,
                                "steps": Kp, "launch": "the same plan with persistent tile kernels (CTAs take "
                                                       "work items from an atomic counter)"},
            "recheck_fraction": rechecked / pixels, "structural_tie_fraction": ties / pixels, "overflow": overflow,
            "gpu_launches": (groups + 1) * K, "roofline": roofline, "clocks": clk.summary()}
    if emit:
        print(json.dumps(line), flush=True)
    return line


def run_autograd_workload(args, emit: bool = True):
    """The differentiable workload: DDF 3x3 (p = 0.25) forward on a float32
    32 x 3 x 512 x 512 batch in [0, 1] (the FP32 certified path for float
    input, with its FP64 recheck) plus the gather-form backward; the backward
    kernel is HBM-bound at 25 B/px.  The plain FP64 forward is timed beside."""
    import torch

    from paper_1009_0958_gb300 import build as vbuild
    from paper_1009_0958_gb300 import synth, vdf
    vbuild.build()
    dev = torch.device("cuda", 0)
    B, Mf, Nf = 32, 512, 512
    field = np.stack([synth.make_image(Mf, Nf, 300 + b, NOISE)[1] for b in range(B)])
    x = torch.from_numpy(synth.to_float_nchw(field)).to(dev)
    gy = torch.randn_like(x)
    y, idx, gx = torch.empty_like(x), torch.empty((B, Mf, Nf), dtype=torch.int8, device=dev), torch.empty_like(x)
    stream = torch.cuda.current_stream(dev)

    ws = vdf.alloc_workspace(B * Mf, Nf, "fp32", dev)

    def step():
        vdf.filter_f32(x, 3, "ddf", P, precision="fp32", out=y, index=idx, workspace=ws)
        vdf.backward_f32(gy, idx, 3, grad_x=gx)
    for _ in range(args.warmup):
        step()
    K = max(3, min(args.steps, 20))
    ev = [[torch.cuda.Event(enable_timing=True) for _ in range(3)] for _ in range(K)]
    torch.cuda.synchronize(dev)
    with ClockSampler(0) as clk:
        for k in range(K):
            ev[k][0].record(stream)
            vdf.filter_f32(x, 3, "ddf", P, precision="fp32", out=y, index=idx, workspace=ws)
            ev[k][1].record(stream)
            vdf.backward_f32(gy, idx, 3, grad_x=gx)
            ev[k][2].record(stream)
        torch.cuda.synchronize(dev)
    fwd = statistics.mean(a.elapsed_time(b) for a, b, _ in ev)
    bwd = statistics.mean(b.elapsed_time(c) for _, b, c in ev)
    rechecked = vdf.workspace_stats(ws)[0]
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    vdf.filter_f32(x, 3, "ddf", P, precision="fp64", out=y, index=idx)
    e0.record(stream)
    for _ in range(3):
        vdf.filter_f32(x, 3, "ddf", P, precision="fp64", out=y, index=idx)
    e1.record(stream)
    torch.cuda.synchronize(dev)
    fwd64 = e0.elapsed_time(e1) / 3
    px = B * Mf * Nf
    bw = 25.0 * px / (bwd * 1e-3) / 1e9   # grad_y 12 B + index 1 B + grad_x 12 B per pixel
    hbm = measured_peaks().get("hbm_gbs") or 6800.0
    line = {"metric": "Mpix/s, DDF 3x3 forward + backward on float32 32x3x512x512 (differentiable path)",
            "value": px / ((fwd + bwd) * 1e-3) / 1e6, "unit": UNIT, "n_gpus": 1, "steps": K,
            "warmup": args.warmup, "ms_per_step": fwd + bwd, "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "f32+f64 forward, f32 backward", "data": "synthetic",
            "config": {"workload": "32 x 3 x 512 x 512 float32 in [0, 1]: sinusoid field / 255 + 10% impulses, "
                                   "DDF 3x3, p = 0.25, exact arccos"},
            "forward_ms": fwd, "backward_ms": bwd, "forward_fp64_ms": fwd64,
            "forward_recheck_fraction": rechecked / px,
            "roofline": {"bound": "hbm", "kernel": "vdf::backward_gather<R=1>", "achieved": bw,
                         "peak": hbm, "unit": "GB/s", "frac": bw / hbm,
                         "peak_basis": "measured copy bandwidth (MEASURED_PEAKS.json hbm_gbs)",
                         "traffic": BACKWARD_TRAFFIC_BY_SOURCE.get(backward_source_hash()),
                         "algorithmic_bytes_per_pixel": 25},
            "gpu_launches": 2 * K, "clocks": clk.summary()}
    if emit:
        print(json.dumps(line), flush=True)
    return line


def measure_frames(L, vdf, torch, dev, sp, stream, Mh, Nh, noise, nframes, seed0, K, warmup, shape_arg, K64,
                   ws, e2e_frames=0):
    """The FP32 certified step on ``nframes`` distinct Mh x Nh frames in
    rotation (the FP64 recheck of frame i on a second stream, three
    workspaces), then, untimed, its recheck and structural-tie counts per
    frame; the plain FP64 path on the first K64 frames; every pixel of those
    frames compared between the two precisions; optionally the end-to-end
    host-frame call over ``e2e_frames`` frames.  Times are max over ranks."""
    from paper_1009_0958_gb300 import synth
    host_frames = [synth.make_image(Mh, Nh, seed0 + i, noise, rectangles=RECTS)[1] for i in range(nframes)]
    ins = [torch.from_numpy(f).to(dev) for f in host_frames]
    outs = [torch.empty_like(x) for x in ins]
    idxs = [torch.empty((Mh, Nh), dtype=torch.int8, device=dev) for _ in ins]
    wsb = vdf.workspace_bytes(Mh, Nh, "fp32")
    wst = [torch.empty(wsb + 256, dtype=torch.uint8, device=dev) for _ in range(3)]
    wsp = [vdf._aligned(w) for w in wst]
    side = torch.cuda.Stream(dev)
    sp2 = ctypes.c_void_p(side.cuda_stream)
    VP = ctypes.c_void_p

    def check(rc):
        if rc != 0:
            raise RuntimeError(f"libvdf: {L.vdf_strerror(rc).decode()} {L.vdf_last_cuda_error().decode()}")

    def fp32_pass(x, o, ix, w=0):
        return L.vdf_fp32_pass(VP(x.data_ptr()), Mh, Nh, WIN, 1, P, 0, Q, VP(o.data_ptr()), VP(ix.data_ptr()),
                               wsp[w][0], wsp[w][1], sp)

    def recheck(x, o, ix, w=0, on_side=False):
        return L.vdf_fp64_recheck(VP(x.data_ptr()), Mh, Nh, WIN, 1, P, 0, Q, VP(o.data_ptr()), VP(ix.data_ptr()),
                                  wsp[w][0], wsp[w][1], sp2 if on_side else sp)

    def fp64_step(i):
        return L.vdf_filter(VP(ins[i].data_ptr()), Mh, Nh, WIN, 1, P, 0, Q, 0, VP(outs[i].data_ptr()),
                            VP(idxs[i].data_ptr()), None, None, 0, sp)

    def barrier():
        if ws > 1:
            torch.distributed.barrier()
        torch.cuda.synchronize(dev)

    if shape_arg is None:
        shape, _ = vdf.autotune(ins[0], WIN, FILTER, P, DIST, Q, reps=5)
    else:
        shape = shape_arg
        vdf.set_tuned_shape(WIN, FILTER, DIST, shape)
    tw, th = vdf.tile_shapes()[shape]
    for s in range(warmup):
        i = s % nframes
        check(fp32_pass(ins[i], outs[i], idxs[i]))
        check(recheck(ins[i], outs[i], idxs[i]))
    ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True),
           torch.cuda.Event(enable_timing=True)) for _ in range(K)]
    t_start, t_end = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    barrier()
    t_wall = time.perf_counter()
    t_start.record(stream)
    for s in range(K):
        i, w = s % nframes, s % 3
        if s >= 3:
            stream.wait_event(ev[s - 3][2])    # workspace w is free again
        ev[s][0].record(stream)
        check(fp32_pass(ins[i], outs[i], idxs[i], w))
        ev[s][1].record(stream)
        side.wait_event(ev[s][1])
        check(recheck(ins[i], outs[i], idxs[i], w, on_side=True))
        ev[s][2].record(side)
    stream.wait_event(ev[K - 1][2])
    t_end.record(stream)
    barrier()
    t_wall = time.perf_counter() - t_wall
    kernel_ms = [a.elapsed_time(b) for a, b, _ in ev]
    step_ms = [a.elapsed_time(c) for a, _, c in ev]
    total_ms = reduce_max(t_start.elapsed_time(t_end), ws, dev)

    # untimed: the FP32 path once more on the first frames (into spare
    # buffers), its counters per frame
    o32 = [torch.empty_like(ins[0]) for _ in range(K64)]
    i32 = [torch.empty_like(idxs[0]) for _ in range(K64)]
    rechecked, ties = [], []
    for i in range(min(nframes, K)):
        if i < K64:
            o, ix = o32[i], i32[i]
        else:
            o, ix = outs[i], idxs[i]
        check(fp32_pass(ins[i], o, ix))
        check(recheck(ins[i], o, ix))
        st = vdf.read_stats(wst[0])
        rechecked.append(st["rechecked"])
        ties.append(st["structural_ties"])

    # the plain FP64 GPU path (the metric's denominator)
    for s in range(3):
        check(fp64_step(s % nframes))
    barrier()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    for s in range(K64):
        check(fp64_step(s % nframes))
    e1.record(stream)
    barrier()
    fp64_ms = reduce_max(e0.elapsed_time(e1), ws, dev) / K64

    # every pixel of the frames both paths filtered: member index and RGB
    mism = 0
    for i in range(min(K64, nframes, K)):
        bad = (i32[i] != idxs[i]) | (o32[i] != outs[i]).any(dim=2)
        mism += int(bad.sum().item())
    compared = min(K64, nframes, K)

    res = {"total_ms": total_ms, "K": K, "kernel_ms": statistics.mean(kernel_ms),
           "step_ms_mean": statistics.mean(step_ms), "wall_s": t_wall, "shape": (tw, th),
           "fp64_ms": fp64_ms, "K64": K64,
           "recheck_fraction": float(np.mean(rechecked)) / (Mh * Nh) if rechecked else None,
           "structural_tie_fraction": float(np.mean(ties)) / (Mh * Nh) if ties else None,
           "mismatches_vs_fp64": mism, "frames_compared": compared}

    if e2e_frames:
        # vdf_filter_host_frames: frames from pinned host memory to pinned
        # host memory in one call; every frame's upload and download is inside
        # the timed region, overlapped with the filtering of its neighbours
        pin_in = [torch.from_numpy(f).pin_memory() for f in host_frames[:4]]
        pin_out = [torch.empty((Mh, Nh, 3), dtype=torch.uint8).pin_memory() for _ in range(2)]
        pin_idx = [torch.empty((Mh, Nh), dtype=torch.int8).pin_memory() for _ in range(2)]
        dbuf = torch.empty(vdf.host_frames_buffer_bytes(Mh, Nh, "fp32") + 256, dtype=torch.uint8, device=dev)
        bp, bl = vdf._aligned(dbuf)

        def e2e_call(count):
            a = (VP * count)(*[pin_in[s % 4].data_ptr() for s in range(count)])
            b = (VP * count)(*[pin_out[s % 2].data_ptr() for s in range(count)])
            c = (VP * count)(*[pin_idx[s % 2].data_ptr() for s in range(count)])
            return L.vdf_filter_host_frames(a, b, c, count, Mh, Nh, WIN, 1, P, 0, Q, 1, bp, bl, sp)
        check(e2e_call(3))
        barrier()
        t0 = time.perf_counter()
        check(e2e_call(e2e_frames))
        barrier()
        res["e2e_s"] = reduce_max(time.perf_counter() - t0, ws, dev)
        res["e2e_frames"] = e2e_frames
    return res


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=1000)
    ap.add_argument("--warmup", type=int, default=10)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-extras", action="store_true",
                    help="skip the 4K, batch and differentiable results added to the headline line")
    ap.add_argument("--fp64-steps", type=int, default=None)
    ap.add_argument("--workload", default="ddf5_1080p",
                    choices=["ddf5_1080p", "ddf5_4k", "batch", "autograd", "vmf5_1080p", "acwddf_1080p"])
    ap.add_argument("--shape", type=int, default=None, help="force this FP32 tile shape instead of autotuning")
    args = ap.parse_args()
    args.warmup = max(args.warmup, 3)
    if args.workload == "ddf5_4k":
        use_4k_workload()
    if args.impl == "reference":
        return run_reference(args)
    if args.workload == "batch":
        return run_batch_workload(args)
    if args.workload == "autograd":
        return run_autograd_workload(args)
    if args.workload == "vmf5_1080p":
        return run_vmf_workload(args)
    if args.workload == "acwddf_1080p":
        return run_acwddf_workload(args)

    import torch
    import torch.distributed as dist

    from paper_1009_0958_gb300 import build as vbuild
    from paper_1009_0958_gb300 import vdf

    ws, rank, local = dist_env()
    if ws > 1:
        dist.init_process_group("nccl", init_method="env://")
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    vbuild.build()
    L = vdf.lib()
    stream = torch.cuda.current_stream(dev)
    sp = ctypes.c_void_p(stream.cuda_stream)
    K = args.steps
    K64 = args.fp64_steps or max(3, min(K, 10))

    # clocks are sampled every 20 ms over the FP32 timed region, the FP64 leg
    # and the end-to-end leg (the FP32 region alone is a few milliseconds)
    Mh, Nh, metric, config = M, N, METRIC, dict(CONFIG)
    with ClockSampler(local) as clk:
        r = measure_frames(L, vdf, torch, dev, sp, stream, M, N, NOISE, FRAMES, frame_seed(rank), K, args.warmup,
                           args.shape, K64, ws, e2e_frames=max(3, min(K, 100)))
    clocks = clk.summary()
    clocks["span"] = "FP32 timed region + FP64 leg + end-to-end leg"
    value = whole_job_rate(K * Mh * Nh, ws, r["total_ms"])
    fp64_value = whole_job_rate(Mh * Nh, ws, r["fp64_ms"])
    e2e_value = whole_job_rate(r["e2e_frames"] * Mh * Nh, ws, r["e2e_s"] * 1e3)

    # ---- roofline of the dominant kernel (FP32 tile kernel) -----------------
    ops = opcount(WIN, FILTER, DIST)
    k_ms = r["kernel_ms"]
    achieved = ops * Mh * Nh / (k_ms * 1e-3) / 1e12
    peak = SMS * FP32_LANES_PER_SM * 2.070e9 / 1e12
    tw, th = r["shape"]
    roofline = {"bound": "alu", "achieved": achieved, "peak": peak, "unit": "T FP32-pipe ops/s",
                "frac": achieved / peak, "traffic": TRAFFIC_BY_SOURCE.get(kernel_source_hash()),
                "kernel": f"vdf::tile_kernel<R=2,DDF,EXACT,FP32,score slots> {tw}x{th} tile (autotuned)",
                "kernel_ms": k_ms,
                "ops_per_pixel": ops,
                "ops_basis": "opcount(5, 'ddf', 'exact'): 40 pair terms x (25 angle + 7 L2) + 600 aggregation "
                             "adds + 24 compares + 50 logs, fixed before tuning",
                "peak_basis": "nominal: 152 SMs x 128 FP32 lanes x 2070 MHz max SM clock",
                "sm_mhz_sampled": clocks.get("sm_mhz"),
                "hbm_gbs_achieved": 7.0 * Mh * Nh / (k_ms * 1e-3) / 1e9,
                "hbm_gbs_peak_measured": measured_peaks().get("hbm_gbs")}

    extras = {}
    saved = (M, N, NOISE, FRAMES, WORKLOAD, METRIC, CONFIG)
    if ws == 1 and not args.no_extras:
        Ke = max(3, min(K, 20))
        use_4k_workload()
        with ClockSampler(local) as clk4:
            r4 = measure_frames(L, vdf, torch, dev, sp, stream, M, N, NOISE, FRAMES, 100, Ke, args.warmup, args.shape,
                                max(3, min(Ke, 4)), ws)
        extras["ddf5_4k"] = {
            "workload": WORKLOAD, "value": Ke * M * N / (r4["total_ms"] * 1e-3) / 1e6, "unit": UNIT,
            "ms_per_step": r4["total_ms"] / Ke, "steps": Ke, "kernel_ms": r4["kernel_ms"],
            "fp64_value": M * N / (r4["fp64_ms"] * 1e-3) / 1e6, "speedup_vs_fp64": r4["fp64_ms"] * Ke / r4["total_ms"],
            "recheck_fraction": r4["recheck_fraction"], "structural_tie_fraction": r4["structural_tie_fraction"],
            "mismatches_vs_fp64": r4["mismatches_vs_fp64"], "frames_compared": r4["frames_compared"],
            "roofline_frac": opcount(WIN, FILTER, DIST) * M * N / (r4["kernel_ms"] * 1e-3) / 1e12 / peak,
            "clocks": clk4.summary()}
        ba = argparse.Namespace(steps=Ke, warmup=args.warmup)
        b = run_batch_workload(ba, emit=False)
        extras["batch"] = {k: b[k] for k in ("metric", "value", "unit", "ms_per_step", "steps", "recheck_fraction",
                                             "structural_tie_fraction", "gpu_launches", "clocks")}
        extras["batch"]["roofline_frac"] = b["roofline"]["frac"]
        extras["batch"]["persistent_form_value"] = b["persistent_form"]["value"]
        a = run_autograd_workload(ba, emit=False)
        extras["autograd"] = {k: a[k] for k in ("metric", "value", "unit", "ms_per_step", "steps", "forward_ms",
                                                "backward_ms", "forward_fp64_ms", "forward_recheck_fraction",
                                                "gpu_launches", "clocks")}
        extras["autograd"]["backward_roofline"] = a["roofline"]
    set_workload(*saved)

    if rank != 0:
        if ws > 1:
            dist.destroy_process_group()
        return
    cpu = None
    if not args.no_cpu_baseline and ws == 1:
        cpu = cpu_oracle_rate()
    line = {"metric": metric, "value": value, "unit": UNIT, "n_gpus": ws, "steps": K, "warmup": args.warmup,
            "ms_per_step": r["total_ms"] / K, "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
            "dtype": "f32+f64", "data": "synthetic", "config": config,
            "fp64_path": {"value": fp64_value, "unit": UNIT, "ms_per_step": r["fp64_ms"], "steps": K64},
            "speedup_vs_fp64": value / fp64_value,
            "mismatches_vs_fp64": r["mismatches_vs_fp64"],
            "mismatch_check": f"member index and RGB of every pixel of {r['frames_compared']} frames, FP32 path "
                              "(with its recheck) against the plain FP64 path",
            "recheck_fraction": r["recheck_fraction"], "structural_tie_fraction": r["structural_tie_fraction"],
            "step_ms_mean": r["step_ms_mean"], "wall_s": r["wall_s"],
            "pipelining": "FP64 recheck of frame i on a second stream overlaps the FP32 passes of frames "
                          "i+1 and i+2 (three workspaces)",
            "e2e": {"value": e2e_value, "unit": UNIT, "h2d_bytes_per_step": 3 * Mh * Nh,
                    "d2h_bytes_per_step": 4 * Mh * Nh, "steps": r["e2e_frames"],
                    "api": "vdf_filter_host_frames (pinned host frames in and out; uploads and downloads "
                           "overlapped with the filtering of neighbouring frames)"},
            "gpu_launches": 2 * K,
            "roofline": roofline, "cpu_baseline": cpu, "clocks": clocks}
    if extras:
        line["extra"] = extras
    print(json.dumps(line), flush=True)
    if ws > 1:
        dist.destroy_process_group()


if __name__ == "__main__":
    main()
