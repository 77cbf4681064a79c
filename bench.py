#!/usr/bin/env python3
"""Benchmark of the FLoD splatting path on GB300.

Workload (the headline configuration): the finest level of the 5-level scene -- 3,000,000
Gaussians (64 clusters, radius 20, SH degree 3, level-by-level initialised with Eq. 5 from
levels 1..4), one 1920x1080 pinhole camera at distance 40, upstream image gradient
N(0, 1e-3). A step is one training iteration of that level: preprocess, binning + radix
sort, forward blending, blending backward, preprocess backward (gradients to means, s_opt,
quaternions, opacity logits and SH). The forward-only frame rate is reported beside it.

``value`` = fwd+bwd iterations per second over all ranks (inputs resident in HBM; the 708 MB
parameter set and the per-step buffers exceed the 129 MB L2, so no flush is needed).
``e2e`` = the same through the Python API with the step's input (the upstream image
gradient) copied from pinned host memory and the rendered image read back, every step; the
copies run on a second stream, double-buffered, overlapped with the neighbouring steps.
``--impl reference`` times the FP64 CPU oracle on a bounded sample of the same step.

Launch: python bench.py [--gpus N --steps K --warmup W]; for N > 1 under torchrun each rank
runs an independent replica (the path has no exchange step).
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

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "1080p frames/s fwd & fwd+bwd it/s (3M Gaussians), batched vs per-view"
WORKLOAD = "FLoD 5-level scene, level 5 (3M Gaussians, SH3), 1920x1080, fwd+bwd per level"
# peak of plain float32 ALU work: 152 SMs x 128 FP32 lanes x 2 (FMA) x 2070 MHz
ALU_PEAK_TFLOPS = 152 * 128 * 2 * 2.070e9 / 1e12
# FP32 operations (an FFMA counts 2) of the blending kernels: per evaluated (pixel, Gaussian)
# pair -- the offset, q and its threshold test, with the per-column terms shared by the
# thread's pixels -- and on top for each pair the forward blended (alpha, transmittance,
# colour; backward: T recovery, colour, alpha and moment gradients). The nine-value warp
# reduction is overhead, not counted.
FLOP_FWD_EVAL, FLOP_FWD_BLEND = 8, 13
FLOP_BWD_EVAL, FLOP_BWD_BLEND = 7, 31


def measured_traffic(kernel: str):
    """DRAM bytes per launch of `kernel` from its committed full-size ncu summary, or None when
    there is none or the kernel's sources changed since the counters were taken."""
    import hashlib
    path = os.path.join(ROOT, "profiles", f"{kernel}_dram_level5_3M_1080p.md")
    if not os.path.exists(path):
        return None
    fields = {}
    for line in open(path):
        if ":" in line and not line.startswith(("|", "#", " ")):
            k, v = line.split(":", 1)
            fields[k.strip()] = v.strip()
    try:
        srcs = [p.strip() for p in fields["sources"].split(",")]
        sha = hashlib.sha256(b"".join(open(os.path.join(ROOT, p), "rb").read() for p in srcs)).hexdigest()
        return int(fields["traffic_bytes_per_launch"]) if sha == fields["sources_sha256"] else None
    except (KeyError, OSError, ValueError):
        return None


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=200)
    ap.add_argument("--warmup", type=int, default=5)
    ap.add_argument("--impl", default="flod", choices=["flod", "reference"])
    ap.add_argument("--small", action="store_true", help="300k-Gaussian level (smoke runs)")
    ap.add_argument("--scale", type=float, default=1.0,
                    help="multiply every level count (profiling cases; not a bench line)")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-selective", action="store_true", help="skip the selective-rendering section")
    ap.add_argument("--no-batched", action="store_true", help="skip the batched multi-view section")
    ap.add_argument("--batched-views", type=int, default=64)
    return ap.parse_args()


# ---------------------------------------------------------------------------------------
# workload
# ---------------------------------------------------------------------------------------

def level_counts(small: bool, scale: float = 1.0):
    from paper_2408_12894_gb300 import synth
    base = (2_000, 8_000, 30_000, 100_000, 300_000) if small else synth.LEVEL_COUNTS
    return tuple(int(round(c * scale)) for c in base)


def make_level(small: bool, scale: float = 1.0):
    """Numpy arrays of the finest level (s_opt as drawn: Eq. 5 is applied on the device)."""
    from paper_2408_12894_gb300 import synth
    levels = synth.level_scene(counts=level_counts(small, scale))
    return levels[-1][0]


def clock_sampler(dev_index: int):
    """Samples SM clocks and throttle reasons with nvidia-smi while running."""
    q = ("clocks.sm,clocks.max.sm,clocks_event_reasons.active,clocks_event_reasons.hw_slowdown,"
         "clocks_event_reasons.hw_thermal_slowdown,clocks_event_reasons.sw_thermal_slowdown,"
         "clocks_event_reasons.sw_power_cap")
    try:
        p = subprocess.Popen(["nvidia-smi", "-i", str(dev_index), f"--query-gpu={q}",
                              "--format=csv,noheader,nounits", "-lms", "50"],
                             stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
    except OSError:
        return None
    rows = []

    def pump():
        for line in p.stdout:
            rows.append([x.strip() for x in line.split(",")])

    th = threading.Thread(target=pump, daemon=True)
    th.start()
    return p, th, rows


def clock_summary(s):
    if s is None:
        return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
    p, th, rows = s
    p.terminate()
    try:
        p.wait(timeout=5)
    except subprocess.TimeoutExpired:
        p.kill()
    th.join(timeout=2)
    sm, mx, reasons = [], [], set()
    names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
    for r in rows:
        try:
            sm.append(float(r[0]))
            mx.append(float(r[1]))
        except (ValueError, IndexError):
            continue
        for n, v in zip(names, r[3:7]):
            if v.strip().lower() == "active":
                reasons.add(n)
    return {"sm_mhz": statistics.median(sm) if sm else None,
            "sm_max_mhz": max(mx) if mx else None, "reasons": sorted(reasons),
            "samples": len(sm)}


# ---------------------------------------------------------------------------------------
# CPU oracle timing (the reference arm and the cpu_baseline key)
# ---------------------------------------------------------------------------------------

def cpu_model() -> str:
    """The host CPU's model name (lscpu, else /proc/cpuinfo, else platform)."""
    import platform
    try:
        out = subprocess.run(["lscpu"], capture_output=True, text=True, timeout=10).stdout
        for line in out.splitlines():
            if line.strip().startswith("Model name:"):
                return line.split(":", 1)[1].strip()
    except (OSError, subprocess.SubprocessError):
        pass
    try:
        for line in open("/proc/cpuinfo"):
            if line.lower().startswith("model name"):
                return line.split(":", 1)[1].strip()
    except OSError:
        pass
    return platform.processor() or platform.machine()


class OracleStep:
    """Times the FP64 oracle on a bounded sample of one training step and scales it to the
    full step: preprocess forward+backward and binning on a slice of the Gaussians (scaled by
    N / slice) plus blending forward+backward on a stratified sample of tiles. The tiles are
    ordered by pair count and cut into `tiles` strata of equal size; the middle tile of each
    stratum is timed and stands for its stratum. The tile lists come from an untimed FP64
    preprocess of the whole level. The sample depends only on the workload, so every arm and
    every run times the same work."""

    def __init__(self, g, cam, s_min, slice_n=20_000, tiles=64):
        import numpy as np
        import torch
        from oracle import raster as R
        self.R, self.np, self.torch = R, np, torch
        self.g, self.cam, self.s_min = g, cam, s_min
        self.cfg = R.Config()
        self.n = g["means"].shape[0]
        self.slice_n = min(slice_n, self.n)
        with torch.no_grad():
            pre = R.preprocess(R.params(g), 3, s_min, cam, self.cfg)
        self.pre = {k: pre[k] for k in ("mean2d", "conic", "opacity", "rgb")}
        self.lists = R.tile_lists(pre, cam, self.cfg)
        ranges = self.lists[2]
        counts = ranges[:, 1] - ranges[:, 0]
        order = np.argsort(counts, kind="stable")
        strata = np.array_split(order, min(tiles, order.size))
        self.sample = np.array([st[st.size // 2] for st in strata])
        self.weight = np.array([st.size for st in strata], dtype=np.float64)
        self.sample_pairs = counts[self.sample]
        self.n_tiles = ranges.shape[0]
        rng = np.random.default_rng(11)
        self.grad_out = rng.normal(0, 1e-3, (3, cam["height"], cam["width"]))

    def step_seconds(self, threads=None) -> float:
        R, np, torch = self.R, self.np, self.torch
        prev = torch.get_num_threads()
        if threads:
            torch.set_num_threads(threads)
        try:
            return self._step()
        finally:
            torch.set_num_threads(prev)

    def _step(self) -> float:
        R, np, torch = self.R, self.np, self.torch
        sub = {k: (v[:self.slice_n] if k != "sh_degree" else v) for k, v in self.g.items()}
        t0 = time.perf_counter()
        p = R.params(sub, requires_grad=True)
        pre = R.preprocess(p, 3, self.s_min, self.cam, self.cfg)
        k, v = R.bin_segments(pre["segments"], pre["depth"].detach().numpy(), self.lists[3],
                              self.n_tiles)
        R.sort_pairs(k, v)
        outs = [pre[n] for n in ("mean2d", "conic", "opacity", "rgb")]
        torch.autograd.backward(outs, [torch.ones_like(o) for o in outs])
        t_slice = time.perf_counter() - t0
        keys, vals, ranges, tx, ty = self.lists
        leaves = {n: self.pre[n].detach().clone().requires_grad_(True) for n in self.pre}
        bg = torch.zeros(3, dtype=torch.float64)
        t_tiles = 0.0
        for tile, w in zip(self.sample, self.weight):
            t0 = time.perf_counter()
            s, e = ranges[tile]
            if e > s:
                gi = torch.as_tensor(vals[s:e].astype(np.int64))
                x0, y0, x1, y1 = R.tile_pixels(int(tile), tx, self.cam, self.cfg)
                gx, gy = np.meshgrid(np.arange(x0, x1), np.arange(y0, y1))
                pix = torch.as_tensor(np.stack([gx.ravel() + 0.5, gy.ravel() + 0.5], 1))
                a = R.alpha_raw(pix, leaves["mean2d"][gi], leaves["conic"][gi], leaves["opacity"][gi])
                col, _, _ = R.blend(a, leaves["rgb"][gi], bg)
                go = torch.as_tensor(self.grad_out[:, y0:y1, x0:x1].reshape(3, -1).T)
                (col * go).sum().backward()
            t_tiles += (time.perf_counter() - t0) * w
        return t_slice * self.n / self.slice_n + t_tiles

    def describe(self) -> str:
        np = self.np
        return (f"preprocess fwd+bwd and binning of {self.slice_n} of {self.n} Gaussians "
                f"(x{self.n / self.slice_n:.0f}) + blend fwd+bwd of {len(self.sample)} of "
                f"{self.n_tiles} 16x16 tiles, one per equal-size stratum of the tiles ordered by "
                f"pair count (pairs {int(self.sample_pairs.min())}..{int(self.sample_pairs.max())}, "
                f"median {int(np.median(self.sample_pairs))}), each standing for its stratum")


def cpu_baseline_line(ost, value_all=None):
    """The cpu_baseline object: the oracle sample on every host core and on one."""
    import torch
    cores = os.cpu_count() or 1
    t_all = ost.step_seconds(threads=cores) if value_all is None else 1.0 / value_all
    t_one = ost.step_seconds(threads=1)
    return {"value": 1.0 / t_all, "unit": "it/s", "cores": cores, "kind": "oracle",
            "value_1_thread": 1.0 / t_one, "cpu_model": cpu_model(),
            "torch_threads_default": torch.get_num_threads(), "sample": ost.describe()}


def run_reference(a):
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    if rank != 0:
        return
    import torch
    from paper_2408_12894_gb300 import synth
    g = make_level(a.small, a.scale)
    g["s_opt"] = adjust_chain_numpy(g["s_opt"], level_counts(a.small, a.scale))
    cam = synth.level_camera()
    # each step times the same bounded sample as the main arm's cpu_baseline, on every core
    ost = OracleStep(g, cam, synth.LEVEL_SMIN[-1])
    cores = os.cpu_count() or 1
    for _ in range(a.warmup):
        ost.step_seconds(threads=cores)
    secs = [ost.step_seconds(threads=cores) for _ in range(a.steps)]
    mean = sum(secs) / len(secs)
    v = 1.0 / mean
    line = {"impl": "reference", "metric": METRIC, "value": v, "unit": "it/s", "n_gpus": world,
            "steps": a.steps, "warmup": a.warmup, "ms_per_step": 1e3 * mean,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
            "data": "synthetic", "config": {"workload": WORKLOAD, "gaussians": g["means"].shape[0],
                                            "resolution": "1920x1080", "sh_degree": 3},
            "cpu_baseline": {"value": v, "unit": "it/s", "cores": cores, "kind": "oracle",
                             "cpu_model": cpu_model(), "sample": ost.describe()},
            "e2e": {"value": v, "unit": "it/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


def adjust_chain_numpy(s_opt, counts):
    """Eq. 5 chain for the oracle arm (FP64): Gaussians present at level l are moved from
    level l's constraint to level l+1's, l = 1..4."""
    import numpy as np
    import torch
    from oracle import gaussians as OG
    from paper_2408_12894_gb300 import synth
    s = torch.as_tensor(s_opt.astype(np.float64))
    for l in range(4):
        s[:counts[l]] = OG.adjust_scale(s[:counts[l]], synth.LEVEL_SMIN[l], synth.LEVEL_SMIN[l + 1])
    return s.numpy().astype(np.float32)


# ---------------------------------------------------------------------------------------
# GPU arm
# ---------------------------------------------------------------------------------------

def run_flod(a):
    import numpy as np
    import torch
    from paper_2408_12894_gb300 import replicas
    rank, world, local = replicas.world()
    torch.cuda.set_device(local)
    dist = None
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl")
    from paper_2408_12894_gb300 import _build, flod, synth
    _build.build()
    counts = level_counts(a.small, a.scale)
    g = make_level(a.small, a.scale)
    gs = flod.GaussianSet.from_numpy(g, synth.LEVEL_SMIN[-1])
    for l in range(4):   # level-by-level initialisation (Eq. 5), on the device
        flod.flod_adjust_scale(gs.s_opt[:counts[l]], synth.LEVEL_SMIN[l], synth.LEVEL_SMIN[l + 1])
    cam = synth.level_camera()
    view = flod.view_struct(cam)
    rast = flod.Rasterizer([gs], [view])
    rgb, T, nc = rast.forward()                    # sizes the pair capacity once
    torch.cuda.synchronize()
    pairs = int(rast.pair_count.item())
    rast.pair_capacity = int(pairs * 1.2) + 4096
    rast._alloc()
    H, W = cam["height"], cam["width"]
    dL_host = torch.as_tensor(synth.upstream_gradient(11, [cam])).pin_memory()
    dL = dL_host.to("cuda")
    grads = [[torch.zeros_like(getattr(gs, f)) for f in flod.GaussianSet.FIELDS]]
    # one view renders the level: the backward writes every gradient (no zero-fill needed)
    grads_c = flod.grads_struct(grads, overwrite=True)
    st = torch.cuda.current_stream()

    def fwd():
        rast.preprocess()
        rast.bin_sort()
        rast.render_fwd(rgb, T, nc)

    def step(ev=None, ev_blend=None):
        # ev: events at every stage boundary; ev_blend: only around the two blending stages
        if ev:
            ev[0].record(st)
        rast.preprocess()
        if ev:
            ev[1].record(st)
        rast.bin_sort()
        if ev:
            ev[2].record(st)
        if ev_blend:
            ev_blend[0].record(st)
        rast.render_fwd(rgb, T, nc)
        if ev:
            ev[3].record(st)
            ev[4].record(st)
        if ev_blend:
            ev_blend[1].record(st)
        rast.blend_bwd(dL, T, nc)
        if ev:
            ev[5].record(st)
        if ev_blend:
            ev_blend[2].record(st)
        rast.preprocess_bwd(grads_c)
        if ev:
            ev[6].record(st)

    for _ in range(max(a.warmup, 3)):
        step()
    torch.cuda.synchronize()
    assert flod.flod_read_status(rast.ws) == 0, "device status error"

    def barrier():
        replicas.barrier()

    # ---- forward frames
    barrier()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record(st)
    for _ in range(a.steps):
        fwd()
    e1.record(st)
    barrier()
    fwd_ms = e0.elapsed_time(e1) / a.steps

    # ---- fwd+bwd training steps (the headline): K steps between two events; inside, events
    # only around the two blending stages (the roofline kernels, timed live here)
    clk = clock_sampler(local)
    ev_before = rast.eval_counts()
    evb = [[torch.cuda.Event(enable_timing=True) for _ in range(3)] for _ in range(a.steps)]
    h0, h1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    barrier()
    t_wall = time.perf_counter()
    h0.record(st)
    for i in range(a.steps):
        step(ev_blend=evb[i])
    h1.record(st)
    barrier()
    t_wall = time.perf_counter() - t_wall
    clocks = clock_summary(clk)
    ev_after = rast.eval_counts()
    ms = h0.elapsed_time(h1) / a.steps
    blend_ms = {"render_fwd": sum(e[0].elapsed_time(e[1]) for e in evb) / a.steps,
                "blend_bwd": sum(e[1].elapsed_time(e[2]) for e in evb) / a.steps}
    # ---- the same steps again with events at every stage boundary (stage times and the
    # per-step spread; not the headline)
    evs = [[torch.cuda.Event(enable_timing=True) for _ in range(7)] for _ in range(a.steps)]
    for i in range(a.steps):
        step(evs[i])
    torch.cuda.synchronize()
    step_ms = [evs[i][0].elapsed_time(evs[i][6]) for i in range(a.steps)]
    names = ["preprocess", "bin_sort", "render_fwd", "(none)", "blend_bwd", "preprocess_bwd"]
    stage_ms = {n: sum(evs[i][j].elapsed_time(evs[i][j + 1]) for i in range(a.steps)) / a.steps
                for j, n in enumerate(names) if n != "(none)"}
    ms, fwd_ms = replicas.max_over_ranks([ms, fwd_ms], device="cuda")

    # ---- end to end: upstream gradient in from pinned host memory, image back, every step.
    # The copies run on a second stream, double-buffered: step i+1's gradient is copied in
    # while step i computes, and step i's image is copied out while its backward runs.
    cs = torch.cuda.Stream()
    dLs, rgbs = [dL, torch.empty_like(dL)], [rgb, torch.empty_like(rgb)]
    img_hosts = [torch.empty(3 * H * W, dtype=torch.float32).pin_memory() for _ in range(2)]
    ev_in = [torch.cuda.Event() for _ in range(2)]     # gradient j is on the device
    ev_used = [torch.cuda.Event() for _ in range(2)]   # the backward that read gradient j ended
    ev_img = [torch.cuda.Event() for _ in range(2)]    # image j is rendered
    ev_out = [torch.cuda.Event() for _ in range(2)]    # image j is on the host

    def e2e_step(i):
        j = i % 2
        st.wait_event(ev_in[j])
        if i + 1 < a.steps:
            if i >= 1:
                cs.wait_event(ev_used[1 - j])
            with torch.cuda.stream(cs):
                dLs[1 - j].copy_(dL_host, non_blocking=True)
                ev_in[1 - j].record(cs)
        if i >= 2:
            st.wait_event(ev_out[j])
        rast.preprocess()
        rast.bin_sort()
        rast.render_fwd(rgbs[j], T, nc)
        ev_img[j].record(st)
        rast.blend_bwd(dLs[j], T, nc)
        ev_used[j].record(st)
        rast.preprocess_bwd(grads_c)
        cs.wait_event(ev_img[j])
        with torch.cuda.stream(cs):
            img_hosts[j].copy_(rgbs[j], non_blocking=True)
            ev_out[j].record(cs)

    barrier()
    e2e0, e2e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e2e0.record(st)
    cs.wait_event(e2e0)
    with torch.cuda.stream(cs):
        dLs[0].copy_(dL_host, non_blocking=True)
        ev_in[0].record(cs)
    for i in range(a.steps):
        e2e_step(i)
    st.wait_stream(cs)
    e2e1.record(st)
    barrier()
    e2e_ms = e2e0.elapsed_time(e2e1) / a.steps
    e2e_ms, = replicas.max_over_ranks([e2e_ms], device="cuda")

    fwd_evals = (ev_after[0] - ev_before[0]) / a.steps
    bwd_evals = (ev_after[1] - ev_before[1]) / a.steps
    blended = (ev_after[2] - ev_before[2]) / a.steps
    kernels = {"render_fwd": (blend_ms["render_fwd"],
                              fwd_evals * FLOP_FWD_EVAL + blended * FLOP_FWD_BLEND),
               "blend_bwd": (blend_ms["blend_bwd"],
                             bwd_evals * FLOP_BWD_EVAL + blended * FLOP_BWD_BLEND)}
    dom = max(kernels, key=lambda k: kernels[k][0])
    d_ms, d_flop = kernels[dom]
    achieved = d_flop / (d_ms * 1e-3) / 1e12
    n_tiles = int(rast.layout.tiles)
    n_passes = (max(1, math.ceil(math.log2(max(n_tiles, 2)))) + 8) // 9   # 9-bit tile digits
    # preprocess 2 (status clear, preprocess); bin_sort: visible counts, their scan, unit
    # keys, 4 depth passes of 3 kernels (count, scan, scatter; a pass above the keys'
    # significant bits exits at once), block sums, scan, light, big-unit and sliced emission,
    # n_passes tile passes of 3, ranges; render_fwd 1; blend_bwd 2 (2D-gradient zero-fill,
    # blend); preprocess_bwd 1
    launches_per_step = 2 + (3 + 12 + 2 + 3 + 3 * n_passes + 1) + 1 + 2 + 1

    if rank == 0:
        line = {
            "metric": METRIC, "value": world * 1e3 / ms, "unit": "it/s", "n_gpus": world,
            "steps": a.steps, "warmup": a.warmup, "ms_per_step": ms,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f32",
            "data": "synthetic",
            "config": {"workload": WORKLOAD, "gaussians": int(gs.n), "resolution": f"{W}x{H}",
                       "sh_degree": 3, "tile": "16x16", "pairs_per_step": pairs,
                       "l2": "inputs larger than L2 (708 MB parameters, no flush)",
                       "parallelism": f"replicas x{world}"},
            "fwd_fps": world * 1e3 / fwd_ms, "fwd_ms": fwd_ms,
            "stage_ms": {k: round(v, 4) for k, v in stage_ms.items()},
            "step_ms_median": statistics.median(step_ms),
            "wall_ms_per_step": 1e3 * t_wall / a.steps,
            "evals_per_step": {"fwd": fwd_evals, "bwd": bwd_evals, "blended": blended},
            "roofline": {"kernel": dom, "bound": "alu", "achieved": achieved,
                         "peak": ALU_PEAK_TFLOPS, "unit": "TFLOP/s",
                         "frac": achieved / ALU_PEAK_TFLOPS,
                         "traffic": measured_traffic("k_render_bwd") if dom == "blend_bwd" else None,
                         "peak_source": "152 SMs x 128 FP32 lanes x 2 x 2070 MHz (derived)"},
            "e2e": {"value": world * 1e3 / e2e_ms, "unit": "it/s",
                    "h2d_bytes_per_step": int(dL.numel() * 4),
                    "d2h_bytes_per_step": int(rgb.numel() * 4)},
            "gpu_launches": launches_per_step * a.steps,
            "clocks": clocks,
        }
        if not a.no_selective:
            line["selective"] = selective_section(a)
        if not a.no_batched:
            line["batched"] = batched_section(a)
        if not a.no_cpu_baseline and world == 1:
            try:
                g_np = dict(g)
                g_np["s_opt"] = gs.s_opt.cpu().numpy()
                ost = OracleStep(g_np, cam, synth.LEVEL_SMIN[-1])
                sec = ost.step_seconds()
                line["cpu_baseline"] = {"value": 1.0 / sec, "unit": "it/s",
                                        "cores": torch.get_num_threads(), "kind": "oracle",
                                        "sample": ost.describe()}
            except Exception as ex:   # report, never hide
                line["cpu_baseline"] = {"value": None, "unit": "it/s", "kind": "oracle",
                                        "error": repr(ex)}
        print(json.dumps(line), flush=True)
    if dist is not None:
        dist.destroy_process_group()


def timed(fn, steps, warmup):
    """Mean ms of fn() over `steps` calls on the current stream (CUDA events)."""
    import torch
    for _ in range(warmup):
        fn()
    torch.cuda.synchronize()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record()
    for _ in range(steps):
        fn()
    e1.record()
    torch.cuda.synchronize()
    return e0.elapsed_time(e1) / steps


def selective_sets(scale: float = 1.0):
    """The selective scene: the 5-level scene stretched x5 (positions and minimum scales)."""
    from paper_2408_12894_gb300 import flod, synth
    counts = tuple(int(round(c * scale)) for c in synth.LEVEL_COUNTS)
    levels = synth.stretch_levels(synth.level_scene(counts=counts), 5.0)
    sets = [flod.GaussianSet.from_numpy(g, 5.0 * s) for (g, _), s in zip(levels, synth.LEVEL_SMIN)]
    for l in range(4):
        flod.flod_adjust_scale(sets[4].s_opt[:counts[l]], 5 * synth.LEVEL_SMIN[l], 5 * synth.LEVEL_SMIN[l + 1])
        for k in range(l + 1, 4):
            flod.flod_adjust_scale(sets[k].s_opt[:counts[l]], 5 * synth.LEVEL_SMIN[l], 5 * synth.LEVEL_SMIN[l + 1])
    return sets


def selective_section(a):
    """Per-view selective rendering (Eq. 6 per frame from the camera position) along the
    32-frame path, forward only, at 1920x1080 and 3840x2160."""
    import torch
    from paper_2408_12894_gb300 import flod, multiview, synth
    sets = selective_sets(a.scale)
    th = list(synth.SELECTIVE_THRESHOLDS[::-1])
    out = {"workload": "5-level scene x5 (radius 100), thresholds {10,25,50,100}, 32-frame path, "
                       "per-view selection every frame, forward", "resolutions": {}}
    for (w, h) in ((1920, 1080), (3840, 2160)):
        path = synth.camera_path(width=w, height=h)
        st = multiview.BatchedStep(sets, [multiview.Job(path[0], levels=[0, 1, 2, 3, 4], thresholds=th)],
                                   flod.default_config())
        # size the pairs for the whole path and record the selected working set per frame
        need, sel = 0, []
        for cam in path:
            st.set_camera(0, cam)
            need = max(need, st.size_capacity())
            sel.append(st.selected_count(0))
        st.rast.pair_capacity = int(need * 1.1) + 4096
        st.rast._alloc()
        st.set_camera(0, path[0])
        frames = [0]

        def frame():
            st.set_camera(0, path[frames[0] % len(path)])
            frames[0] += 1
            st.run()
        ms = timed(frame, max(a.steps, len(path)), 3)
        units = st.rast.layout.units
        per_frame_bytes = [int(n * (236 + 84) + units * 4 + st.rast.pair_capacity * 16 + w * h * 20)
                           for n in sel]
        out["resolutions"][f"{w}x{h}"] = {
            "fps": 1e3 / ms, "ms_per_frame": ms,
            "selected_per_frame": {"min": min(sel), "max": max(sel), "mean": sum(sel) / len(sel)},
            "selected_param_bytes_per_frame_mean": 236 * sum(sel) / len(sel),
            "working_set_bytes_per_frame_max": max(per_frame_bytes),
            "all_levels_param_bytes": 236 * sum(s.n for s in sets)}
        del st
        torch.cuda.empty_cache()
    del sets
    torch.cuda.empty_cache()
    return out


def batched_section(a):
    """64 cameras of mixed resolution, each rendering one level of the 5-level scene or the
    per-view selective mix of the stretched scene, forward+backward: one autotuned,
    persistent, graph-captured batch vs the same jobs as 64 per-view calls (16x16 tiles,
    one CTA per tile, eager)."""
    import torch
    from paper_2408_12894_gb300 import flod, multiview, synth
    sel_sets = selective_sets(a.scale)
    counts = tuple(int(round(c * a.scale)) for c in synth.LEVEL_COUNTS)
    levels = synth.level_scene(counts=counts)
    lvl_sets = []
    for li, (g, _) in enumerate(levels):
        s = flod.GaussianSet.from_numpy(g, synth.LEVEL_SMIN[li])
        for l in range(li):
            flod.flod_adjust_scale(s.s_opt[:counts[l]], synth.LEVEL_SMIN[l], synth.LEVEL_SMIN[l + 1])
        lvl_sets.append(s)
    sets = sel_sets + lvl_sets
    cams, job_ids = synth.batched_jobs(n_cams=a.batched_views)
    th = list(synth.SELECTIVE_THRESHOLDS[::-1])
    jobs = [multiview.Job(c, levels=[0, 1, 2, 3, 4], thresholds=th) if j == 5
            else multiview.Job(c, set_index=5 + j) for c, j in zip(cams, job_ids)]
    dL = torch.as_tensor(synth.upstream_gradient(11, cams), device="cuda")
    t0 = time.perf_counter()
    cfg, times = multiview.autotune(sets, jobs, backward=True, dL=dL, steps=2)
    tune_s = time.perf_counter() - t0
    st = multiview.BatchedStep(sets, jobs, cfg, backward=True, dL=dL)
    pairs = st.size_capacity()
    st.capture()
    ms_batched = timed(st.replay, max(3, a.steps // 4), 2)
    del st
    torch.cuda.empty_cache()
    # the same jobs as per-view calls of the plain rasterizer
    singles = []
    off = 0
    for j in jobs:
        n = 3 * j.cam["width"] * j.cam["height"]
        s1 = multiview.BatchedStep(sets, [j], flod.default_config(), backward=True, dL=dL[off:off + n])
        s1.size_capacity()
        singles.append(s1)
        off += n

    def per_view():
        for s1 in singles:
            s1.run()
    ms_single = timed(per_view, max(3, a.steps // 4), 1)
    res = {"workload": f"{len(jobs)} views, resolutions {{640x480,1280x720,1920x1080,3840x2160}}, "
                       "jobs {levels 1..5, per-view selective}, fwd+bwd",
           "views": len(jobs), "pixels": int(sum(c["width"] * c["height"] for c in cams)),
           "pairs": pairs, "batched_ms": ms_batched, "per_view_ms": ms_single,
           "batched_views_per_s": len(jobs) * 1e3 / ms_batched,
           "per_view_views_per_s": len(jobs) * 1e3 / ms_single,
           "speedup": ms_single / ms_batched,
           "autotuned": {"tile": f"{cfg.tile_w}x{cfg.tile_h}", "batch": cfg.batch,
                         "tuning_s": tune_s,
                         "candidates_ms": {f"{k[0]}x{k[1]}/{k[2]}": round(v, 3) for k, v in times.items()}}}
    del singles
    torch.cuda.empty_cache()
    return res


def main():
    a = parse()
    if a.impl == "reference":
        run_reference(a)
    else:
        run_flod(a)


if __name__ == "__main__":
    main()
