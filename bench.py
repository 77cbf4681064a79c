#!/usr/bin/env python3
"""Benchmark of the FLoD splatting path on GB300.

Workload (the headline configuration): the finest level of the 5-level scene -- 3,000,000
Gaussians (64 clusters, radius 20, SH degree 3, level-by-level initialised with Eq. 5 from
levels 1..4), one 1920x1080 pinhole camera at distance 40. A step is one training iteration
of that level (the loop body of Algorithm 1): preprocess (Eq. 4, Eq. 1, projection, SH),
binning + radix sort, forward blending, the L1 + D-SSIM loss against the target image and
its gradient, the blending backward, and the preprocess backward fused with the Adam step
of every parameter. The target is the level rendered with its DC colours perturbed
(seed 12). The forward-only frame rate and the rasterizer-only forward+backward rate (a
synthetic upstream gradient, no loss, no optimiser) are reported beside it.

``value`` = training iterations per second over all ranks (inputs resident in HBM; the
708 MB parameter set and the 1.4 GB of Adam moments exceed the 129 MB L2, so no flush is
needed). Each timed loop starts from the initial parameters and zero moments.
``e2e`` = the same iterations through the Python API with the step's input (the target
image) copied from pinned host memory and the step's result (the loss) read back, every
step; the copies run on a second stream, double-buffered.
``rooflines`` = every stage's achieved fraction of its bound, from CUDA-event times of a
pass with events at every stage boundary and the algorithmic work of each stage.
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
WORKLOAD = ("FLoD 5-level scene, level 5 (3M Gaussians, SH3), 1920x1080, one training iteration "
            "per step (render, L1 + D-SSIM loss, backward, Adam)")
# FP32 operations (an FFMA counts 2) of the blending kernels: per evaluated (pixel, Gaussian)
# pair -- the offset, q and its threshold test, with the per-column terms shared by the
# thread's pixels -- and on top for each pair the forward blended (alpha, transmittance,
# colour; backward: T recovery, colour, alpha and moment gradients). The nine-value warp
# reduction is overhead, not counted.
FLOP_FWD_EVAL, FLOP_FWD_BLEND = 8, 13
FLOP_BWD_EVAL, FLOP_BWD_BLEND = 7, 31
# FP32 operations of the loss per pixel and channel: the separable 11-tap window (22 FMA) on
# the five moment maps and on the three gradient maps, plus the SSIM value, its three
# derivatives, the L1 term and the combination (about 40)
FLOP_LOSS_PX = 2 * 22 * (5 + 3) + 40


def hbm_peak():
    """(GB/s, source): the driver's measured copy bandwidth, else the recipe's fallback."""
    try:
        d = json.load(open(os.path.join(ROOT, "MEASURED_PEAKS.json")))
        return float(d["hbm_gbs"]), "measured (MEASURED_PEAKS.json hbm_gbs, a copy kernel)"
    except (OSError, KeyError, ValueError):
        return 6800.0, "fallback 6.8 TB/s (an earlier GB300 copy measurement)"


def alu_peak_tflops(sms: int, mhz: float) -> float:
    """Plain float32 peak: SMs x 128 FP32 lanes x 2 (FMA) x SM clock."""
    return sms * 128 * 2 * mhz * 1e6 / 1e12


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
    ap.add_argument("--no-pruning", action="store_true", help="skip the overlap-pruning section")
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
    full step: preprocess forward+backward, binning and Adam on a slice of the Gaussians
    (scaled by N / slice), the loss and its gradient on a crop (scaled by the image area),
    plus blending forward+backward on a stratified sample of tiles. The tiles are
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
        # the loss on a 256 x 256 crop (scaled by the image area) and Adam on the slice
        self.crop = (rng.random((3, 256, 256)), rng.random((3, 256, 256)))
        self.adam_grads = {k: rng.normal(size=np.shape(g[k][:self.slice_n]))
                           for k in ("means", "quats", "s_opt", "opacity_logit", "sh")}

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
        from oracle import adam as AD
        from oracle import loss as LS
        t0 = time.perf_counter()
        LS.loss_and_grad(*self.crop)
        t_loss = (time.perf_counter() - t0) * self.cam["width"] * self.cam["height"] / (256 * 256)
        par = {k: np.asarray(sub[k], dtype=np.float64) for k in self.adam_grads}
        zero = {k: np.zeros_like(v) for k, v in par.items()}
        lrs = {"means": 3.2e-3, "quats": 1e-3, "s_opt": 5e-3, "opacity_logit": 5e-2,
               "sh_dc": 2.5e-3, "sh_rest": 1.25e-4}
        t0 = time.perf_counter()
        AD.adam_set(par, self.adam_grads, zero, zero, 1, lrs)
        t_adam = (time.perf_counter() - t0) * self.n / self.slice_n
        return t_slice * self.n / self.slice_n + t_tiles + t_loss + t_adam

    def describe(self) -> str:
        np = self.np
        return (f"preprocess fwd+bwd, binning and Adam of {self.slice_n} of {self.n} Gaussians "
                f"(x{self.n / self.slice_n:.0f}) + the loss and its gradient on a 256x256 crop "
                f"(x{self.cam['width'] * self.cam['height'] / 65536:.1f}) + blend fwd+bwd of "
                f"{len(self.sample)} of "
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

def stage_work(n, n_vis, pairs, tiles, depth_passes, tile_passes, deg, evals, pixels):
    """Algorithmic work of each stage of one training iteration: (bound, amount, unit).
    Bytes are the minimum DRAM traffic of the stage's definition, FLOPs its arithmetic
    (FLOP_* above); n Gaussians (one unit each), n_vis of them with tiles, `pairs` (unit,
    tile) pairs, `tiles` tiles, the sort passes that moved keys, SH degree deg."""
    par = 12 + 16 + 12 + 4 + 12 * (deg + 1) ** 2          # 236 B of parameters at SH3
    fwd_ev, bwd_ev, blended = evals
    return {
        # parameters in; xy, depth, conic, colour, radius, ellipse, tile record, count out
        "preprocess": ("hbm", n * (par + 84), "B"),
        # tile counts of all units; compaction (depth in, key + index out) and per pass
        # 4 B counted + 16 B scattered per visible unit
        "depth_sort": ("hbm", 4 * n + 12 * n_vis + 20 * n_vis * depth_passes, "B"),
        # per visible unit its count, slot count, unit id and tile record; 8 B per pair out
        "emission": ("hbm", 36 * n_vis + 8 * pairs, "B"),
        # per pass: 4 B counted + 16 B scattered per pair
        "tile_sort": ("hbm", 20 * pairs * tile_passes, "B"),
        # one tile id per pair in, one range per tile out
        "ranges": ("hbm", 4 * pairs + 8 * tiles, "B"),
        "render_fwd": ("alu", fwd_ev * FLOP_FWD_EVAL + blended * FLOP_FWD_BLEND, "FLOP"),
        "loss": ("alu", 3 * pixels * FLOP_LOSS_PX, "FLOP"),
        "blend_bwd": ("alu", bwd_ev * FLOP_BWD_EVAL + blended * FLOP_BWD_BLEND, "FLOP"),
        # parameters, both Adam moments in and out, and the tile count of every Gaussian;
        # the 2D gradient record and colour of the visible ones
        "bwd_adam": ("hbm", n * (6 * par + 4) + n_vis * (36 + 16), "B"),
    }


def rooflines(stage_ms, work, hbm_gbs, alu_tflops):
    out = {}
    for k, (bound, amount, unit) in work.items():
        ms = stage_ms.get(k)
        if not ms:
            continue
        if bound == "hbm":
            ach = amount / (ms * 1e-3) / 1e9
            out[k] = {"bound": "hbm", "ms": round(ms, 4), "work": int(amount), "achieved": ach,
                      "peak": hbm_gbs, "unit": "GB/s", "frac": ach / hbm_gbs}
        else:
            ach = amount / (ms * 1e-3) / 1e12
            out[k] = {"bound": "alu", "ms": round(ms, 4), "work": int(amount), "achieved": ach,
                      "peak": alu_tflops, "unit": "TFLOP/s", "frac": ach / alu_tflops}
    return out


def dc_perturbed_target(gs, view, seed=12, sigma=0.2):
    """The target image: the level rendered with its DC colours perturbed (untimed data)."""
    import numpy as np
    import torch
    from paper_2408_12894_gb300 import flod
    rng = np.random.default_rng(seed)
    sh = gs.sh.clone()
    noise = rng.normal(0.0, sigma, (gs.n, 3)).astype(np.float32)
    sh[:, 0, :] += torch.as_tensor(noise, device=sh.device)
    tg = flod.GaussianSet(gs.means, gs.quats, gs.s_opt, gs.opacity_logit, sh, gs.sh_degree, gs.s_min)
    r = flod.Rasterizer([tg], [view])
    rgb, _, _ = r.forward()
    torch.cuda.synchronize()
    out = rgb.clone()
    del r, sh, tg
    torch.cuda.empty_cache()
    return out


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
    from paper_2408_12894_gb300 import _build, flod, synth, train
    _build.build()
    counts = level_counts(a.small, a.scale)
    g = make_level(a.small, a.scale)
    gs = flod.GaussianSet.from_numpy(g, synth.LEVEL_SMIN[-1])
    for l in range(4):   # level-by-level initialisation (Eq. 5), on the device
        flod.flod_adjust_scale(gs.s_opt[:counts[l]], synth.LEVEL_SMIN[l], synth.LEVEL_SMIN[l + 1])
    cam = synth.level_camera()
    view = flod.view_struct(cam)
    H, W = cam["height"], cam["width"]
    st = torch.cuda.current_stream()
    props = torch.cuda.get_device_properties(local)

    def barrier():
        replicas.barrier()

    # ---------------- rasterizer alone: forward frames, and forward + backward with a
    # synthetic upstream gradient (no loss, no optimiser)
    rast = flod.Rasterizer([gs], [view])
    rgb, T, nc = rast.forward()                    # sizes the pair capacity once
    torch.cuda.synchronize()
    pairs = int(rast.pair_count.item())
    rast.pair_capacity = int(pairs * 1.2) + 4096
    rast._alloc()
    dL = torch.as_tensor(synth.upstream_gradient(11, [cam]), device="cuda")
    grads = [[torch.empty_like(getattr(gs, f)) for f in flod.GaussianSet.FIELDS]]
    grads_c = flod.grads_struct(grads, overwrite=True)   # one view: every gradient written

    def fwd():
        rast.preprocess()
        rast.bin_sort()
        rast.render_fwd(rgb, T, nc)

    def raster_step():
        fwd()
        rast.blend_bwd(dL, T, nc)
        rast.preprocess_bwd(grads_c)

    for _ in range(max(a.warmup, 3)):
        raster_step()
    torch.cuda.synchronize()
    assert flod.flod_read_status(rast.ws) == 0, "device status error"
    barrier()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record(st)
    for _ in range(a.steps):
        fwd()
    e1.record(st)
    barrier()
    fwd_ms = e0.elapsed_time(e1) / a.steps
    e0.record(st)
    for _ in range(a.steps):
        raster_step()
    e1.record(st)
    barrier()
    raster_ms = e0.elapsed_time(e1) / a.steps
    del rast, grads, grads_c, rgb, T, nc, dL
    torch.cuda.empty_cache()

    # ---------------- the training iteration
    target = dc_perturbed_target(gs, view)
    init = {f: getattr(gs, f).clone() for f in flod.GaussianSet.FIELDS}
    ts = train.TrainStep([gs], [view], target, lrs=train.default_lrs(extent=20.0))
    assert ts.fused, "one view renders the level: the fused backward + Adam applies"
    pairs = ts.size_capacity(headroom=1.5)
    r = ts.rast
    rgb, T, nc = ts.out

    def reset():
        """Initial parameters, zero moments, step counter 0 (untimed, between loops)."""
        for f in flod.GaussianSet.FIELDS:
            getattr(gs, f).copy_(init[f])
        for t in ts.m[0] + ts.v[0]:
            t.zero_()
        ts.d_step.zero_()

    def iteration(ev=None, ev_k=None):
        # ev: events at every stage boundary; ev_k: (stage, [before, after]) around the
        # dominant kernel only
        def rec(i):
            if ev:
                ev[i].record(st)
        rec(0)
        r.preprocess()
        rec(1)
        for ph in (flod.BIN_PHASE_DEPTH, flod.BIN_PHASE_EMIT, flod.BIN_PHASE_TILES,
                   flod.BIN_PHASE_RANGES):
            r.bin_sort_phase(ph)
            rec(1 + ph)
        r.render_fwd(rgb, T, nc)
        rec(6)
        flod.flod_loss(rgb, ts.target, ts.sizes, ts.dL, ts.scratch, ts.loss, ts.lam)
        rec(7)
        if ev_k and ev_k[0] == "blend_bwd":
            ev_k[1][0].record(st)
        r.blend_bwd(ts.dL, T, nc)
        rec(8)
        if ev_k and ev_k[0] == "blend_bwd":
            ev_k[1][1].record(st)
        if ev_k and ev_k[0] == "bwd_adam":
            ev_k[1][0].record(st)
        r.preprocess_bwd_adam(ts.states_c, ts.acfg)
        rec(9)
        if ev_k and ev_k[0] == "bwd_adam":
            ev_k[1][1].record(st)

    for _ in range(max(a.warmup, 3)):
        iteration()
    torch.cuda.synchronize()
    assert flod.flod_read_status(r.ws) == 0, "device status error"

    # ---- stage times (events at every boundary) and the blending evaluation counts
    reset()
    ev_before = r.eval_counts()
    evs = [[torch.cuda.Event(enable_timing=True) for _ in range(10)] for _ in range(a.steps)]
    for i in range(a.steps):
        iteration(evs[i])
    torch.cuda.synchronize()
    ev_after = r.eval_counts()
    names = ["preprocess", "depth_sort", "emission", "tile_sort", "ranges", "render_fwd",
             "loss", "blend_bwd", "bwd_adam"]
    stage_ms = {n: sum(evs[i][j].elapsed_time(evs[i][j + 1]) for i in range(a.steps)) / a.steps
                for j, n in enumerate(names)}
    step_ms = [evs[i][0].elapsed_time(evs[i][9]) for i in range(a.steps)]
    plan = r.region("plan", torch.int32, 64).cpu().numpy()
    n_vis = int(r.region("plan", torch.int64, 32)[8].item())
    pairs_now = int(r.pair_count.item())
    evals = tuple((ev_after[k] - ev_before[k]) / a.steps for k in range(3))

    # ---- the headline: K iterations between two events; inside, events only around the
    # dominant kernel (the longer of the blending backward and the fused backward + Adam in
    # the stage pass), timed live
    reset()
    clk = clock_sampler(local)
    dom_stage = max(("blend_bwd", "bwd_adam"), key=lambda k: stage_ms[k])
    evk = [[torch.cuda.Event(enable_timing=True) for _ in range(2)] for _ in range(a.steps)]
    h0, h1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    barrier()
    t_wall = time.perf_counter()
    h0.record(st)
    for i in range(a.steps):
        iteration(ev_k=(dom_stage, evk[i]))
    h1.record(st)
    barrier()
    t_wall = time.perf_counter() - t_wall
    clocks = clock_summary(clk)
    ms = h0.elapsed_time(h1) / a.steps
    live_ms = {dom_stage: sum(e[0].elapsed_time(e[1]) for e in evk) / a.steps}
    loss_end = float(ts.loss[0].item())
    status = flod.flod_read_status(r.ws)
    assert status == 0, f"device status {status} during the timed iterations"
    ms, fwd_ms, raster_ms = replicas.max_over_ranks([ms, fwd_ms, raster_ms], device="cuda")

    # ---- end to end through TrainStep: the target image in from pinned host memory and
    # the loss back, every step, on a second stream, double-buffered
    reset()
    cs = torch.cuda.Stream()
    tgt_host = target.cpu().pin_memory()
    tgts = [target, torch.empty_like(target)]
    losses = [ts.loss, torch.zeros_like(ts.loss)]
    loss_hosts = [torch.zeros(1, dtype=torch.float32).pin_memory() for _ in range(2)]
    ev_in = [torch.cuda.Event() for _ in range(2)]     # target j is on the device
    ev_used = [torch.cuda.Event() for _ in range(2)]   # the loss that read target j ended
    ev_out = [torch.cuda.Event() for _ in range(2)]    # loss j is on the host

    def e2e_step(i):
        j = i % 2
        st.wait_event(ev_in[j])
        if i + 1 < a.steps:
            if i >= 1:
                cs.wait_event(ev_used[1 - j])
            with torch.cuda.stream(cs):
                tgts[1 - j].copy_(tgt_host, non_blocking=True)
                ev_in[1 - j].record(cs)
        if i >= 2:
            st.wait_event(ev_out[j])
        ts.target, ts.loss = tgts[j], losses[j]
        ts.run()
        ev_used[j].record(st)
        cs.wait_event(ev_used[j])
        with torch.cuda.stream(cs):
            loss_hosts[j].copy_(losses[j], non_blocking=True)
            ev_out[j].record(cs)

    barrier()
    e2e0, e2e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e2e0.record(st)
    cs.wait_event(e2e0)
    with torch.cuda.stream(cs):
        tgts[0].copy_(tgt_host, non_blocking=True)
        ev_in[0].record(cs)
    for i in range(a.steps):
        e2e_step(i)
    st.wait_stream(cs)
    e2e1.record(st)
    barrier()
    e2e_ms = e2e0.elapsed_time(e2e1) / a.steps
    e2e_ms, = replicas.max_over_ranks([e2e_ms], device="cuda")
    ts.target, ts.loss = target, losses[0]

    # ---- the same iteration written as a framework training loop: flod.rasterize under
    # torch autograd (its backward writes the gradients itself), the library's loss, the
    # gradients handed to flod_adam_step, .grad released (no torch fill or add kernels)
    reset()
    ag = flod.Rasterizer([gs], [view], pair_capacity=r.pair_capacity)
    params = [getattr(gs, f) for f in flod.GaussianSet.FIELDS]
    for t in params:
        t.requires_grad_(True)
    ag_dL = torch.empty_like(rgb)

    def ag_step():
        rgb_a, _, _ = flod.rasterize(ag, check_capacity=False)
        flod.flod_loss(rgb_a.detach(), target, ts.sizes, ag_dL, ts.scratch, ts.loss, ts.lam)
        rgb_a.backward(ag_dL)
        flod.flod_adam_step([params], [[t.grad for t in params]], ts.m, ts.v, [gs.n],
                            [gs.sh_degree], ts.acfg)
        for t in params:
            t.grad = None
    for _ in range(max(a.warmup, 3)):
        ag_step()
    barrier()
    a0, a1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    a0.record(st)
    for _ in range(a.steps):
        ag_step()
    a1.record(st)
    barrier()
    autograd_ms = a0.elapsed_time(a1) / a.steps
    assert flod.flod_read_status(ag.ws) == 0, "device status error (autograd path)"
    for t in params:
        t.requires_grad_(False)
    del ag, ag_dL

    # ---- the same iteration captured once in a CUDA graph and replayed (no host launches)
    reset()
    ts.capture()
    for _ in range(max(a.warmup, 3)):
        ts.replay()
    barrier()
    g0, g1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    g0.record(st)
    for _ in range(a.steps):
        ts.replay()
    g1.record(st)
    barrier()
    graph_ms = g0.elapsed_time(g1) / a.steps
    assert flod.flod_read_status(r.ws) == 0, "device status error (graph replay)"
    ts.graph = None
    graph_ms, = replicas.max_over_ranks([graph_ms], device="cuda")

    # ---- rooflines
    hbm, hbm_src = hbm_peak()
    mhz = clocks.get("sm_max_mhz") or 2070.0
    alu = alu_peak_tflops(props.multi_processor_count, mhz)
    depth_passes = int(sum(plan[0:4]))
    tile_passes = int(sum(plan[4:8]))
    work = stage_work(gs.n, n_vis, pairs_now, int(r.layout.tiles), depth_passes, tile_passes,
                      gs.sh_degree, evals, W * H)
    roof = rooflines(stage_ms, work, hbm, alu)
    live = rooflines(live_ms, {k: work[k] for k in live_ms}, hbm, alu)
    dom = max(live, key=lambda k: live[k]["ms"])
    d = live[dom]
    traffic = measured_traffic({"blend_bwd": "k_render_bwd", "bwd_adam": "k_preprocess_bwd_adam"}[dom])
    roofline = {"kernel": dom, "bound": d["bound"], "achieved": d["achieved"], "peak": d["peak"],
                "unit": d["unit"], "frac": d["frac"], "traffic": traffic,
                "peak_source": hbm_src if d["bound"] == "hbm" else
                f"{props.multi_processor_count} SMs x 128 FP32 lanes x 2 x {mhz:.0f} MHz (derived)"}
    # launches per iteration: status clear + preprocess; depth sort (visible counts, scan,
    # unit keys, 4 x (count, scan, scatter)); block sums, scan, light, big-unit and sliced
    # emission; tile passes x (count, scan, scatter); ranges; render; 2 loss kernels;
    # 2D-gradient zero-fill + blend backward; fused backward + Adam and the step tick
    launches_per_step = 2 + (3 + 12) + 5 + 3 * max(1, (int(math.ceil(math.log2(max(int(r.layout.tiles), 2)))) + 8) // 9) + 1 + 1 + 2 + 2 + 2

    if rank == 0:
        line = {
            "metric": METRIC, "value": world * 1e3 / ms, "unit": "it/s", "n_gpus": world,
            "steps": a.steps, "warmup": a.warmup, "ms_per_step": ms,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f32",
            "data": "synthetic (seeded cluster scene; target = the level rendered with perturbed "
                    "DC colours)",
            "config": {"workload": WORKLOAD, "gaussians": int(gs.n), "resolution": f"{W}x{H}",
                       "sh_degree": 3, "tile": "16x16", "pairs_per_step": pairs,
                       "pairs_after_training_steps": pairs_now, "loss": "L1 + 0.2 D-SSIM",
                       "optimizer": "Adam (3DGS learning rates, scene extent 20)",
                       "l2": "inputs larger than L2 (708 MB parameters + 1.4 GB Adam moments, no flush)",
                       "parallelism": f"replicas x{world}"},
            "fwd_fps": world * 1e3 / fwd_ms, "fwd_ms": fwd_ms,
            "raster_fwd_bwd_it_s": world * 1e3 / raster_ms, "raster_fwd_bwd_ms": raster_ms,
            "graph_replay": {"it_s": world * 1e3 / graph_ms, "ms": graph_ms,
                             "what": "the same iteration captured once in a CUDA graph"},
            "autograd_path": {"it_s": 1e3 / autograd_ms, "ms": autograd_ms,
                              "what": "flod.rasterize under torch autograd + flod_loss + "
                                      "flod_adam_step on the .grad tensors (gradient then "
                                      "Adam, unfused)"},
            "stage_ms": {k: round(v, 4) for k, v in stage_ms.items()},
            "step_ms_median": statistics.median(step_ms),
            "wall_ms_per_step": 1e3 * t_wall / a.steps,
            "loss_after_steps": loss_end,
            "evals_per_step": {"fwd": evals[0], "bwd": evals[1], "blended": evals[2]},
            "sort_passes": {"depth": depth_passes, "tile": tile_passes},
            "visible_units": n_vis,
            "roofline": roofline,
            "rooflines": roof,
            "device": {"name": props.name, "sms": props.multi_processor_count,
                       "alu_peak_tflops": alu, "alu_peak_clock_mhz": mhz, "hbm_peak_gbs": hbm},
            "e2e": {"value": world * 1e3 / e2e_ms, "unit": "it/s",
                    "h2d_bytes_per_step": int(target.numel() * 4),
                    "d2h_bytes_per_step": 4},
            "gpu_launches": launches_per_step * a.steps,
            "clocks": clocks,
        }
        if not a.no_selective:
            line["selective"] = selective_section(a)
        if not a.no_batched:
            line["batched"] = batched_section(a)
        if not a.no_pruning:
            line["overlap_pruning"] = pruning_section(a)
        if not a.no_cpu_baseline and world == 1:
            try:
                g_np = dict(g)
                g_np["s_opt"] = init["s_opt"].cpu().numpy()
                ost = OracleStep(g_np, cam, synth.LEVEL_SMIN[-1])
                line["cpu_baseline"] = cpu_baseline_line(ost)
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
    """Selective rendering along the 32-frame path, forward only, at 1920x1080 and 3840x2160:
    per-view selection (Eq. 6 every frame from the camera position) over resident levels; the
    predetermined set (Sec. 5.2) gathered once into one compact resident set; and per-view
    selection with the levels streamed from pinned host memory."""
    import torch
    from paper_2408_12894_gb300 import flod, multiview, selective, synth
    sets = selective_sets(a.scale)
    th = list(synth.SELECTIVE_THRESHOLDS[::-1])
    out = {"workload": "5-level scene x5 (radius 100), thresholds {10,25,50,100}, 32-frame path, "
                       "per-view selection every frame, forward", "resolutions": {}}
    for (w, h) in ((1920, 1080), (3840, 2160)):
        path = synth.camera_path(width=w, height=h)
        st = multiview.BatchedStep(sets, [multiview.Job(path[0], levels=[0, 1, 2, 3, 4], thresholds=th)],
                                   flod.default_config())
        # the selection buffer (the view's units) sized to the path's longest selection + 10%
        # instead of every Gaussian of the five levels
        st.fit_selection({0: path}, headroom=1.1)
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
        res = {
            "fps": 1e3 / ms, "ms_per_frame": ms,
            "selected_per_frame": {"min": min(sel), "max": max(sel), "mean": sum(sel) / len(sel)},
            "selected_param_bytes_per_frame_mean": 236 * sum(sel) / len(sel),
            "selection_capacity": st.selection_capacity(0),
            "working_set_bytes_per_frame_max": max(per_frame_bytes),
            "all_levels_param_bytes": 236 * sum(s.n for s in sets)}
        del st
        torch.cuda.empty_cache()
        # predetermined set (Sec. 5.2): selected once from the mean camera position of the
        # path, gathered into one compact resident set; frames render only that set
        origin = selective.mean_camera_position(path)
        compact, n_pre = selective.predetermined_set(sets, origin, th)
        r = flod.Rasterizer([compact], [flod.view_struct(path[0])])
        need = 0
        for cam in path:
            r.views[0] = flod.view_struct(cam)
            r.refresh_structs()
            r.forward()
            torch.cuda.synchronize()
            need = max(need, int(r.pair_count.item()))
        r.pair_capacity = int(need * 1.1) + 4096
        r._alloc()
        outs = r.new_outputs()
        fr = [0]

        def pre_frame():
            r.views[0] = flod.view_struct(path[fr[0] % len(path)])
            r.refresh_structs()
            fr[0] += 1
            r.preprocess()
            r.bin_sort()
            r.render_fwd(*outs)
        ms_pre = timed(pre_frame, max(a.steps, len(path)), 3)
        res["predetermined"] = {"fps": 1e3 / ms_pre, "ms_per_frame": ms_pre, "selected": n_pre,
                                "resident_param_bytes": 236 * n_pre,
                                "resident_vs_all_levels": n_pre / sum(s.n for s in sets)}
        del r, outs, compact
        torch.cuda.empty_cache()
        # per-view selection streamed from pinned host memory: only the means of every
        # level and a buffer for the largest selection stay on the device
        sl = selective.StreamedLevels(sets, th, capacity=int(max(sel) * 1.05) + 1024)
        sl.size_capacity(path)
        fr = [0]

        def stream_frame():
            sl.frame(path[fr[0] % len(path)])
            fr[0] += 1
        ms_st = timed(stream_frame, max(a.steps, len(path)), 3)
        res["streamed_per_view"] = {"fps": 1e3 / ms_st, "ms_per_frame": ms_st,
                                    "device_param_bytes": sl.device_bytes(),
                                    "host_param_bytes": sl.host_bytes(),
                                    "gathered_bytes_per_frame_mean": 224 * sum(sel) / len(sel)}
        del sl
        torch.cuda.empty_cache()
        out["resolutions"][f"{w}x{h}"] = res
    del sets
    torch.cuda.empty_cache()
    return out


def pruning_section(a):
    """Overlap pruning (Sec. 4.3) of level 4 of the 5-level scene (1M Gaussians, s_min 0.0625,
    d_OP = 0.03125; it runs at every level but the last) right after a densification step
    (10% of the Gaussians cloned and moved by N(0, d_OP^2)): the 3-nearest search and mask,
    and the compaction of the kept Gaussians into a new set."""
    import torch
    from paper_2408_12894_gb300 import flod, synth
    counts = tuple(int(round(c * a.scale)) for c in synth.LEVEL_COUNTS)
    levels = synth.level_scene(counts=counts[:4])
    d_op = 0.5 * synth.LEVEL_SMIN[3]
    g = synth.with_jittered_clones(levels[3][0], 0.1, d_op)
    gs = flod.GaussianSet.from_numpy(g, synth.LEVEL_SMIN[3])
    n = gs.n
    keep = torch.empty(n, dtype=torch.uint8, device="cuda")
    kept = torch.empty(n, dtype=torch.int32, device="cuda")
    cnt = torch.zeros(1, dtype=torch.int32, device="cuda")
    nb = flod.flod_prune_scratch_size(n)
    scr = torch.empty(nb + 256, dtype=torch.uint8, device="cuda")
    scr = scr[(-scr.data_ptr()) % 256:][:nb]
    out = [torch.empty(n, 3, device="cuda"), torch.empty(n, 4, device="cuda"),
           torch.empty(n, 3, device="cuda"), torch.empty(n, device="cuda"),
           torch.empty(n, 16, 3, device="cuda")]

    def mask():
        flod.flod_overlap_prune(gs, d_op, keep, cnt, scr, out_kept=kept)

    def prune_and_compact():
        mask()
        flod.flod_gather([gs], kept, cnt, n, out, 3, False)
    ms_mask = timed(mask, max(10, a.steps // 4), 3)
    ms_all = timed(prune_and_compact, max(10, a.steps // 4), 3)
    m = int(cnt.item())
    res = {"workload": f"level 4 of the 5-level scene with 10% jittered clones: {n} Gaussians, "
                       f"d_OP = {d_op}",
           "mask_ms": ms_mask, "prune_and_compact_ms": ms_all, "kept": m, "pruned": n - m,
           "gaussians_per_s": n * 1e3 / ms_mask}
    del gs, keep, kept, scr, out
    torch.cuda.empty_cache()
    return res


def batched_section(a):
    """64 cameras of mixed resolution, each rendering one level of the 5-level scene or the
    per-view selective mix of the stretched scene, forward+backward: one autotuned,
    persistent, graph-captured batch vs the same jobs as 64 per-view calls (16x16 tiles,
    one CTA per tile), issued eagerly and also captured in one CUDA graph (so the second
    ratio holds no host launch cost)."""
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
    # each selective job's selection buffer sized to its selection + 10% (kept on the jobs,
    # so the batch, the autotuner and the per-view arm all use the same units)
    fit = multiview.BatchedStep(sets, jobs, flod.default_config(), backward=True, dL=dL)
    fit.fit_selection(headroom=1.1)
    del fit
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
    # the same per-view calls captured in one CUDA graph: no host launch cost in either arm
    g_pv = torch.cuda.CUDAGraph()
    side = torch.cuda.Stream()
    side.wait_stream(torch.cuda.current_stream())
    with torch.cuda.stream(side):
        per_view()
    torch.cuda.current_stream().wait_stream(side)
    torch.cuda.synchronize()
    with torch.cuda.graph(g_pv):
        per_view()
    ms_single_graph = timed(g_pv.replay, max(3, a.steps // 4), 1)
    del g_pv
    res = {"workload": f"{len(jobs)} views, resolutions {{640x480,1280x720,1920x1080,3840x2160}}, "
                       "jobs {levels 1..5, per-view selective}, fwd+bwd",
           "views": len(jobs), "pixels": int(sum(c["width"] * c["height"] for c in cams)),
           "pairs": pairs, "batched_ms": ms_batched, "per_view_ms": ms_single,
           "batched_views_per_s": len(jobs) * 1e3 / ms_batched,
           "per_view_views_per_s": len(jobs) * 1e3 / ms_single,
           "speedup": ms_single / ms_batched,
           "per_view_graph_ms": ms_single_graph,
           "speedup_vs_graph_per_view": ms_single_graph / ms_batched,
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
