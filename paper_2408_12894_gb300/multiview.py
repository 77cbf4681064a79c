"""Batched multi-view, multi-level rendering: one launch per stage for every view of a batch,
persistent render CTAs over a largest-first tile queue, the whole step captured in a CUDA
graph, and an autotuner for the tile shape and the shared-memory batch size.

A batch is a list of jobs. A job is one camera rendering either a whole Gaussian set (a FLoD
level) or a per-view selective mix of levels (Eq. 6 with the given distance thresholds,
selected from the camera's own position every step, Sec. 5.2 "per-view Gaussian set").
Everything below only orders calls into the C ABI; every stage runs in the CUDA library.
"""
from __future__ import annotations

import ctypes as C
import itertools

import torch

from . import flod

TILE_SHAPES = ((16, 16), (8, 8), (32, 8))
BATCH_SIZES = (256, 128, 64, 32)


class Job:
    """One camera and what it renders: ``set_index`` (a whole set) or, when ``levels`` is
    given, the selective mix of those set indices (coarse to fine) with ``thresholds``."""

    def __init__(self, cam: dict, set_index: int = 0, levels=None, thresholds=None,
                 capacity: int | None = None):
        self.cam = cam
        self.set_index = set_index
        self.levels = None if levels is None else list(levels)
        self.thresholds = None if thresholds is None else [float(t) for t in thresholds]
        # selection entries reserved (the view's units); None: every Gaussian of the levels
        self.capacity = capacity


class BatchedStep:
    """All jobs of a batch rendered (and optionally differentiated) as one step.

    ``run()`` enqueues the step on the current stream; ``capture()`` records it into a CUDA
    graph and ``replay()`` launches the graph. Selection lists live in buffers owned here and
    are refilled by flod_select_levels inside the step."""

    def __init__(self, sets, jobs, cfg=None, pair_capacity=None, backward=False, dL=None):
        self.sets = list(sets)
        self.jobs = list(jobs)
        self.backward = backward
        self.cfg = cfg if cfg is not None else flod.default_config(persistent=1)
        self._build(pair_capacity)
        self.out = self.rast.new_outputs()
        self.dL = dL
        self.graph = None
        if backward:
            # gradients of the sets the jobs render (directly or through a selection); the
            # others get none (NULL buffers: not written, not zero-filled)
            rendered = set()
            for j in self.jobs:
                rendered.update(j.levels if j.levels is not None else [j.set_index])
            self.grads = [[torch.empty_like(getattr(s, f)) for f in flod.GaussianSet.FIELDS]
                          if k in rendered else [None] * 5 for k, s in enumerate(self.sets)]
            # the library writes (mode 1) or zero-fills then accumulates (mode 2) every set's
            # gradients inside the step: no fill kernels of its own are needed here
            self.grads_c = flod.grads_struct(self.grads, self.rast.grad_modes())

    def _build(self, pair_capacity):
        """Selection buffers, views and the rasterizer (workspace) for the jobs."""
        dev = self.sets[0].means.device
        self.sel = []
        views = []
        for j in self.jobs:
            if j.levels is None:
                views.append(flod.view_struct(j.cam, j.set_index))
                self.sel.append(None)
            else:
                lv = [self.sets[i] for i in j.levels]
                cap = sum(s.n for s in lv)
                if j.capacity is not None:
                    cap = max(1, min(cap, int(j.capacity)))
                buf = torch.zeros(cap, dtype=torch.int32, device=dev)
                cnt = torch.zeros(1, dtype=torch.int32, device=dev)
                scr = torch.zeros(max(flod.flod_select_scratch_size(lv), 4), dtype=torch.uint8,
                                  device=dev)
                # selection entries are (level index << 28) | i and index the sets array
                # directly, so a selective job's levels must be sets 0 .. n-1
                if j.levels != list(range(len(j.levels))):
                    raise flod.FlodError("selective levels must be the first sets, in order")
                self.sel.append((lv, buf, cnt, scr))
                views.append(flod.view_struct(j.cam, 0, sel=buf, sel_count=cnt, sel_capacity=cap))
        self.rast = flod.Rasterizer(self.sets, views, self.cfg, pair_capacity)
        if getattr(self, "grads", None) is not None:
            self.grads_c = flod.grads_struct(self.grads, self.rast.grad_modes())

    def selection_capacity(self, i: int) -> int:
        """Entries reserved for job i's selection (its view's units)."""
        return int(self.sel[i][1].numel()) if self.sel[i] is not None else self.sets[self.jobs[i].set_index].n

    def fit_selection(self, cams=None, headroom: float = 1.1, grow_only: bool = False):
        """Size each selective job's selection buffer (its view's units) to the longest
        selection over ``cams[i]`` (a list of cameras for job i; by default its current
        camera) times ``headroom``, then rebuild the views and the workspace, keeping the
        pair capacity (synchronises; invalidates a captured graph). Fewer units make every
        stage that runs over a view's units cheaper; a later selection longer than the
        capacity sets DEV_SELECTION in the device status and renders only the first
        capacity entries."""
        cams = cams or {}
        changed = False
        for i, (j, s) in enumerate(zip(self.jobs, self.sel)):
            if s is None:
                continue
            lv, buf, cnt, scr = s
            need = 0
            for cam in cams.get(i, [j.cam]):
                flod.flod_select_levels(lv, cam["cam_pos"], buf, cnt, scr, d_thresh=j.thresholds)
                torch.cuda.synchronize()
                need = max(need, int(cnt.item()))
            cap = int(need * headroom) + 1024
            if grow_only:
                cap = max(cap, int(buf.numel()))
            if cap != buf.numel():
                j.capacity = cap
                changed = True
        if changed:
            self._build(self.rast.pair_capacity)
            self.graph = None

    def set_camera(self, i: int, cam: dict):
        """Move job i's camera (and, for a selective job, its selection origin). A captured
        graph keeps the cameras it was captured with."""
        self.jobs[i].cam = cam
        self.rast.views[i].cam = flod.camera_struct(cam)
        self.rast.refresh_structs()

    def selected_count(self, i: int) -> int:
        """Entries selected for job i by the last step (synchronises)."""
        return int(self.sel[i][2].item()) if self.sel[i] is not None else self.sets[self.jobs[i].set_index].n

    def _select(self, stream=None):
        for j, s in zip(self.jobs, self.sel):
            if s is None:
                continue
            lv, buf, cnt, scr = s
            flod.flod_select_levels(lv, j.cam["cam_pos"], buf, cnt, scr, d_thresh=j.thresholds,
                                    stream=stream)

    def run(self, stream=None):
        """Enqueue one step (no host synchronisation)."""
        self._select(stream)
        r = self.rast
        r.preprocess(stream)
        r.bin_sort(stream)
        r.render_fwd(*self.out, stream)
        if self.backward:
            r.blend_bwd(self.dL, self.out[1], self.out[2], stream)
            r.preprocess_bwd(self.grads_c, stream)

    def size_capacity(self, headroom: float = 1.15):
        """Run once eagerly and grow the pair capacity to fit, and any selection buffer
        that the current cameras' selections overflow (synchronises)."""
        for _ in range(4):
            self.run()
            torch.cuda.synchronize()
            if flod.flod_read_status(self.rast.ws) & flod.DEV_SELECTION:
                self.fit_selection(grow_only=True)
                continue
            need = int(self.rast.pair_count.item())
            if need <= self.rast.pair_capacity:
                return need
            self.rast.pair_capacity = min(flod.MAX_PAIRS, int(need * headroom) + 4096)
            self.rast._alloc()
        raise flod.FlodError("pair capacity did not converge")

    def capture(self):
        """Record one step into a CUDA graph (the pair capacity must already fit)."""
        s = torch.cuda.Stream()
        s.wait_stream(torch.cuda.current_stream())
        with torch.cuda.stream(s):
            self.run()                      # warm up on the side stream
        torch.cuda.current_stream().wait_stream(s)
        torch.cuda.synchronize()
        self.graph = torch.cuda.CUDAGraph()
        with torch.cuda.graph(self.graph):
            self.run()
        torch.cuda.synchronize()

    def replay(self):
        self.graph.replay()


def signature(sets, jobs, backward: bool):
    return (tuple(s.n for s in sets), backward,
            tuple((j.cam["width"], j.cam["height"], j.set_index,
                   None if j.levels is None else tuple(j.levels), j.capacity) for j in jobs))


_cache: dict = {}


def autotune(sets, jobs, backward=False, dL=None, steps=3, shapes=TILE_SHAPES,
             batches=BATCH_SIZES):
    """Time every (tile shape, batch size) candidate on the batch itself (persistent
    launch, eager) and return (best config, {candidate: ms}). Results are cached per
    workload signature for the life of the process."""
    key = signature(sets, jobs, backward)
    if key in _cache:
        return _cache[key]
    times = {}
    best = None
    for (tw, th), bs in itertools.product(shapes, batches):
        cfg = flod.default_config(tile_w=tw, tile_h=th, batch=bs, persistent=1)
        try:
            step = BatchedStep(sets, jobs, cfg, backward=backward, dL=dL)
            step.size_capacity()
        except (flod.FlodError, torch.cuda.OutOfMemoryError):
            times[(tw, th, bs)] = float("inf")      # does not fit: never chosen
            torch.cuda.empty_cache()
            continue
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record()
        for _ in range(steps):
            step.run()
        e1.record()
        torch.cuda.synchronize()
        ms = e0.elapsed_time(e1) / steps
        times[(tw, th, bs)] = ms
        if best is None or ms < times[best]:
            best = (tw, th, bs)
        del step
        torch.cuda.empty_cache()
    cfg = flod.default_config(tile_w=best[0], tile_h=best[1], batch=best[2], persistent=1)
    _cache[key] = (cfg, times)
    return cfg, times
