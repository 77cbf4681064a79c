"""Selective rendering with less resident memory (Sec. 5.2 and the Limitation section).

* ``predetermined_set``: the predetermined Gaussian set of Sec. 5.2. Eq. 6 selects, once,
  from the mean position of the training cameras; ``flod_gather`` copies the selected
  Gaussians of every level into one compact set with each level's s_min folded into s_opt
  (the set renders at s_min = 0 with each Gaussian's own Eq. 4 scale). Only that set needs
  to stay on the GPU: the levels can be released.
* ``StreamedLevels``: per-view selection with the levels kept in pinned host memory. The
  means of every level stay on the GPU (Eq. 6 needs only them); each frame selects from the
  camera position and gathers the selected Gaussians' other parameters across the CPU-GPU
  link into one device buffer sized for the largest selection, which the frame renders
  through an identity selection list bounded by the device count (no host round trip).

Both only order calls into the C ABI (flod_select_levels, flod_gather, the rasterizer).
"""
from __future__ import annotations

import ctypes as C

import numpy as np
import torch

from . import flod

FIELDS = flod.GaussianSet.FIELDS


def mean_camera_position(cams) -> np.ndarray:
    return np.mean([np.asarray(c["cam_pos"], dtype=np.float64) for c in cams], axis=0).astype(np.float32)


def predetermined_set(levels, origin, thresholds=None, gamma: float = 1.0, focal: float = 0.0):
    """(compact GaussianSet at s_min 0, number selected) of the levels (coarse to fine) for
    the reference position ``origin`` (Eq. 6; Eq. 7 thresholds when none are given)."""
    dev = levels[0].means.device
    cap = sum(s.n for s in levels)
    sel = torch.empty(cap, dtype=torch.int32, device=dev)
    cnt = torch.zeros(1, dtype=torch.int32, device=dev)
    scr = torch.empty(max(flod.flod_select_scratch_size(levels), 4), dtype=torch.uint8, device=dev)
    flod.flod_select_levels(levels, origin, sel, cnt, scr, d_thresh=thresholds, gamma=gamma,
                            focal=focal)
    n = int(cnt.item())   # once: the set is fixed from here on
    deg = max(s.sh_degree for s in levels)
    out = flod.gather_set(levels, sel, cnt, max(n, 1), deg, fold_s_min=True, device=dev)
    return out, n


def _host_struct(arrays, n, deg, s_min) -> flod.Gaussians:
    g = flod.Gaussians()
    g.means, g.quats, g.s_opt = (t.data_ptr() for t in arrays[:3])
    g.opacity_logit, g.sh = arrays[3].data_ptr(), arrays[4].data_ptr()
    g.n, g.sh_degree, g.s_min = n, deg, s_min
    return g


class StreamedLevels:
    """The levels' parameters in pinned host memory, their means also on the device; one
    frame = select on the device from the camera, gather the selection from host memory,
    render it."""

    def __init__(self, levels, thresholds, capacity: int, cfg=None, device="cuda"):
        self.thresholds = thresholds
        self.n_levels = len(levels)
        self.deg = max(s.sh_degree for s in levels)
        self.host = [[getattr(s, f).detach().cpu().pin_memory() for f in FIELDS] for s in levels]
        self.s_mins = [s.s_min for s in levels]
        self.ns = [s.n for s in levels]
        # selection reads only the means: device copies, the other pointers stay on the host
        self.dev_means = [s.means.detach().clone() for s in levels]
        self.sel_structs = []
        for k in range(self.n_levels):
            g = _host_struct(self.host[k], self.ns[k], levels[k].sh_degree, self.s_mins[k])
            g.means = self.dev_means[k].data_ptr()
            self.sel_structs.append(g)
        self.src_structs = [_host_struct(self.host[k], self.ns[k], levels[k].sh_degree,
                                         self.s_mins[k]) for k in range(self.n_levels)]
        self.capacity = int(capacity)
        total = sum(self.ns)
        self.sel = torch.empty(total, dtype=torch.int32, device=device)
        self.cnt = torch.zeros(1, dtype=torch.int32, device=device)
        self.scr = torch.empty(max(flod.flod_select_scratch_size(self.sel_structs), 4),
                               dtype=torch.uint8, device=device)
        K = (self.deg + 1) ** 2
        cap = self.capacity
        self.buf = flod.GaussianSet(torch.zeros(cap, 3, device=device), torch.zeros(cap, 4, device=device),
                                    torch.zeros(cap, 3, device=device), torch.zeros(cap, device=device),
                                    torch.zeros(cap, K, 3, device=device), self.deg, 0.0)
        self.ident = torch.arange(cap, dtype=torch.int32, device=device)
        self.cfg = cfg if cfg is not None else flod.default_config()
        self.rast = None
        self._cam = None

    def device_bytes(self) -> int:
        """Device bytes held for the parameters: every level's means + the frame buffer."""
        return 12 * sum(self.ns) + self.capacity * (12 + 16 + 12 + 4 + 12 * (self.deg + 1) ** 2)

    def host_bytes(self) -> int:
        return sum(t.numel() * 4 for per in self.host for t in per)

    def frame(self, cam: dict, stream=None):
        """Enqueue select -> gather -> render for one camera; returns (rgb, T, nc)."""
        flod.flod_select_levels(self.sel_structs, cam["cam_pos"], self.sel, self.cnt, self.scr,
                                d_thresh=self.thresholds, stream=stream)
        flod.flod_gather(self.src_structs, self.sel, self.cnt, self.capacity,
                         [getattr(self.buf, f) for f in FIELDS], self.deg, True, None, stream)
        view = flod.view_struct(cam, 0, sel=self.ident, sel_count=self.cnt,
                                sel_capacity=self.capacity)
        if self.rast is None:
            self.rast = flod.Rasterizer([self.buf], [view], self.cfg)
            self.out = self.rast.new_outputs()
        else:
            self.rast.views[0] = view
            self.rast.refresh_structs()
        self.rast.preprocess(stream)
        self.rast.bin_sort(stream)
        self.rast.render_fwd(*self.out, stream)
        return self.out

    def size_capacity(self, cams, headroom: float = 1.1):
        """Pair capacity for the given camera path (synchronises; run before timing)."""
        need = 0
        for cam in cams:
            self.frame(cam)
            torch.cuda.synchronize()
            n = int(self.cnt.item())
            if n > self.capacity:
                raise flod.FlodError(f"selection of {n} exceeds the buffer of {self.capacity}")
            need = max(need, int(self.rast.pair_count.item()))
            if not self.rast.ensure_capacity():
                self.frame(cam)
                torch.cuda.synchronize()
        self.rast.pair_capacity = int(need * headroom) + 4096
        self.rast._alloc()
        return need
