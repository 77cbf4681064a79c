"""One training iteration of a FLoD level (the loop body of Algorithm 1): Eq. 4 inside
Rasterize, then Loss, then Adam on the gradient, all through the C ABI.

``TrainStep`` owns what the iteration needs besides the parameters: the rasterizer
workspace, the rendered image, the loss gradient and its scratch, the Adam moments and the
device step counter. ``run()`` enqueues one iteration on the current stream without any
host synchronisation, so it can be captured in a CUDA graph:

    preprocess -> bin_sort -> render_fwd -> loss (L1 + D-SSIM) -> blend_bwd ->
        preprocess_bwd fused with Adam          (each set rendered by one view, whole)
        preprocess_bwd (zero-first) + Adam step (any other batch of views)

The learning rates default to the 3DGS backbone's (which the paper keeps, Sec. 5.1.4):
means 1.6e-4 x the scene extent, rotations 1e-3, s_opt 5e-3, opacity logits 5e-2, SH DC
2.5e-3 and the higher SH coefficients 2.5e-3 / 20.
"""
from __future__ import annotations

import torch

from . import flod


def default_lrs(extent: float = 1.0) -> dict:
    return {"means": 1.6e-4 * extent, "quats": 1e-3, "s_opt": 5e-3, "opacity_logit": 5e-2,
            "sh_dc": 2.5e-3, "sh_rest": 2.5e-3 / 20.0}


class TrainStep:
    """One training iteration of every view of a batch against its target image.

    ``targets``: device float32, the planar layout of the render ([3][H][W] per view,
    views concatenated). The parameters of ``sets`` are updated in place."""

    def __init__(self, sets, views, targets: torch.Tensor, cfg=None, lrs=None, extent: float = 1.0,
                 pair_capacity=None, lam: float = flod.LOSS_LAMBDA):
        self.sets = list(sets)
        self.rast = flod.Rasterizer(self.sets, views, cfg, pair_capacity)
        self.views = self.rast.views
        dev = self.sets[0].means.device
        self.out = self.rast.new_outputs()
        self.target = targets
        if targets.numel() != self.out[0].numel():
            raise flod.FlodError("targets must hold 3 H W floats per view")
        self.sizes = [(v.cam.width, v.cam.height) for v in self.views]
        self.dL = torch.empty_like(self.out[0])
        self.loss = torch.zeros(len(self.views), dtype=torch.float32, device=dev)
        self.scratch = _aligned_bytes(flod.flod_loss_scratch_size(self.sizes), dev)
        self.lam = lam
        self.lrs = lrs if lrs is not None else default_lrs(extent)
        self.d_step = torch.zeros(1, dtype=torch.int32, device=dev)
        self.acfg = flod.adam_config(self.lrs, self.d_step)
        self.m = [[torch.zeros_like(getattr(s, f)) for f in flod.GaussianSet.FIELDS] for s in self.sets]
        self.v = [[torch.zeros_like(getattr(s, f)) for f in flod.GaussianSet.FIELDS] for s in self.sets]
        modes = self.rast.grad_modes()
        self.fused = all(m == flod.GRAD_OVERWRITE for m in modes)
        params = [[getattr(s, f) for f in flod.GaussianSet.FIELDS] for s in self.sets]
        if self.fused:
            self.states_c = flod.adam_states(list(zip(params, self.m, self.v)))
        else:
            self.grads = [[torch.empty_like(getattr(s, f)) for f in flod.GaussianSet.FIELDS]
                          for s in self.sets]
            self.grads_c = flod.grads_struct(self.grads, flod.GRAD_ZERO_FIRST)
            self.params = params
        self.graph = None

    def run(self, stream=None):
        """Enqueue one iteration (no host synchronisation)."""
        r = self.rast
        r.preprocess(stream)
        r.bin_sort(stream)
        rgb, T, nc = self.out
        r.render_fwd(rgb, T, nc, stream)
        flod.flod_loss(rgb, self.target, self.sizes, self.dL, self.scratch, self.loss, self.lam,
                       stream)
        r.blend_bwd(self.dL, T, nc, stream)
        if self.fused:
            r.preprocess_bwd_adam(self.states_c, self.acfg, stream)
        else:
            r.preprocess_bwd(self.grads_c, stream)
            flod.flod_adam_step(self.params, self.grads, self.m, self.v,
                                [s.n for s in self.sets], [s.sh_degree for s in self.sets],
                                self.acfg, stream)

    def size_capacity(self, headroom: float = 1.5):
        """Render once (without a training update) and size the pair capacity with headroom
        for the scene to change as it trains (synchronises)."""
        r = self.rast
        for _ in range(4):
            r.preprocess()
            r.bin_sort()
            torch.cuda.synchronize()
            need = int(r.pair_count.item())
            if need * headroom <= r.pair_capacity:
                return need
            r.pair_capacity = min(flod.MAX_PAIRS, int(need * headroom) + 4096)
            r._alloc()
        raise flod.FlodError("pair capacity did not converge")

    def capture(self):
        """Record one iteration into a CUDA graph (replays advance the Adam step counter)."""
        self.graph = torch.cuda.CUDAGraph()
        s = torch.cuda.Stream()
        s.wait_stream(torch.cuda.current_stream())
        torch.cuda.current_stream().wait_stream(s)
        with torch.cuda.graph(self.graph):
            self.run()
        torch.cuda.synchronize()

    def replay(self):
        self.graph.replay()


def _aligned_bytes(n: int, dev) -> torch.Tensor:
    buf = torch.empty(n + 256, dtype=torch.uint8, device=dev)
    off = (-buf.data_ptr()) % 256
    return buf[off:off + n]
