"""Python binding of the C ABI in include/flod.h (ctypes; argument marshalling only).

Every stage of the path runs in the CUDA library ``_lib/libflod.so``; this module only turns
torch tensors and camera dicts into the C structs, passes ``data_ptr()`` values and the
current torch stream, and checks the returned status. There is no CPU fallback: loading
raises if the library is missing or the device is not sm_103.

The functions named like the C entry points (``flod_preprocess`` ...) are one-to-one
wrappers. ``Rasterizer`` keeps a workspace and chains them for one batch of views;
``rasterize`` is a torch.autograd.Function over the whole path.
"""
from __future__ import annotations

import ctypes as C
import math
import os

import numpy as np
import torch

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "_lib", "libflod.so")

MAX_VIEWS = 128
MAX_SETS = 16
SEL_SHIFT = 28
MAX_PAIRS = (1 << 32) - 8192
DEV_CAPACITY = 0x1
DEV_TIMEOUT = 0x2
DEV_TILESET = 0x4
DEV_GRID = 0x8
DEV_SELECTION = 0x10

STATUS = {0: "ok", 1: "invalid argument", 2: "pair capacity exceeded", 3: "device wait timed out",
          4: "CUDA error", 5: "unsupported device (needs sm_103)", 6: "workspace too small"}


class FlodError(RuntimeError):
    pass


class Camera(C.Structure):
    _fields_ = [("viewmat", C.c_float * 12), ("fx", C.c_float), ("fy", C.c_float),
                ("cx", C.c_float), ("cy", C.c_float), ("width", C.c_int), ("height", C.c_int),
                ("cam_pos", C.c_float * 3)]


class Gaussians(C.Structure):
    _fields_ = [("means", C.c_void_p), ("quats", C.c_void_p), ("s_opt", C.c_void_p),
                ("opacity_logit", C.c_void_p), ("sh", C.c_void_p), ("n", C.c_int),
                ("sh_degree", C.c_int), ("s_min", C.c_float)]


class View(C.Structure):
    _fields_ = [("cam", Camera), ("set", C.c_int), ("sel", C.c_void_p), ("sel_count", C.c_void_p),
                ("sel_capacity", C.c_uint32)]


class RasterConfig(C.Structure):
    _fields_ = [("tile_w", C.c_int), ("tile_h", C.c_int), ("batch", C.c_int),
                ("dilation", C.c_float), ("z_near", C.c_float), ("bg", C.c_float * 3),
                ("extent_rule", C.c_int), ("persistent", C.c_int)]


class Grads(C.Structure):
    _fields_ = [("means", C.c_void_p), ("quats", C.c_void_p), ("s_opt", C.c_void_p),
                ("opacity_logit", C.c_void_p), ("sh", C.c_void_p), ("overwrite", C.c_int)]


class ParamArrays(C.Structure):
    _fields_ = [("means", C.c_void_p), ("quats", C.c_void_p), ("s_opt", C.c_void_p),
                ("opacity_logit", C.c_void_p), ("sh", C.c_void_p)]


class AdamConfig(C.Structure):
    _fields_ = [("lr_means", C.c_float), ("lr_quats", C.c_float), ("lr_s_opt", C.c_float),
                ("lr_opacity", C.c_float), ("lr_sh_dc", C.c_float), ("lr_sh_rest", C.c_float),
                ("beta1", C.c_double), ("beta2", C.c_double), ("eps", C.c_double),
                ("d_step", C.c_void_p)]


class AdamState(C.Structure):
    _fields_ = [("params", ParamArrays), ("m", ParamArrays), ("v", ParamArrays)]


class WsLayout(C.Structure):
    _fields_ = [(n, C.c_size_t) for n in ("total", "status", "pair_count", "plan", "xy", "depth",
                                          "conic_o", "rgb", "radius", "ext", "trec", "tiles_touched",
                                          "block_sums", "slices")] + \
               [("ukeys", C.c_size_t * 2), ("uvals", C.c_size_t * 2),
                ("keys", C.c_size_t * 2), ("vals", C.c_size_t * 2)] + \
               [(n, C.c_size_t) for n in ("hist", "counts", "ranges", "grad2d", "queue")] + \
               [(n, C.c_uint64) for n in ("units", "tiles", "pixels", "pair_capacity")]


_lib = None


def lib() -> C.CDLL:
    """The loaded CUDA library; raises if it was not built (no fallback)."""
    global _lib
    if _lib is None:
        if not os.path.exists(LIB_PATH):
            raise FlodError(f"CUDA library not built: {LIB_PATH} is missing "
                            "(run paper_2408_12894_gb300._build.build())")
        L = C.CDLL(LIB_PATH)
        P, I, U64, SZ = C.c_void_p, C.c_int, C.c_uint64, C.c_size_t
        L.flod_default_config.argtypes = [P]
        L.flod_default_config.restype = None
        L.flod_workspace_size.argtypes = [P, I, P, I, U64, P]
        L.flod_workspace_size.restype = SZ
        L.flod_workspace_layout.argtypes = [P, I, P, I, U64, P, P, P, P, P]
        L.flod_preprocess.argtypes = [P, I, P, I, P, P, SZ, U64, P]
        L.flod_bin_sort.argtypes = [P, I, P, I, P, P, SZ, U64, P, P]
        L.flod_bin_sort_phase.argtypes = [P, I, P, I, P, P, SZ, U64, P, I, P]
        L.flod_render_fwd.argtypes = [P, I, P, I, P, P, SZ, U64, P, P, P, P]
        L.flod_render_bwd.argtypes = [P, I, P, I, P, P, SZ, U64, P, P, P, P, P]
        L.flod_blend_bwd.argtypes = [P, I, P, I, P, P, SZ, U64, P, P, P, P]
        L.flod_preprocess_bwd.argtypes = [P, I, P, I, P, P, SZ, U64, P, P]
        L.flod_select_scratch_size.argtypes = [P, I]
        L.flod_select_scratch_size.restype = SZ
        L.flod_select_levels.argtypes = [P, I, P, C.c_float, C.c_float, P, P, C.c_uint32, P, P,
                                         SZ, P]
        L.flod_select_levels_noalloc.argtypes = [P, I, P, C.c_float, C.c_float, P, P,
                                                 C.c_uint32, P, P]
        L.flod_adjust_scale.argtypes = [P, C.c_int64, C.c_float, C.c_float, P]
        L.flod_loss_scratch_size.argtypes = [P, P, I]
        L.flod_loss_scratch_size.restype = SZ
        L.flod_loss.argtypes = [P, P, P, P, I, C.c_float, P, P, P, SZ, P]
        L.flod_adam_step.argtypes = [P, P, P, P, P, P, I, P, P]
        L.flod_preprocess_bwd_adam.argtypes = [P, I, P, I, P, P, SZ, U64, P, P, P]
        L.flod_gather.argtypes = [P, I, P, P, C.c_uint32, P, I, I, P, P]
        L.flod_densify_stats.argtypes = [P, I, P, I, P, P, SZ, U64, P, P, P]
        L.flod_densify_scratch_size.argtypes = [I]
        L.flod_densify_scratch_size.restype = SZ
        L.flod_densify.argtypes = [P, P, P, P, C.c_float, C.c_float, C.c_float, P, P, P, P, P,
                                   C.c_uint32, P, P, P, SZ, P]
        L.flod_prune_scratch_size.argtypes = [I]
        L.flod_prune_scratch_size.restype = SZ
        L.flod_overlap_prune.argtypes = [P, C.c_float, P, P, P, P, P, P, SZ, P]
        L.flod_read_status.argtypes = [P, P, P]
        L.flod_status_string.argtypes = [I]
        L.flod_status_string.restype = C.c_char_p
        for name in ("flod_workspace_layout", "flod_preprocess", "flod_bin_sort",
                     "flod_bin_sort_phase",
                     "flod_render_fwd", "flod_render_bwd", "flod_blend_bwd",
                     "flod_preprocess_bwd", "flod_select_levels", "flod_select_levels_noalloc",
                     "flod_adjust_scale", "flod_read_status", "flod_loss", "flod_adam_step",
                     "flod_preprocess_bwd_adam", "flod_gather", "flod_overlap_prune",
                     "flod_densify_stats", "flod_densify"):
            getattr(L, name).restype = I
        _lib = L
    return _lib


def _check(status: int, what: str):
    if status != 0:
        raise FlodError(f"{what}: {STATUS.get(status, status)}")


def _stream(stream=None) -> int:
    s = torch.cuda.current_stream() if stream is None else stream
    return s.cuda_stream


def _ptr(t) -> int | None:
    return None if t is None else t.data_ptr()


# ---------------------------------------------------------------------------------------
# struct builders
# ---------------------------------------------------------------------------------------

def default_config(**kw) -> RasterConfig:
    c = RasterConfig()
    lib().flod_default_config(C.byref(c))
    for k, v in kw.items():
        if k == "bg":
            c.bg = (C.c_float * 3)(*v)
        else:
            setattr(c, k, v)
    return c


def camera_struct(cam: dict) -> Camera:
    c = Camera()
    c.viewmat = (C.c_float * 12)(*np.asarray(cam["viewmat"], dtype=np.float32).reshape(-1))
    c.fx, c.fy, c.cx, c.cy = cam["fx"], cam["fy"], cam["cx"], cam["cy"]
    c.width, c.height = int(cam["width"]), int(cam["height"])
    c.cam_pos = (C.c_float * 3)(*np.asarray(cam["cam_pos"], dtype=np.float32))
    return c


class GaussianSet:
    """Device-resident SoA parameters of one Gaussian set (one FLoD level)."""

    FIELDS = ("means", "quats", "s_opt", "opacity_logit", "sh")

    def __init__(self, means, quats, s_opt, opacity_logit, sh, sh_degree: int, s_min: float):
        self.means, self.quats, self.s_opt = means, quats, s_opt
        self.opacity_logit, self.sh = opacity_logit, sh
        self.sh_degree = int(sh_degree)
        self.s_min = float(s_min)
        for f in self.FIELDS:
            t = getattr(self, f)
            if not (t.is_cuda and t.dtype == torch.float32 and t.is_contiguous()):
                raise FlodError(f"{f} must be a contiguous float32 CUDA tensor")

    @classmethod
    def from_numpy(cls, g: dict, s_min: float, device="cuda"):
        t = {k: torch.as_tensor(np.ascontiguousarray(g[k], dtype=np.float32), device=device)
             for k in cls.FIELDS}
        return cls(**t, sh_degree=g["sh_degree"], s_min=s_min)

    @property
    def n(self) -> int:
        return self.means.shape[0]

    def struct(self) -> Gaussians:
        s = Gaussians()
        s.means, s.quats, s.s_opt = _ptr(self.means), _ptr(self.quats), _ptr(self.s_opt)
        s.opacity_logit, s.sh = _ptr(self.opacity_logit), _ptr(self.sh)
        s.n, s.sh_degree, s.s_min = self.n, self.sh_degree, self.s_min
        return s


def view_struct(cam: dict, set_index: int = 0, sel=None, sel_count=None, sel_capacity: int = 0) -> View:
    v = View()
    v.cam = camera_struct(cam)
    v.set = set_index
    v.sel = _ptr(sel)
    v.sel_count = _ptr(sel_count)
    v.sel_capacity = sel_capacity if sel is not None else 0
    return v


def _array(typ, items):
    return (typ * len(items))(*items)


# ---------------------------------------------------------------------------------------
# one-to-one wrappers of the C entry points
# ---------------------------------------------------------------------------------------

def flod_workspace_size(sets, views, pair_capacity: int, cfg: RasterConfig) -> int:
    n = lib().flod_workspace_size(sets, len(sets), views, len(views), pair_capacity, C.byref(cfg))
    if n == 0:
        raise FlodError("flod_workspace_size: invalid arguments")
    return n


def flod_workspace_layout(sets, views, pair_capacity: int, cfg: RasterConfig):
    lay = WsLayout()
    nv = len(views)
    uo, to, po = ((C.c_uint64 * (nv + 1))() for _ in range(3))
    _check(lib().flod_workspace_layout(sets, len(sets), views, nv, pair_capacity, C.byref(cfg),
                                       C.byref(lay), uo, to, po), "flod_workspace_layout")
    return lay, list(uo), list(to), list(po)


def flod_preprocess(sets, views, cfg, ws: torch.Tensor, pair_capacity: int, stream=None):
    _check(lib().flod_preprocess(sets, len(sets), views, len(views), C.byref(cfg), ws.data_ptr(),
                                 ws.numel(), pair_capacity, _stream(stream)), "flod_preprocess")


def flod_bin_sort(sets, views, cfg, ws: torch.Tensor, pair_capacity: int, d_pair_count=None,
                  stream=None):
    _check(lib().flod_bin_sort(sets, len(sets), views, len(views), C.byref(cfg), ws.data_ptr(),
                               ws.numel(), pair_capacity, _ptr(d_pair_count), _stream(stream)),
           "flod_bin_sort")


#: flod_bin_sort_phase phases, in call order
BIN_PHASE_DEPTH, BIN_PHASE_EMIT, BIN_PHASE_TILES, BIN_PHASE_RANGES = 1, 2, 3, 4


def flod_bin_sort_phase(sets, views, cfg, ws: torch.Tensor, pair_capacity: int, phase: int,
                        d_pair_count=None, stream=None):
    _check(lib().flod_bin_sort_phase(sets, len(sets), views, len(views), C.byref(cfg),
                                     ws.data_ptr(), ws.numel(), pair_capacity, _ptr(d_pair_count),
                                     phase, _stream(stream)), "flod_bin_sort_phase")


def flod_render_fwd(sets, views, cfg, ws, pair_capacity, out_rgb, out_T, out_nc, stream=None):
    _check(lib().flod_render_fwd(sets, len(sets), views, len(views), C.byref(cfg), ws.data_ptr(),
                                 ws.numel(), pair_capacity, out_rgb.data_ptr(), out_T.data_ptr(),
                                 out_nc.data_ptr(), _stream(stream)), "flod_render_fwd")


def flod_render_bwd(sets, views, cfg, ws, pair_capacity, dL_drgb, fwd_T, fwd_nc, grads,
                    stream=None):
    _check(lib().flod_render_bwd(sets, len(sets), views, len(views), C.byref(cfg), ws.data_ptr(),
                                 ws.numel(), pair_capacity, dL_drgb.data_ptr(), fwd_T.data_ptr(),
                                 fwd_nc.data_ptr(), grads, _stream(stream)), "flod_render_bwd")


def flod_blend_bwd(sets, views, cfg, ws, pair_capacity, dL_drgb, fwd_T, fwd_nc, stream=None):
    _check(lib().flod_blend_bwd(sets, len(sets), views, len(views), C.byref(cfg), ws.data_ptr(),
                                ws.numel(), pair_capacity, dL_drgb.data_ptr(), fwd_T.data_ptr(),
                                fwd_nc.data_ptr(), _stream(stream)), "flod_blend_bwd")


def flod_preprocess_bwd(sets, views, cfg, ws, pair_capacity, grads, stream=None):
    _check(lib().flod_preprocess_bwd(sets, len(sets), views, len(views), C.byref(cfg),
                                     ws.data_ptr(), ws.numel(), pair_capacity, grads,
                                     _stream(stream)), "flod_preprocess_bwd")


#: flod_grads.overwrite values
GRAD_ACCUMULATE, GRAD_OVERWRITE, GRAD_ZERO_FIRST = 0, 1, 2


def grads_struct(grads, overwrite=False):
    """grads: per set, a sequence of 5 tensors (or None) in GaussianSet.FIELDS order.
    overwrite: one flod_grads.overwrite value for every set, or a sequence with one per set
    (0 / False: add to the buffers; 1 / True: write every gradient of a set rendered by one
    view; 2: the library zero-fills the buffers first, then adds)."""
    modes = list(overwrite) if isinstance(overwrite, (list, tuple)) else [overwrite] * len(grads)
    if len(modes) != len(grads):
        raise FlodError("grads_struct: one overwrite value per set")
    return _array(Grads, [Grads(*[_ptr(t) for t in gr], int(m)) for gr, m in zip(grads, modes)])


def flod_select_scratch_size(levels) -> int:
    arr = _array(Gaussians, [g.struct() if isinstance(g, GaussianSet) else g for g in levels])
    return lib().flod_select_scratch_size(arr, len(levels))


def flod_select_levels(levels, origin, out_sel: torch.Tensor, d_count: torch.Tensor,
                       scratch: torch.Tensor, d_thresh=None, gamma: float = 1.0,
                       focal: float = 0.0, stream=None):
    arr = _array(Gaussians, [g.struct() if isinstance(g, GaussianSet) else g for g in levels])
    th = None if d_thresh is None else _array(C.c_float, [float(x) for x in d_thresh])
    org = _array(C.c_float, [float(x) for x in origin])
    _check(lib().flod_select_levels(arr, len(levels), th, gamma, focal, org, out_sel.data_ptr(),
                                    out_sel.numel(), d_count.data_ptr(), scratch.data_ptr(),
                                    scratch.numel(), _stream(stream)), "flod_select_levels")


SELECT_NOALLOC_MAX_BLOCKS = 16384


def flod_select_levels_noalloc(levels, origin, out_sel: torch.Tensor, d_count: torch.Tensor,
                               d_thresh=None, gamma: float = 1.0, focal: float = 0.0,
                               stream=None):
    """flod_select_levels for callers that cannot allocate device memory: the library's own
    fixed scratch replaces the caller's (at most 2^25 Gaussians over all levels; calls that
    overlap on the GPU race on that scratch). The first call on a device looks the scratch up;
    make it before any stream capture."""
    arr = _array(Gaussians, [g.struct() if isinstance(g, GaussianSet) else g for g in levels])
    blocks = sum(-(-int(g.n) // 2048) for g in arr)
    if blocks > SELECT_NOALLOC_MAX_BLOCKS:
        raise FlodError(f"flod_select_levels_noalloc: {blocks} blocks of 2048 Gaussians exceed the "
                        f"fixed scratch ({SELECT_NOALLOC_MAX_BLOCKS} blocks)")
    th = None if d_thresh is None else _array(C.c_float, [float(x) for x in d_thresh])
    org = _array(C.c_float, [float(x) for x in origin])
    _check(lib().flod_select_levels_noalloc(arr, len(levels), th, gamma, focal, org,
                                            out_sel.data_ptr(), out_sel.numel(),
                                            d_count.data_ptr(), _stream(stream)),
           "flod_select_levels_noalloc")


# ---------------------------------------------------------------------------------------
# training step: loss and Adam
# ---------------------------------------------------------------------------------------

#: the loss weight and the Adam settings of the 3DGS backbone the paper keeps (Sec. 5.1.4)
LOSS_LAMBDA = 0.2
ADAM_BETAS = (0.9, 0.999)
ADAM_EPS = 1e-15


def param_arrays(tensors) -> ParamArrays:
    """ParamArrays of five tensors in GaussianSet.FIELDS order."""
    return ParamArrays(*[_ptr(t) for t in tensors])


def flod_loss_scratch_size(sizes) -> int:
    """sizes: [(width, height), ...] of the images."""
    w = _array(C.c_int, [int(a) for a, _ in sizes])
    h = _array(C.c_int, [int(b) for _, b in sizes])
    n = lib().flod_loss_scratch_size(w, h, len(sizes))
    if n == 0:
        raise FlodError("flod_loss_scratch_size: invalid sizes")
    return n


def flod_loss(img: torch.Tensor, target: torch.Tensor, sizes, dL: torch.Tensor,
              scratch: torch.Tensor, d_loss: torch.Tensor | None = None,
              lam: float = LOSS_LAMBDA, stream=None):
    w = _array(C.c_int, [int(a) for a, _ in sizes])
    h = _array(C.c_int, [int(b) for _, b in sizes])
    _check(lib().flod_loss(img.data_ptr(), target.data_ptr(), w, h, len(sizes), lam,
                           _ptr(d_loss), dL.data_ptr(), scratch.data_ptr(), scratch.numel(),
                           _stream(stream)), "flod_loss")


def adam_config(lrs: dict, d_step: torch.Tensor, betas=ADAM_BETAS, eps=ADAM_EPS) -> AdamConfig:
    """lrs: means, quats, s_opt, opacity_logit, sh_dc, sh_rest; d_step: a device int32 [1]
    counter of the steps taken (start at 0)."""
    return AdamConfig(lrs["means"], lrs["quats"], lrs["s_opt"], lrs["opacity_logit"],
                      lrs["sh_dc"], lrs["sh_rest"], betas[0], betas[1], eps, d_step.data_ptr())


def flod_adam_step(params, grads, m, v, ns, sh_degrees, cfg: AdamConfig, stream=None):
    """One Adam step of several sets: params, grads, m, v are per-set lists of five tensors
    (GaussianSet.FIELDS order); ns, sh_degrees per set."""
    k = len(params)
    P_, G_, M_, V_ = (_array(ParamArrays, [param_arrays(t) for t in x]) for x in (params, grads, m, v))
    _check(lib().flod_adam_step(P_, G_, M_, V_, _array(C.c_int, [int(n) for n in ns]),
                                _array(C.c_int, [int(d) for d in sh_degrees]), k, C.byref(cfg),
                                _stream(stream)), "flod_adam_step")


def adam_states(states) -> C.Array:
    """states: per set, (params out, m, v), each five tensors."""
    return _array(AdamState, [AdamState(param_arrays(p), param_arrays(m), param_arrays(v))
                              for p, m, v in states])


def flod_preprocess_bwd_adam(sets, views, cfg, ws, pair_capacity, states_c, acfg: AdamConfig,
                             stream=None):
    _check(lib().flod_preprocess_bwd_adam(sets, len(sets), views, len(views), C.byref(cfg),
                                          ws.data_ptr(), ws.numel(), pair_capacity, states_c,
                                          C.byref(acfg), _stream(stream)),
           "flod_preprocess_bwd_adam")


def flod_gather(sets, entries, d_count, capacity: int, out, out_sh_degree: int,
                fold_s_min: bool = False, out_s_min=None, stream=None):
    """sets: GaussianSets (or Gaussians structs, e.g. of host-mapped arrays); entries: device
    int32 selection entries or None (identity over set 0); d_count: device int32 [1]; out:
    five device tensors with room for `capacity` Gaussians."""
    arr = _array(Gaussians, [g.struct() if isinstance(g, GaussianSet) else g for g in sets])
    o = param_arrays(out)
    _check(lib().flod_gather(arr, len(sets), _ptr(entries), d_count.data_ptr(), capacity,
                             C.byref(o), out_sh_degree, int(fold_s_min), _ptr(out_s_min),
                             _stream(stream)), "flod_gather")


def gather_set(sets, entries, d_count, capacity: int, sh_degree: int, fold_s_min=True,
               device="cuda", stream=None) -> "GaussianSet":
    """A new GaussianSet of `capacity` Gaussians gathered by flod_gather (s_min 0 when folded;
    entries past *d_count are left zero)."""
    K = (sh_degree + 1) ** 2
    out = [torch.zeros(capacity, 3, device=device), torch.zeros(capacity, 4, device=device),
           torch.zeros(capacity, 3, device=device), torch.zeros(capacity, device=device),
           torch.zeros(capacity, K, 3, device=device)]
    flod_gather(sets, entries, d_count, capacity, out, sh_degree, fold_s_min, None, stream)
    s_min = 0.0 if fold_s_min else (sets[0].s_min if isinstance(sets[0], GaussianSet) else sets[0].s_min)
    return GaussianSet(*out, sh_degree=sh_degree, s_min=s_min)


def flod_overlap_prune(gs: "GaussianSet", d_op: float, keep: torch.Tensor, d_kept: torch.Tensor,
                       scratch: torch.Tensor, d_avg=None, out_kept=None, d_status=None,
                       stream=None):
    st = gs.struct()
    _check(lib().flod_overlap_prune(C.byref(st), d_op, keep.data_ptr(), _ptr(d_avg),
                                    _ptr(out_kept), d_kept.data_ptr(), _ptr(d_status),
                                    scratch.data_ptr(), scratch.numel(), _stream(stream)),
           "flod_overlap_prune")


def overlap_prune(gs: "GaussianSet", d_op: float | None = None, stream=None):
    """Overlap pruning of one level (Sec. 4.3) with d_OP = s_min / 2 by default: returns
    (the pruned GaussianSet, the keep mask). Reads the kept count back (synchronises)."""
    dev = gs.means.device
    d_op = 0.5 * gs.s_min if d_op is None else d_op
    n = gs.n
    keep = torch.empty(max(n, 1), dtype=torch.uint8, device=dev)
    kept = torch.empty(max(n, 1), dtype=torch.int32, device=dev)
    cnt = torch.zeros(1, dtype=torch.int32, device=dev)
    scr = torch.empty(flod_prune_scratch_size(n) + 256, dtype=torch.uint8, device=dev)
    scr = scr[(-scr.data_ptr()) % 256:][:flod_prune_scratch_size(n)]
    flod_overlap_prune(gs, d_op, keep, cnt, scr, out_kept=kept, stream=stream)
    m = int(cnt.item())
    out = gather_set([gs], kept, cnt, max(m, 1), gs.sh_degree, fold_s_min=False, device=dev,
                     stream=stream)
    return GaussianSet(*[getattr(out, f)[:m] for f in GaussianSet.FIELDS], gs.sh_degree,
                       gs.s_min), keep[:n]


def flod_densify_stats(sets, views, cfg, ws, pair_capacity, accum, denom, stream=None):
    """accum, denom: per set a device float tensor [n] (or None to skip the set)."""
    a = (C.c_void_p * len(accum))(*[_ptr(t) for t in accum])
    d = (C.c_void_p * len(denom))(*[_ptr(t) for t in denom])
    _check(lib().flod_densify_stats(sets, len(sets), views, len(views), C.byref(cfg),
                                    ws.data_ptr(), ws.numel(), pair_capacity, a, d,
                                    _stream(stream)), "flod_densify_stats")


#: density-control settings of the 3DGS backbone (gradient threshold, the fraction of the
#: scene extent below which a Gaussian is cloned rather than split, minimum opacity)
DENSIFY_TAU, PERCENT_DENSE, MIN_OPACITY = 2e-4, 0.01, 0.005


def densify(gs: "GaussianSet", accum, denom, normals, tau=DENSIFY_TAU, max_clone_scale=None,
            extent: float = 1.0, min_opacity=MIN_OPACITY, m=None, v=None, stream=None):
    """The density-control step of one level: returns (new GaussianSet, new m, new v,
    (kept in place, clones, split)); m, v are five tensors each or None. Reads the new size
    back (synchronises)."""
    dev = gs.means.device
    n = gs.n
    mcs = PERCENT_DENSE * extent if max_clone_scale is None else max_clone_scale
    cap = 3 * n + 1
    K = (gs.sh_degree + 1) ** 2

    def arrays():
        return [torch.zeros(cap, 3, device=dev), torch.zeros(cap, 4, device=dev),
                torch.zeros(cap, 3, device=dev), torch.zeros(cap, device=dev),
                torch.zeros(cap, K, 3, device=dev)]
    out = arrays()
    mo, vo = (arrays(), arrays()) if m is not None else (None, None)
    cnt = torch.zeros(1, dtype=torch.int32, device=dev)
    c3 = torch.zeros(3, dtype=torch.int32, device=dev)
    nb = lib().flod_densify_scratch_size(n)
    scr = torch.empty(max(nb, 4), dtype=torch.uint8, device=dev)
    st = gs.struct()
    pa = [C.byref(param_arrays(x)) if x is not None else None for x in (m, v, out, mo, vo)]
    _check(lib().flod_densify(C.byref(st), accum.data_ptr(), denom.data_ptr(), normals.data_ptr(),
                              tau, mcs, min_opacity, pa[0], pa[1], pa[2], pa[3], pa[4], cap,
                              cnt.data_ptr(), c3.data_ptr(), scr.data_ptr(), scr.numel(),
                              _stream(stream)), "flod_densify")
    k = int(cnt.item())
    new = GaussianSet(*[t[:k] for t in out], gs.sh_degree, gs.s_min)
    return (new, None if mo is None else [t[:k] for t in mo],
            None if vo is None else [t[:k] for t in vo], tuple(int(x) for x in c3.cpu()))


def flod_prune_scratch_size(n: int) -> int:
    return lib().flod_prune_scratch_size(int(n))


def flod_adjust_scale(s_opt: torch.Tensor, s_min_cur: float, s_min_next: float, stream=None):
    _check(lib().flod_adjust_scale(s_opt.data_ptr(), s_opt.numel(), s_min_cur, s_min_next,
                                   _stream(stream)), "flod_adjust_scale")


def flod_read_status(ws: torch.Tensor, stream=None) -> int:
    v = C.c_uint32(0)
    _check(lib().flod_read_status(ws.data_ptr(), C.byref(v), _stream(stream)), "flod_read_status")
    return v.value


# ---------------------------------------------------------------------------------------
# convenience: one batch of views over a list of Gaussian sets
# ---------------------------------------------------------------------------------------

class Rasterizer:
    """Runs preprocess -> bin_sort -> render_fwd (and render_bwd) for one batch of views.

    The workspace is a torch uint8 tensor sized by flod_workspace_size for ``pair_capacity``.
    ``ensure_capacity`` regrows it when the last bin_sort reported more pairs (this reads the
    pair count back, so it synchronises; timed loops size the workspace once)."""

    def __init__(self, sets, views, cfg: RasterConfig | None = None, pair_capacity: int | None = None):
        self.sets = list(sets)
        self.cfg = cfg if cfg is not None else default_config()
        self.views = list(views)
        self.refresh_structs()
        npix = sum(v.cam.width * v.cam.height for v in self.views)
        units = sum(v.sel_capacity if v.sel else self.sets[v.set].n for v in self.views)
        if pair_capacity is None:
            pair_capacity = max(1 << 16, min(MAX_PAIRS, 4 * units + npix // 16))
        self.pair_capacity = int(pair_capacity)
        self._alloc()
        dev = self.sets[0].means.device
        self.pair_count = torch.zeros(1, dtype=torch.int64, device=dev)
        self.npix = npix
        self.generation = 0     # workspace rewrites so far (preprocess, bin_sort calls)
        _, self.unit_off, self.tile_off, self.pix_off = flod_workspace_layout(
            self.c_sets, self.c_views, self.pair_capacity, self.cfg)

    def refresh_structs(self):
        self.c_sets = _array(Gaussians, [s.struct() for s in self.sets])
        self.c_views = _array(View, self.views)

    def _alloc(self):
        n = flod_workspace_size(self.c_sets, self.c_views, self.pair_capacity, self.cfg)
        dev = self.sets[0].means.device
        self.ws = torch.zeros(n + 256, dtype=torch.uint8, device=dev)
        off = (-self.ws.data_ptr()) % 256
        self.ws = self.ws[off:off + n]
        self.layout = flod_workspace_layout(self.c_sets, self.c_views, self.pair_capacity, self.cfg)[0]

    def new_outputs(self):
        dev = self.sets[0].means.device
        return (torch.empty(3 * self.npix, dtype=torch.float32, device=dev),
                torch.empty(self.npix, dtype=torch.float32, device=dev),
                torch.empty(self.npix, dtype=torch.int32, device=dev))

    def preprocess(self, stream=None):
        self.generation += 1
        flod_preprocess(self.c_sets, self.c_views, self.cfg, self.ws, self.pair_capacity, stream)

    def bin_sort(self, stream=None):
        self.generation += 1
        flod_bin_sort(self.c_sets, self.c_views, self.cfg, self.ws, self.pair_capacity,
                      self.pair_count, stream)

    def bin_sort_phase(self, phase: int, stream=None):
        """One part of bin_sort (BIN_PHASE_*); the four in order equal bin_sort."""
        self.generation += 1
        flod_bin_sort_phase(self.c_sets, self.c_views, self.cfg, self.ws, self.pair_capacity,
                            phase, self.pair_count, stream)

    def render_fwd(self, out_rgb, out_T, out_nc, stream=None):
        flod_render_fwd(self.c_sets, self.c_views, self.cfg, self.ws, self.pair_capacity, out_rgb,
                        out_T, out_nc, stream)

    def render_bwd(self, dL, out_T, out_nc, grads, stream=None, overwrite=False):
        flod_render_bwd(self.c_sets, self.c_views, self.cfg, self.ws, self.pair_capacity, dL, out_T,
                        out_nc, grads_struct(grads, overwrite), stream)

    def blend_bwd(self, dL, out_T, out_nc, stream=None):
        flod_blend_bwd(self.c_sets, self.c_views, self.cfg, self.ws, self.pair_capacity, dL, out_T,
                       out_nc, stream)

    def preprocess_bwd(self, grads_c, stream=None):
        """grads_c: the result of grads_struct (built once, reused every step)."""
        flod_preprocess_bwd(self.c_sets, self.c_views, self.cfg, self.ws, self.pair_capacity,
                            grads_c, stream)

    def preprocess_bwd_adam(self, states_c, acfg: AdamConfig, stream=None):
        """states_c: the result of adam_states (built once, reused every step)."""
        flod_preprocess_bwd_adam(self.c_sets, self.c_views, self.cfg, self.ws, self.pair_capacity,
                                 states_c, acfg, stream)

    def densify_stats(self, accum, denom, stream=None):
        """Accumulate the density-control statistics of the last blending backward."""
        flod_densify_stats(self.c_sets, self.c_views, self.cfg, self.ws, self.pair_capacity,
                           accum, denom, stream)

    def eval_counts(self):
        """Running counts of (pixel, Gaussian) pairs: (forward evaluations, backward
        evaluations, pairs the forward blended)."""
        plan = self.region("plan", torch.int64, 32)
        return int(plan[24].item()), int(plan[25].item()), int(plan[26].item())

    def ensure_capacity(self) -> bool:
        """True if the last bin_sort fitted; otherwise regrow (caller re-runs the stages)."""
        p = int(self.pair_count.item())
        if p <= self.pair_capacity:
            return True
        if p > MAX_PAIRS:
            raise FlodError(f"{p} pairs exceed the library maximum {MAX_PAIRS}")
        self.pair_capacity = min(MAX_PAIRS, int(p * 1.25) + 1024)
        self._alloc()
        return False

    def forward(self, stream=None, check_capacity: bool = True):
        """preprocess -> bin_sort (regrowing the pair capacity if needed) -> render_fwd.
        check_capacity=False skips the host read of the pair count (no synchronisation; an
        overflow then only sets FLOD_DEV_CAPACITY in the status word)."""
        out = self.new_outputs()
        if not check_capacity:
            self.preprocess(stream)
            self.bin_sort(stream)
            self.render_fwd(*out, stream)
            return out
        for _ in range(3):
            self.preprocess(stream)
            self.bin_sort(stream)
            if self.ensure_capacity():
                break
        else:
            raise FlodError("pair capacity did not converge in three attempts")
        self.render_fwd(*out, stream)
        return out

    def grad_modes(self):
        """Per set, the cheapest legal flod_grads.overwrite value for a backward into fresh
        (uninitialised) buffers: 1 where exactly one view renders the set as a whole set and
        no view uses a selection list, else 2 (zero-filled by the library first)."""
        direct = [0] * len(self.sets)
        n_sel = 0
        for v in self.views:
            if v.sel:
                n_sel += 1
            else:
                direct[v.set] += 1
        return [GRAD_OVERWRITE if d == 1 and n_sel == 0 else GRAD_ZERO_FIRST for d in direct]

    def region(self, name: str, dtype, count: int, index: int | None = None) -> torch.Tensor:
        """A typed view of a workspace region (for tests and diagnostics)."""
        off = getattr(self.layout, name)
        if index is not None:
            off = off[index]
        nbytes = torch.tensor([], dtype=dtype).element_size() * count
        return self.ws[off:off + nbytes].view(dtype)


def image_views(flat: torch.Tensor, views, channels: int = 1):
    """Split a concatenated per-view output into [channels, H, W] tensors."""
    out, off = [], 0
    for v in views:
        n = v.cam.width * v.cam.height * channels
        out.append(flat[off:off + n].view(channels, v.cam.height, v.cam.width))
        off += n
    return out


# ---------------------------------------------------------------------------------------
# autograd
# ---------------------------------------------------------------------------------------

class _Rasterize(torch.autograd.Function):
    @staticmethod
    def forward(ctx, rast: Rasterizer, check_capacity: bool, *params):
        rgb, T, nc = rast.forward(check_capacity=check_capacity)
        ctx.rast = rast
        # the backward re-walks the workspace this forward sorted: remember which one
        ctx.generation = rast.generation
        ctx.ws_ptr = rast.ws.data_ptr()
        ctx.save_for_backward(T, nc)
        ctx.mark_non_differentiable(T, nc)
        return rgb, T, nc

    @staticmethod
    def backward(ctx, d_rgb, d_T, d_nc):
        rast = ctx.rast
        if rast.generation != ctx.generation or rast.ws.data_ptr() != ctx.ws_ptr:
            raise FlodError("rasterize backward: the Rasterizer ran another forward (or regrew "
                            "its workspace) after this one; its sorted pairs are gone. Use one "
                            "Rasterizer per differentiated render.")
        T, nc = ctx.saved_tensors
        # fresh buffers, written (or zero-filled) by the library itself: no torch fill kernels
        grads = [[torch.empty_like(getattr(s, f)) for f in GaussianSet.FIELDS] for s in rast.sets]
        rast.render_bwd(d_rgb.contiguous(), T, nc, grads, overwrite=rast.grad_modes())
        flat = [g for per_set in grads for g in per_set]
        return (None, None, *flat)


def rasterize(rast: Rasterizer, check_capacity: bool = True):
    """Differentiable render of every view of ``rast``: returns (rgb, T, n_contrib), the
    concatenated per-view outputs; gradients flow to every parameter tensor of every set
    (each set's tensors must have requires_grad set by the caller). check_capacity=False
    skips the pair-capacity read-back (for loops that sized the capacity once)."""
    params = [getattr(s, f) for s in rast.sets for f in GaussianSet.FIELDS]
    return _Rasterize.apply(rast, check_capacity, *params)


def focal_from_hfov(width: int, hfov_deg: float) -> float:
    return width / (2.0 * math.tan(math.radians(hfov_deg) / 2.0))
