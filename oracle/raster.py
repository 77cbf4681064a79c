"""Preprocess, binning and depth-ordered alpha blending, FP64, plus their gradient.

What is computed (Sec. 3, Eq. 1, Eq. 2 and the sentence after it: the image is the alpha
blend of the projected Gaussians in depth order), with the readings of what the paper
leaves open (the rasterizer is that of the 3DGS framework the paper builds on, Sec. 5.1.4):

* opacity o = sigmoid(logit); per pixel alpha = min(0.99, o exp(-q/2)) with
  q = d^T Sigma'^-1 d, d = pixel centre - mu';
* front to back in (view depth t_z, Gaussian index) order: a Gaussian with
  alpha < 1/255 is skipped; if T (1 - alpha) < 1e-4 blending stops before that Gaussian;
  otherwise C += rgb alpha T and T <- T (1 - alpha); output C + T bg;
* n_contrib = 1-based position, in the tile's list, of the last blended Gaussian.

Two renders are written: ``render_brute`` blends, for every pixel, all Gaussians of the
scene (the definition); ``render_tiled`` blends only the Gaussians binned to the pixel's
tile, in the order of the sorted (tile, depth) keys. With the opacity-aware extent the
two are equal (the skipped Gaussians are exactly the ones the tiles leave out).

The gradient is the derivative of this piecewise-smooth forward taken by torch autograd
(library differentiation of the code above; the discrete decisions -- culling, rectangles,
skip, early stop -- are constants of the derivative).
"""
from __future__ import annotations

from dataclasses import dataclass, field

import numpy as np
import torch

from . import gaussians as G
from . import projection as P
from . import sh as SH

ALPHA_MAX = 0.99
ALPHA_MIN = 1.0 / 255.0
T_MIN = 1e-4


@dataclass
class Config:
    tile_w: int = 16
    tile_h: int = 16
    dilation: float = 0.3
    z_near: float = 0.2
    bg: tuple = (0.0, 0.0, 0.0)
    extent_rule: int = 2
    extra: dict = field(default_factory=dict)


def to_t(a, requires_grad=False) -> torch.Tensor:
    t = torch.as_tensor(np.asarray(a, dtype=np.float64)).clone()
    t.requires_grad_(requires_grad)
    return t


def params(g: dict, requires_grad=False) -> dict:
    return {k: to_t(g[k], requires_grad) for k in ("means", "quats", "s_opt", "opacity_logit", "sh")}


def preprocess(p: dict, sh_degree: int, s_min: float, cam: dict, cfg: Config) -> dict:
    """Per-Gaussian projection, colour, extent and tile rectangle for one camera."""
    s = G.constrained_scale(p["s_opt"], s_min)                       # Eq. 4
    cov3d = G.covariance(p["quats"], s)                                # Eq. 1
    t, mean2d, cov2d, in_front = P.project(p["means"], cov3d, cam, cfg.dilation, cfg.z_near)
    con, det = P.conic(cov2d)
    o = G.sigmoid(p["opacity_logit"])
    r, ok = P.radius(cov2d.detach(), o.detach(), 1 if cfg.extent_rule == 1 else 0)
    _, _, cam_pos = P.camera_tensors(cam)
    rgb, rgb_raw = SH.colour(p["sh"], p["means"], cam_pos, sh_degree)
    valid = in_front & (det.detach() > 0) & ok
    u, v = mean2d[:, 0].detach().numpy(), mean2d[:, 1].detach().numpy()
    ext, ok2 = P.ellipse_extent(cov2d.detach(), o.detach())   # the support ellipse
    if cfg.extent_rule == 2:
        valid = valid & ok2
        e = ext.numpy()
        px = P.pixel_rect_xy(u, v, e[:, 2], e[:, 3], cam["width"], cam["height"])
        segs, touched = P.ellipse_segments(u, v, e, px, cfg.tile_w, cfg.tile_h, valid.numpy())
        tr = P.tile_rect(px, cfg.tile_w, cfg.tile_h, valid.numpy() & (touched > 0))
    else:
        px = P.pixel_rect(u, v, r.numpy(), cam["width"], cam["height"])
        tr = P.tile_rect(px, cfg.tile_w, cfg.tile_h, valid.numpy())
        touched = tr[4]
        segs = P.rect_segments(tr[:4], touched)
    return {"mean2d": mean2d, "depth": t[:, 2], "conic": con, "opacity": o, "rgb": rgb,
            "rgb_raw": rgb_raw, "radius": r, "ext": ext, "valid": valid, "cov2d": cov2d,
            "t": t, "pixel_rect": px, "tile_rect": tr[:4], "segments": segs,
            "tiles_touched": touched}


def f32_bits(x) -> np.ndarray:
    return np.asarray(x, dtype=np.float32).view(np.uint32).astype(np.uint64)


def bin_segments(segments, depth_f32, tiles_x: int, n_tiles: int, tile_offset: int = 0,
                 unit_offset: int = 0):
    """(tile, depth) keys for every (Gaussian, covered tile), emitted in Gaussian order and
    within a Gaussian row by row, left to right, over its segments (unit, ty, cx0, cx1);
    key = tile << 32 | bits(depth). Returns (keys, values) unsorted, in emission order."""
    unit, ty, cx0, cx1 = (np.asarray(a, dtype=np.int64) for a in segments)
    w = cx1 - cx0 + 1
    s = np.repeat(np.arange(unit.size, dtype=np.int64), w)
    start = np.cumsum(w) - w
    tx = cx0[s] + (np.arange(s.size, dtype=np.int64) - start[s])
    tile = tile_offset + ty[s] * tiles_x + tx
    assert s.size == 0 or (tile.max() < tile_offset + n_tiles and tile.min() >= tile_offset)
    g = unit[s]
    keys = (tile.astype(np.uint64) << np.uint64(32)) | f32_bits(depth_f32)[g]
    return keys, (g + unit_offset).astype(np.uint32)


def bin_pairs(tile_rect, tiles_touched, depth_f32, tiles_x: int, n_tiles: int,
              tile_offset: int = 0, unit_offset: int = 0):
    """bin_segments over full tile rectangles (rules 0 and 1): row-major in each rectangle."""
    return bin_segments(P.rect_segments(tile_rect, tiles_touched), depth_f32, tiles_x, n_tiles,
                        tile_offset, unit_offset)


def sort_pairs(keys: np.ndarray, vals: np.ndarray):
    """Stable sort by key (ties keep emission order, i.e. Gaussian index order)."""
    order = np.argsort(keys, kind="stable")
    return keys[order], vals[order]


def tile_ranges(sorted_keys: np.ndarray, n_tiles_total: int) -> np.ndarray:
    """[start, end) of every tile in the sorted pair list, int64 [n_tiles_total, 2]."""
    tiles = (sorted_keys >> np.uint64(32)).astype(np.int64)
    out = np.zeros((n_tiles_total, 2), dtype=np.int64)
    if tiles.size:
        starts = np.searchsorted(tiles, np.arange(n_tiles_total), side="left")
        ends = np.searchsorted(tiles, np.arange(n_tiles_total), side="right")
        out[:, 0] = starts
        out[:, 1] = ends
        out[ends == starts] = 0
    return out


def alpha_raw(pix_xy: torch.Tensor, mean2d, con, o) -> torch.Tensor:
    """o exp(-q/2) for pixels [P,2] (centres) x Gaussians [K]: [P, K]."""
    dx = pix_xy[:, None, 0] - mean2d[None, :, 0]
    dy = pix_xy[:, None, 1] - mean2d[None, :, 1]
    q = con[None, :, 0] * dx * dx + 2.0 * con[None, :, 1] * dx * dy + con[None, :, 2] * dy * dy
    return o[None, :] * torch.exp(-0.5 * q)


def blend(a_raw: torch.Tensor, rgb: torch.Tensor, bg: torch.Tensor):
    """Front-to-back blend along dim 1 (already depth-ordered). Returns (colour [P,3],
    T_final [P], last [P] 1-based position of the last blended Gaussian, 0 if none)."""
    a = torch.clamp(a_raw, max=ALPHA_MAX)
    kept = (a >= ALPHA_MIN).detach()
    a = torch.where(kept, a, torch.zeros_like(a))
    t_after = torch.cumprod(1.0 - a, dim=1)
    live = (t_after >= T_MIN).detach()
    a = torch.where(live, a, torch.zeros_like(a))
    one_minus = 1.0 - a
    t_incl = torch.cumprod(one_minus, dim=1)
    ones = torch.ones((a.shape[0], 1), dtype=a.dtype)
    t_before = torch.cat([ones, t_incl[:, :-1]], dim=1)
    w = a * t_before
    t_final = t_incl[:, -1] if t_incl.shape[1] else ones[:, 0]
    col = w @ rgb + t_final[:, None] * bg[None, :]
    blended = (kept & live).numpy()
    pos = np.arange(1, blended.shape[1] + 1)[None, :]
    if blended.shape[1]:
        last = np.max(np.where(blended, pos, 0), axis=1)
    else:
        last = np.zeros(blended.shape[0], dtype=np.int64)
    return col, t_final, last


def _pixel_centres(xs, ys) -> torch.Tensor:
    gx, gy = np.meshgrid(xs, ys)
    return torch.as_tensor(np.stack([gx.ravel() + 0.5, gy.ravel() + 0.5], 1).astype(np.float64))


def depth_order(depth: torch.Tensor, idx: np.ndarray) -> np.ndarray:
    """Gaussian indices ``idx`` ordered by (depth, index)."""
    d = depth.detach().numpy()[idx]
    return idx[np.lexsort((idx, d))]


def render_brute(pre: dict, cam: dict, cfg: Config, pixels=None):
    """The definition: every pixel blends every valid Gaussian in (depth, index) order.
    ``pixels`` (optional [P,2] int x,y) restricts the output to those pixels."""
    W, H = cam["width"], cam["height"]
    idx = np.nonzero(pre["valid"].numpy())[0]
    order = depth_order(pre["depth"], idx)
    if pixels is None:
        pix = _pixel_centres(np.arange(W), np.arange(H))
    else:
        pix = torch.as_tensor(np.asarray(pixels, dtype=np.float64) + 0.5)
    bg = torch.as_tensor(np.asarray(cfg.bg, dtype=np.float64))
    sel = torch.as_tensor(order)
    a = alpha_raw(pix, pre["mean2d"][sel], pre["conic"][sel], pre["opacity"][sel])
    col, tf, _ = blend(a, pre["rgb"][sel], bg)
    if pixels is not None:
        return col, tf
    return col.T.reshape(3, H, W), tf.reshape(H, W)


def tile_lists(pre: dict, cam: dict, cfg: Config):
    """Sorted (tile, depth) pairs of one camera from the oracle's own FP64 preprocess."""
    W, H = cam["width"], cam["height"]
    tiles_x = -(-W // cfg.tile_w)
    tiles_y = -(-H // cfg.tile_h)
    keys, vals = bin_segments(pre["segments"], pre["depth"].detach().numpy(), tiles_x,
                              tiles_x * tiles_y)
    keys, vals = sort_pairs(keys, vals)
    return keys, vals, tile_ranges(keys, tiles_x * tiles_y), tiles_x, tiles_y


def tile_pixels(tile: int, tiles_x: int, cam: dict, cfg: Config):
    """Pixel bounds (x0, y0, x1, y1), end exclusive, of one tile of a camera."""
    tx, ty = tile % tiles_x, tile // tiles_x
    x0, y0 = tx * cfg.tile_w, ty * cfg.tile_h
    return x0, y0, min(x0 + cfg.tile_w, cam["width"]), min(y0 + cfg.tile_h, cam["height"])


def render_tiles(pre: dict, cam: dict, cfg: Config, lists, tiles):
    """The tiled render of the listed tiles only: for each tile, (colour [3,h,w], T_final
    [h,w], n_contrib [h,w]) of its pixels, each pixel blending its tile's Gaussians in
    sorted-key order (the same blend as ``render_tiled``)."""
    keys, vals, ranges, tiles_x, tiles_y = lists
    bg = torch.as_tensor(np.asarray(cfg.bg, dtype=np.float64))
    out = {}
    with torch.no_grad():
        for tile in tiles:
            x0, y0, x1, y1 = tile_pixels(int(tile), tiles_x, cam, cfg)
            s, e = ranges[tile]
            g = torch.as_tensor(vals[s:e].astype(np.int64))
            pix = _pixel_centres(np.arange(x0, x1), np.arange(y0, y1))
            a = alpha_raw(pix, pre["mean2d"][g], pre["conic"][g], pre["opacity"][g])
            col, tf, lst = blend(a, pre["rgb"][g], bg)
            h, w = y1 - y0, x1 - x0
            out[int(tile)] = (col.numpy().T.reshape(3, h, w), tf.numpy().reshape(h, w),
                              lst.reshape(h, w))
    return out


def render_tiled(pre: dict, cam: dict, cfg: Config, lists=None, grad_out=None):
    """Tile by tile: each pixel blends its tile's Gaussians in sorted-key order.

    If ``grad_out`` ([3,H,W] dL/dimage) is given, the blend of each tile is differentiated
    on the spot and dL/d(mean2d, conic, opacity, rgb) are returned as a dict (so that large
    images never hold the whole blend graph)."""
    W, H = cam["width"], cam["height"]
    keys, vals, ranges, tiles_x, tiles_y = lists if lists is not None else tile_lists(pre, cam, cfg)
    bg = torch.as_tensor(np.asarray(cfg.bg, dtype=np.float64))
    img = np.zeros((3, H, W))
    t_fin = np.ones((H, W))
    last = np.zeros((H, W), dtype=np.int64)
    names = ("mean2d", "conic", "opacity", "rgb")
    if grad_out is not None:
        leaves = {k: pre[k].detach().clone().requires_grad_(True) for k in names}
        go = torch.as_tensor(np.asarray(grad_out, dtype=np.float64))
    else:
        leaves = {k: pre[k].detach() for k in names}
    for ty in range(tiles_y):
        for tx in range(tiles_x):
            tile = ty * tiles_x + tx
            x0, y0 = tx * cfg.tile_w, ty * cfg.tile_h
            x1, y1 = min(x0 + cfg.tile_w, W), min(y0 + cfg.tile_h, H)
            s, e = ranges[tile]
            g = torch.as_tensor(vals[s:e].astype(np.int64))
            pix = _pixel_centres(np.arange(x0, x1), np.arange(y0, y1))
            a = alpha_raw(pix, leaves["mean2d"][g], leaves["conic"][g], leaves["opacity"][g])
            col, tf, lst = blend(a, leaves["rgb"][g], bg)
            h, w = y1 - y0, x1 - x0
            img[:, y0:y1, x0:x1] = col.detach().numpy().T.reshape(3, h, w)
            t_fin[y0:y1, x0:x1] = tf.detach().numpy().reshape(h, w)
            last[y0:y1, x0:x1] = lst.reshape(h, w)
            if grad_out is not None and e > s:
                gt = go[:, y0:y1, x0:x1].reshape(3, -1).T
                (col * gt).sum().backward()
    if grad_out is None:
        return img, t_fin, last
    return img, t_fin, last, {k: leaves[k].grad for k in names}


def forward_backward(g: dict, sh_degree: int, s_min: float, cam: dict, cfg: Config,
                     grad_out: np.ndarray):
    """Render one camera and return (img, T_final, n_contrib, grads) where grads holds
    dL/d(means, quats, s_opt, opacity_logit, sh) for L = sum(grad_out * img)."""
    p = params(g, requires_grad=True)
    pre = preprocess(p, sh_degree, s_min, cam, cfg)
    img, tf, last, g2 = render_tiled(pre, cam, cfg, grad_out=grad_out)
    outs, gts = [], []
    for k in ("mean2d", "conic", "opacity", "rgb"):
        if g2[k] is not None:
            outs.append(pre[k])
            gts.append(g2[k])
    if outs:
        torch.autograd.backward(outs, gts)
    grads = {k: (p[k].grad.numpy() if p[k].grad is not None else np.zeros(p[k].shape))
             for k in p}
    return img, tf, last, grads


def render(g: dict, sh_degree: int, s_min: float, cam: dict, cfg: Config, tiled=True):
    p = params(g)
    with torch.no_grad():
        pre = preprocess(p, sh_degree, s_min, cam, cfg)
    if tiled:
        return render_tiled(pre, cam, cfg)
    img, tf = render_brute(pre, cam, cfg)
    return img.numpy(), tf.numpy(), None


def discrete_state(pre: dict, cam: dict, cfg: Config, lists=None) -> bytes:
    """Every discrete decision of the forward (culling, rectangles, colour clamp, Jacobian
    clamp, alpha clamp, skip and early stop per pixel), as bytes. Two parameter values
    with equal states lie on the same smooth piece of the forward."""
    t = pre["t"].detach().numpy()
    tz = np.where(t[:, 2] > cfg.z_near, t[:, 2], 1.0)
    lim_x = 1.3 * 0.5 * cam["width"] / cam["fx"]
    lim_y = 1.3 * 0.5 * cam["height"] / cam["fy"]
    parts = [pre["valid"].numpy().tobytes(), np.stack(pre["tile_rect"]).tobytes(),
             np.stack(pre["segments"]).tobytes(),
             (pre["rgb_raw"].detach().numpy() > 0).tobytes(),
             (np.abs(t[:, 0] / tz) > lim_x).tobytes(), (np.abs(t[:, 1] / tz) > lim_y).tobytes()]
    W, H = cam["width"], cam["height"]
    keys, vals, ranges, tiles_x, tiles_y = lists if lists is not None else tile_lists(pre, cam, cfg)
    parts.append(vals.tobytes())
    for ty in range(tiles_y):
        for tx in range(tiles_x):
            s, e = ranges[ty * tiles_x + tx]
            if e == s:
                continue
            g = torch.as_tensor(vals[s:e].astype(np.int64))
            x0, y0 = tx * cfg.tile_w, ty * cfg.tile_h
            pix = _pixel_centres(np.arange(x0, min(x0 + cfg.tile_w, W)),
                                 np.arange(y0, min(y0 + cfg.tile_h, H)))
            with torch.no_grad():
                a = alpha_raw(pix, pre["mean2d"][g], pre["conic"][g], pre["opacity"][g])
                clamped = a > ALPHA_MAX
                a = torch.clamp(a, max=ALPHA_MAX)
                kept = a >= ALPHA_MIN
                a = torch.where(kept, a, torch.zeros_like(a))
                live = torch.cumprod(1.0 - a, dim=1) >= T_MIN
            parts += [clamped.numpy().tobytes(), kept.numpy().tobytes(), live.numpy().tobytes()]
    return b"".join(parts)


def sampled_gradients(g: dict, sh_degree: int, s_min, cam: dict, cfg: Config,
                      grad_out: np.ndarray, sample: np.ndarray, lists=None, pre=None):
    """dL/d(parameters) of the Gaussians ``sample`` only, for L = sum(grad_out * image).

    A Gaussian enters only the tiles it is binned to, so its gradient is the sum over
    those tiles' pixels: each such tile is blended with the sampled Gaussian's 2D values as
    autograd leaves and every other Gaussian held constant, and the resulting 2D gradient is
    chained through that Gaussian's own preprocess. Exact (same definition as
    ``forward_backward``) at any scene size. Returns {name: array [len(sample), ...]}."""
    W, H = cam["width"], cam["height"]
    if pre is None:
        with torch.no_grad():
            pre = preprocess(params(g), sh_degree, s_min, cam, cfg)
    keys, vals, ranges, tiles_x, tiles_y = lists if lists is not None else tile_lists(pre, cam, cfg)
    bg = torch.as_tensor(np.asarray(cfg.bg, dtype=np.float64))
    go = torch.as_tensor(np.asarray(grad_out, dtype=np.float64))
    out = {k: [] for k in ("means", "quats", "s_opt", "opacity_logit", "sh")}
    seg_unit, seg_ty, seg_x0, seg_x1 = (np.asarray(a) for a in pre["segments"])
    names = ("mean2d", "conic", "opacity", "rgb")
    base = {k: pre[k].detach() for k in names}
    for j in np.asarray(sample, dtype=np.int64):
        one = {k: np.asarray(g[k])[j:j + 1] for k in ("means", "quats", "s_opt", "opacity_logit", "sh")}
        pj = params(one, requires_grad=True)
        smj = s_min if np.isscalar(s_min) else s_min[j:j + 1]
        prej = preprocess(pj, sh_degree, smj, cam, cfg)
        leaves = {k: prej[k] for k in names}
        total = None
        for q in np.nonzero(seg_unit == j)[0]:
            ty = int(seg_ty[q])
            for tx in range(int(seg_x0[q]), int(seg_x1[q]) + 1):
                tile = ty * tiles_x + tx
                s, e = ranges[tile]
                gi = vals[s:e].astype(np.int64)
                pos = np.nonzero(gi == j)[0]
                x0, y0 = tx * cfg.tile_w, ty * cfg.tile_h
                x1, y1 = min(x0 + cfg.tile_w, W), min(y0 + cfg.tile_h, H)
                pix = _pixel_centres(np.arange(x0, x1), np.arange(y0, y1))
                sel = torch.as_tensor(gi)
                cols = {}
                for k in names:
                    t = base[k][sel].clone()
                    mask = torch.zeros(len(gi), dtype=torch.bool)
                    mask[torch.as_tensor(pos)] = True
                    shape = (-1,) + (1,) * (t.dim() - 1)
                    cols[k] = torch.where(mask.view(shape), leaves[k].expand_as(t), t)
                a = alpha_raw(pix, cols["mean2d"], cols["conic"], cols["opacity"])
                col, _, _ = blend(a, cols["rgb"], bg)
                gt = go[:, y0:y1, x0:x1].reshape(3, -1).T
                term = (col * gt).sum()
                total = term if total is None else total + term
        if total is not None:
            total.backward()
        for k in out:
            gk = pj[k].grad
            out[k].append(np.zeros(pj[k].shape[1:]) if gk is None else gk.numpy()[0])
    return {k: np.stack(v) for k, v in out.items()}
