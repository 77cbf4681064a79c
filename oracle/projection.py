"""Projection of 3D Gaussians to the image plane, their extent and pixel/tile rectangles.

Sec. 3 (Eq. 2) only says that the Gaussians are "projected to 2D screenspace", giving the
2D mean mu' and covariance Sigma'. The readings used for what the paper leaves open:

* camera: world->camera [R_w | t_w] (3x4), pinhole u = f_x t_x/t_z + c_x,
  v = f_y t_y/t_z + c_y, OpenCV axes; a Gaussian with t_z <= z_near (0.2) is culled;
* local affine (EWA) approximation: Sigma' = J R_w Sigma R_w^T J^T + dilation * I, with
  J the Jacobian of the pinhole map at the view-space mean; for the Jacobian only, t_x/t_z
  and t_y/t_z are clamped to +-1.3 tan(half field of view) (off-screen guard);
  dilation 0.3 px^2 by default (low-pass filter), 0 allowed;
* pixel (i, j) samples the image at (i + 0.5, j + 0.5);
* extent, "opacity-aware" rule (rule 0): r = sqrt(2 ln(255 o) lambda_max(Sigma')),
  culled when o < 1/255. Every pixel where o * exp(-q/2) >= 1/255 lies within r of mu',
  so the tiled render equals the per-pixel render over all Gaussians. Rule 1:
  r = 3 sqrt(lambda_max);
* rectangle: covered pixel columns ceil(u - r - 0.5) .. floor(u + r - 0.5) clamped to
  the image (rows alike); tiles floor(col / tile_w), floor(row / tile_h);
* rule 2 (default), "ellipse rows": the support {d : d^T Sigma'^-1 d <= tau} with
  tau = 2 ln(255 o) (1 + 2^-10) (the same support, widened by a relative 2^-10 so that
  float32 rounding never drops a pixel). Its bounding box (half-widths
  rx = sqrt(tau Sigma'_xx), ry = sqrt(tau Sigma'_yy)) gives the pixel and tile rectangle;
  in each tile row of that rectangle only the tile columns whose pixel centres meet the
  ellipse are listed. Row dy of the ellipse is x in u + m dy +- h sqrt(ry^2 - dy^2),
  m = Sigma'_xy / Sigma'_yy, h = sqrt(det Sigma') / Sigma'_yy (complete the square in x);
  over the band of pixel-centre rows of a tile row, the rightmost point is at
  dy = clamp(m ry^2 / rx) (the ellipse's own rightmost point, dy = m ry^2 / rx, clamped to
  the band; the right boundary is concave in dy) and the leftmost at clamp(-m ry^2 / rx).
  The covered columns of the row are ceil(x_left - 0.5) .. floor(x_right - 0.5) within the
  rectangle. The tiled render still equals the per-pixel render, with fewer (tile,
  Gaussian) pairs than rule 0.
"""
from __future__ import annotations

import math

import numpy as np
import torch

ALPHA_MIN = 1.0 / 255.0


def camera_tensors(cam: dict):
    vm = torch.as_tensor(np.asarray(cam["viewmat"], dtype=np.float64))
    return vm[:, :3], vm[:, 3], torch.as_tensor(np.asarray(cam["cam_pos"], dtype=np.float64))


def view_space(means: torch.Tensor, cam: dict) -> torch.Tensor:
    rw, tw, _ = camera_tensors(cam)
    return means @ rw.T + tw[None, :]


def project(means: torch.Tensor, cov3d: torch.Tensor, cam: dict, dilation: float = 0.3,
            z_near: float = 0.2):
    """Returns (t [N,3] view space, mean2d [N,2], cov2d [N,2,2], in_front [N] bool)."""
    rw, _, _ = camera_tensors(cam)
    t = view_space(means, cam)
    tz = t[:, 2]
    in_front = (tz > z_near).detach()
    tz_s = torch.where(in_front, tz, torch.ones_like(tz))
    fx, fy, cx, cy = (float(cam[k]) for k in ("fx", "fy", "cx", "cy"))
    lim_x = 1.3 * (0.5 * cam["width"] / fx)
    lim_y = 1.3 * (0.5 * cam["height"] / fy)
    kx = torch.clamp(t[:, 0] / tz_s, -lim_x, lim_x)
    ky = torch.clamp(t[:, 1] / tz_s, -lim_y, lim_y)
    zero = torch.zeros_like(tz_s)
    jac = torch.stack([
        fx / tz_s, zero, -fx * kx / tz_s,
        zero, fy / tz_s, -fy * ky / tz_s,
    ], dim=1).reshape(-1, 2, 3)
    m = jac @ rw[None, :, :]
    cov2d = m @ cov3d @ m.transpose(1, 2)
    cov2d = cov2d + dilation * torch.eye(2, dtype=cov2d.dtype)[None]
    mean2d = torch.stack([fx * t[:, 0] / tz_s + cx, fy * t[:, 1] / tz_s + cy], dim=1)
    return t, mean2d, cov2d, in_front


def conic(cov2d: torch.Tensor):
    """Inverse of the 2x2 covariance as (a, b, c) with q = a dx^2 + 2 b dx dy + c dy^2.
    Returns (conic [N,3], det [N])."""
    a, b, c = cov2d[:, 0, 0], cov2d[:, 0, 1], cov2d[:, 1, 1]
    det = a * c - b * b
    det_s = torch.where(det > 0, det, torch.ones_like(det))
    return torch.stack([c / det_s, -b / det_s, a / det_s], dim=1), det


def lambda_max(cov2d: torch.Tensor) -> torch.Tensor:
    a, b, c = cov2d[:, 0, 0], cov2d[:, 0, 1], cov2d[:, 1, 1]
    h = 0.5 * (a + c)
    return h + torch.sqrt(torch.clamp(0.25 * (a - c) ** 2 + b * b, min=0.0))


def radius(cov2d: torch.Tensor, opacity: torch.Tensor, rule: int = 0):
    """Extent radius (pixels) and validity; no gradient flows through it."""
    with torch.no_grad():
        lm = lambda_max(cov2d)
        if rule == 0:
            ok = opacity >= ALPHA_MIN
            arg = torch.where(ok, 2.0 * torch.log(255.0 * opacity), torch.zeros_like(opacity))
            r = torch.sqrt(torch.clamp(arg * lm, min=0.0))
        else:
            ok = torch.ones_like(opacity, dtype=torch.bool)
            r = 3.0 * torch.sqrt(lm)
    return r, ok


def pixel_rect(u: np.ndarray, v: np.ndarray, r: np.ndarray, width: int, height: int):
    """Inclusive covered pixel ranges (x0, x1, y0, y1), FP64; empty when x0 > x1 or y0 > y1."""
    u, v, r = (np.asarray(a, dtype=np.float64) for a in (u, v, r))
    big = 1e9
    x0 = np.clip(np.ceil(u - r - 0.5), -1, big)
    x1 = np.clip(np.floor(u + r - 0.5), -big, width)
    y0 = np.clip(np.ceil(v - r - 0.5), -1, big)
    y1 = np.clip(np.floor(v + r - 0.5), -big, height)
    x0 = np.maximum(x0, 0)
    y0 = np.maximum(y0, 0)
    x1 = np.minimum(x1, width - 1)
    y1 = np.minimum(y1, height - 1)
    return (x0.astype(np.int64), x1.astype(np.int64), y0.astype(np.int64), y1.astype(np.int64))


def pixel_rect_f32(u: np.ndarray, v: np.ndarray, r: np.ndarray, width: int, height: int):
    """The same rectangle with every operation rounded to FP32, as a float32 kernel takes
    the decision: (u - r) - 0.5 and (u + r) - 0.5, each step rounded to nearest."""
    u, v, r = (np.asarray(a, dtype=np.float32) for a in (u, v, r))
    h = np.float32(0.5)
    with np.errstate(invalid="ignore", over="ignore"):
        x0 = np.ceil((u - r) - h)
        x1 = np.floor((u + r) - h)
        y0 = np.ceil((v - r) - h)
        y1 = np.floor((v + r) - h)
    x0 = np.clip(np.nan_to_num(x0, nan=1e9), 0, 1e9)
    y0 = np.clip(np.nan_to_num(y0, nan=1e9), 0, 1e9)
    x1 = np.clip(np.nan_to_num(x1, nan=-1e9), -1e9, width - 1)
    y1 = np.clip(np.nan_to_num(y1, nan=-1e9), -1e9, height - 1)
    return (x0.astype(np.int64), x1.astype(np.int64), y0.astype(np.int64), y1.astype(np.int64))


def tile_rect(px, tile_w: int, tile_h: int, valid: np.ndarray):
    """Tile ranges (tx0, tx1, ty0, ty1) from pixel ranges; tiles_touched = 0 if empty or
    invalid."""
    x0, x1, y0, y1 = px
    empty = (x0 > x1) | (y0 > y1) | ~np.asarray(valid, dtype=bool)
    tx0 = np.where(empty, 0, x0 // tile_w)
    tx1 = np.where(empty, -1, x1 // tile_w)
    ty0 = np.where(empty, 0, y0 // tile_h)
    ty1 = np.where(empty, -1, y1 // tile_h)
    touched = np.where(empty, 0, (tx1 - tx0 + 1) * (ty1 - ty0 + 1))
    return tx0, tx1, ty0, ty1, touched.astype(np.int64)


EXTENT_MARGIN = 2.0 ** -10


def ellipse_extent(cov2d: torch.Tensor, opacity: torch.Tensor):
    """Rule 2: (m, h, rx, ry) [N,4] of the support ellipse and its validity (o >= 1/255 and
    Sigma' positive definite). FP64, no gradient flows through it."""
    with torch.no_grad():
        a, b, c = cov2d[:, 0, 0], cov2d[:, 0, 1], cov2d[:, 1, 1]
        det = a * c - b * b
        ok = (opacity >= ALPHA_MIN) & (det > 0) & (c > 0)
        tau = torch.where(ok, 2.0 * torch.log(255.0 * opacity) * (1.0 + EXTENT_MARGIN),
                          torch.zeros_like(opacity))
        c_s = torch.where(c > 0, c, torch.ones_like(c))
        m = b / c_s
        h = torch.sqrt(torch.clamp(det, min=0.0)) / c_s
        rx = torch.sqrt(torch.clamp(tau * a, min=0.0))
        ry = torch.sqrt(torch.clamp(tau * c, min=0.0))
        ext = torch.stack([m, h, rx, ry], dim=1)
        return torch.where(ok[:, None], ext, torch.zeros_like(ext)), ok


def pixel_rect_xy(u, v, rx, ry, width: int, height: int, dtype=np.float64):
    """Rectangle of pixel columns ceil((u - rx) - 0.5) .. floor((u + rx) - 0.5) and rows
    alike with ry, every operation rounded to ``dtype``; clamped to the image."""
    u, v, rx, ry = (np.asarray(a, dtype=dtype) for a in (u, v, rx, ry))
    h = dtype(0.5)
    with np.errstate(invalid="ignore", over="ignore"):
        x0 = np.ceil((u - rx) - h)
        x1 = np.floor((u + rx) - h)
        y0 = np.ceil((v - ry) - h)
        y1 = np.floor((v + ry) - h)
    x0 = np.clip(np.nan_to_num(x0, nan=1e9), 0, 1e9)
    y0 = np.clip(np.nan_to_num(y0, nan=1e9), 0, 1e9)
    x1 = np.clip(np.nan_to_num(x1, nan=-1e9), -1e9, width - 1)
    y1 = np.clip(np.nan_to_num(y1, nan=-1e9), -1e9, height - 1)
    return (x0.astype(np.int64), x1.astype(np.int64), y0.astype(np.int64), y1.astype(np.int64))


def rect_segments(tile_rect_, touched):
    """Rules 0 and 1: every tile row of a unit's rectangle is one segment of full width.
    Returns (unit, ty, cx0, cx1) int64 arrays in emission order (unit, then row)."""
    tx0, tx1, ty0, ty1 = (np.asarray(a, dtype=np.int64) for a in tile_rect_)
    rows = np.where(np.asarray(touched) > 0, ty1 - ty0 + 1, 0)
    unit = np.repeat(np.arange(rows.size, dtype=np.int64), rows)
    start = np.cumsum(rows) - rows
    ty = ty0[unit] + (np.arange(unit.size, dtype=np.int64) - start[unit])
    return unit, ty, tx0[unit], tx1[unit]


def ellipse_segments(u, v, ext, px, tile_w: int, tile_h: int, valid, dtype=np.float64):
    """Rule 2: per unit and tile row of its rectangle ``px`` (pixel ranges), the tile
    columns [cx0, cx1] whose pixel centres meet the ellipse ``ext`` = (m, h, rx, ry), with
    every operation rounded to ``dtype`` (float64: the rule itself; float32: the decision a
    float32 kernel takes with the same operations in the same order). Rows with no column
    are left out. Returns ((unit, ty, cx0, cx1) in emission order, tiles per unit)."""
    dt = dtype
    u, v = np.asarray(u, dtype=dt), np.asarray(v, dtype=dt)
    ext = np.asarray(ext, dtype=dt)
    m, hh, rx, ry = ext[:, 0], ext[:, 1], ext[:, 2], ext[:, 3]
    x0, x1, y0, y1 = px
    n = u.shape[0]
    ok = np.asarray(valid, dtype=bool) & (x0 <= x1) & (y0 <= y1)
    ty0 = np.where(ok, y0 // tile_h, 0)
    ty1 = np.where(ok, y1 // tile_h, -1)
    with np.errstate(invalid="ignore", over="ignore", divide="ignore"):
        ry2 = ry * ry
        dyx = np.where(rx > 0, (m * ry2) / np.where(rx > 0, rx, dt(1)), dt(0))
    segs = []
    nrows = ty1 - ty0 + 1
    for k in range(int(nrows.max(initial=0))):
        sel = np.nonzero(nrows > k)[0]
        ty = ty0[sel] + k
        jy0 = np.maximum(ty * tile_h, y0[sel])
        jy1 = np.minimum(ty * tile_h + tile_h - 1, y1[sel])
        with np.errstate(invalid="ignore", over="ignore"):
            dy0 = (jy0.astype(dt) + dt(0.5)) - v[sel]
            dy1 = (jy1.astype(dt) + dt(0.5)) - v[sel]
            dr = np.fmin(np.fmax(dyx[sel], dy0), dy1)
            dl = np.fmin(np.fmax(-dyx[sel], dy0), dy1)
            wr = hh[sel] * np.sqrt(np.fmax(ry2[sel] - dr * dr, dt(0)))
            wl = hh[sel] * np.sqrt(np.fmax(ry2[sel] - dl * dl, dt(0)))
            xr = (u[sel] + m[sel] * dr) + wr
            xl = (u[sel] + m[sel] * dl) - wl
            c0 = np.fmax(np.ceil(xl - dt(0.5)), x0[sel].astype(dt))
            c1 = np.fmin(np.floor(xr - dt(0.5)), x1[sel].astype(dt))
        keep = c0 <= c1
        s = sel[keep]
        segs.append((s, ty[keep], c0[keep].astype(np.int64) // tile_w,
                     c1[keep].astype(np.int64) // tile_w))
    if segs:
        unit = np.concatenate([q[0] for q in segs])
        ty = np.concatenate([q[1] for q in segs])
        cx0 = np.concatenate([q[2] for q in segs])
        cx1 = np.concatenate([q[3] for q in segs])
        order = np.lexsort((ty, unit))
        unit, ty, cx0, cx1 = unit[order], ty[order], cx0[order], cx1[order]
    else:
        unit = ty = cx0 = cx1 = np.zeros(0, dtype=np.int64)
    touched = np.bincount(unit, weights=cx1 - cx0 + 1, minlength=n).astype(np.int64)
    return (unit.astype(np.int64), ty.astype(np.int64), cx0, cx1), touched


def focal_from_hfov(width: int, hfov_deg: float) -> float:
    return width / (2.0 * math.tan(math.radians(hfov_deg) / 2.0))
