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
* extent, "opacity-aware" rule (default): r = sqrt(2 ln(255 o) lambda_max(Sigma')),
  culled when o < 1/255. Every pixel where o * exp(-q/2) >= 1/255 lies within r of mu',
  so the tiled render equals the per-pixel render over all Gaussians. Alternative rule:
  r = 3 sqrt(lambda_max);
* rectangle: covered pixel columns ceil(u - r - 0.5) .. floor(u + r - 0.5) clamped to
  the image (rows alike); tiles floor(col / tile_w), floor(row / tile_h).
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


def focal_from_hfov(width: int, hfov_deg: float) -> float:
    return width / (2.0 * math.tan(math.radians(hfov_deg) / 2.0))
