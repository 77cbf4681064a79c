"""Density control of a level (the Densification and Pruning steps of Algorithm 1, with the
backbone's rules kept by the paper, Sec. 5.1.4) -- TEST INFRASTRUCTURE ONLY.

Statistics, every iteration of the densification window: for every Gaussian that touches a
tile of the view, accum += || dL/d(mean2d) || with the 2D mean in normalised device
coordinates (the pixel-space gradient times (W/2, H/2)), and denom += 1.

The step, every densification interval (reading of the backbone's rules; the paper changes
only the intervals and windows, and drops the removal of large Gaussians):
* g = accum / denom (0 where denom = 0); s = exp(s_opt) + s_min (Eq. 4), opacity =
  sigmoid(logit);
* clone: g >= tau and max(s) <= max_clone_scale (percent_dense x scene extent): a copy of
  the Gaussian is appended;
* split: g >= tau and max(s) > max_clone_scale: two children replace it, with means
  mu + R (s * eps) for two standard-normal draws eps (inputs, not drawn here), the learnable
  part of the scale divided by 1.6 (exp(s_opt') = exp(s_opt) / 1.6, so s' >= s_min still),
  every other parameter copied;
* prune: opacity < min_opacity removes the Gaussian, its clone and its children;
* order of the new set: the Gaussians kept in place (neither split nor pruned) by index, then
  the clones by index, then the children by index (two per split Gaussian);
* Adam moments follow the parameters: kept in place for the survivors, zero for clones and
  children.
The integer decisions are taken in float32 (the kernel's precision; the paper fixes none).
"""
from __future__ import annotations

import numpy as np

from . import gaussians as G

SPLIT_SCALE = 1.6
FIELDS = ("means", "quats", "s_opt", "opacity_logit", "sh")


def stats_update(accum, denom, grad_mean2d_px, visible, width: int, height: int):
    """One iteration's statistics from the pixel-space 2D mean gradient [N, 2] (FP64)."""
    g = np.asarray(grad_mean2d_px, dtype=np.float64) * np.array([0.5 * width, 0.5 * height])
    norm = np.sqrt((g * g).sum(axis=1))
    accum = np.asarray(accum, dtype=np.float64) + np.where(visible, norm, 0.0)
    denom = np.asarray(denom, dtype=np.float64) + np.where(visible, 1.0, 0.0)
    return accum, denom


def decisions(g: dict, s_min: float, accum, denom, tau: float, max_clone_scale: float,
              min_opacity: float):
    """(survive, clone, split) boolean masks, decided in float32."""
    acc = np.asarray(accum, dtype=np.float32)
    den = np.asarray(denom, dtype=np.float32)
    with np.errstate(divide="ignore", invalid="ignore"):
        avg = np.where(den > 0, acc / np.where(den > 0, den, np.float32(1)), np.float32(0))
    s = np.exp(np.asarray(g["s_opt"], dtype=np.float32)) + np.float32(s_min)
    big = s.max(axis=1) > np.float32(max_clone_scale)
    op = np.float32(1) / (np.float32(1) + np.exp(-np.asarray(g["opacity_logit"], dtype=np.float32)))
    low = op < np.float32(min_opacity)
    dens = avg >= np.float32(tau)
    clone = dens & ~big & ~low
    split = dens & big & ~low
    survive = ~(dens & big) & ~low
    return survive, clone, split


def densify(g: dict, s_min: float, accum, denom, normals, tau: float, max_clone_scale: float,
            min_opacity: float, m=None, v=None):
    """The new set (dict of float64 arrays) and, with m, v given, its Adam moments.
    normals: [2N, 3] standard-normal draws, rows 2i and 2i + 1 for Gaussian i's children."""
    survive, clone, split = decisions(g, s_min, accum, denom, tau, max_clone_scale, min_opacity)
    p = {k: np.asarray(g[k], dtype=np.float64) for k in FIELDS}
    idx_s, idx_c, idx_p = np.nonzero(survive)[0], np.nonzero(clone)[0], np.nonzero(split)[0]
    out = {k: [p[k][idx_s], p[k][idx_c]] for k in FIELDS}
    # children: two per split Gaussian, in index order
    child = np.repeat(idx_p, 2)
    eps = np.asarray(normals, dtype=np.float64).reshape(-1, 2, 3)[idx_p].reshape(-1, 3)
    import torch
    R = G.rotation(torch.as_tensor(p["quats"][child])).numpy()
    s = np.exp(p["s_opt"][child]) + s_min
    offs = np.einsum("nij,nj->ni", R, s * eps)
    new = {k: p[k][child].copy() for k in FIELDS}
    new["means"] = p["means"][child] + offs
    new["s_opt"] = p["s_opt"][child] - np.log(SPLIT_SCALE)
    for k in FIELDS:
        out[k].append(new[k])
        out[k] = np.concatenate(out[k])
    if m is None:
        return out
    mom = []
    for st in (m, v):
        d = {}
        for k in FIELDS:
            a = np.asarray(st[k], dtype=np.float64)
            z = np.zeros((idx_c.size + 2 * idx_p.size,) + a.shape[1:])
            d[k] = np.concatenate([a[idx_s], z])
        mom.append(d)
    return out, mom[0], mom[1]
