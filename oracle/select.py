"""Level-selective rendering set: Eq. 6 and Eq. 7 (Sec. 5.2).

* Eq. 7: d_proj^(l) = s_min^(l) * f / gamma (gamma = 1 by default, Sec. 5.1.4), with
  d_proj^(L_end) = 0 and d_proj^(L_start - 1) = infinity.
* Eq. 6: G_sel = union over l in [L_start, L_end] of the Gaussians G of level l with
  d_proj^(l-1) > d_G >= d_proj^(l).
* d_G is the Euclidean distance from the Gaussian mean to the reference position: the
  current camera centre (per-view set) or the mean of the training cameras
  (predetermined set).

Levels are passed coarse to fine (index 0 = L_start). ``thresholds[k]`` is d_proj of the
level at index k, k = 0..n-2; the last level's threshold is 0 and the level before the
first has infinity. Selection entries are (level_index << 28) | gaussian_index, ordered by
level then index.

The comparison d_G >= d_proj decides an integer (set membership). The paper fixes no
precision, so it is taken in FP32 like the kernel: dx, dy, dz, their squares and the sum
((dx^2 + dy^2) + dz^2) are each rounded to FP32 and d_G = sqrt of that, correctly rounded.
``select_exact`` takes the same decision in FP64 for comparison.
"""
from __future__ import annotations

import math

import numpy as np

LEVEL_SHIFT = 28


def d_proj(s_min: list, focal: float, gamma: float = 1.0) -> list[float]:
    """Eq. 7 for levels given coarse to fine; the finest level gets 0 (its own d_proj is
    replaced by the endpoint rule) and only the first n-1 entries are returned."""
    return [s * focal / gamma for s in s_min[:-1]]


def band(k: int, thresholds) -> tuple[float, float]:
    """[lo, hi) distance band of level index k (Eq. 6 with the endpoint rule of Eq. 7)."""
    n = len(thresholds) + 1
    hi = math.inf if k == 0 else thresholds[k - 1]
    lo = 0.0 if k == n - 1 else thresholds[k]
    return lo, hi


def distance_f32(means: np.ndarray, origin) -> np.ndarray:
    m = np.asarray(means, dtype=np.float32)
    o = np.asarray(origin, dtype=np.float32)
    dx = m[:, 0] - o[0]
    dy = m[:, 1] - o[1]
    dz = m[:, 2] - o[2]
    return np.sqrt((dx * dx + dy * dy) + dz * dz)


def select(level_means: list, origin, thresholds) -> np.ndarray:
    """Eq. 6, decision in FP32 with FP32 thresholds; returns uint32 entries."""
    th = [np.float32(t) for t in thresholds]
    out = []
    for k, m in enumerate(level_means):
        lo, hi = band(k, th)
        d = distance_f32(m, origin)
        keep = (d >= np.float32(lo)) & (d < np.float32(hi))
        idx = np.nonzero(keep)[0].astype(np.uint64)
        out.append((np.uint64(k) << np.uint64(LEVEL_SHIFT)) | idx)
    return np.concatenate(out).astype(np.uint32) if out else np.zeros(0, np.uint32)


def select_exact(level_means: list, origin, thresholds) -> np.ndarray:
    """Eq. 6 with FP64 distances and thresholds (for counting rounding-boundary cases)."""
    out = []
    o = np.asarray(origin, dtype=np.float64)
    for k, m in enumerate(level_means):
        lo, hi = band(k, thresholds)
        d = np.linalg.norm(np.asarray(m, dtype=np.float64) - o[None, :], axis=1)
        idx = np.nonzero((d >= lo) & (d < hi))[0].astype(np.uint64)
        out.append((np.uint64(k) << np.uint64(LEVEL_SHIFT)) | idx)
    return np.concatenate(out).astype(np.uint32) if out else np.zeros(0, np.uint32)


def select_loop(level_means: list, origin, thresholds) -> list[tuple[int, int]]:
    """Brute-force Python loop over every Gaussian of every level (small inputs only)."""
    res = []
    for k, m in enumerate(level_means):
        lo, hi = band(k, thresholds)
        for i, p in enumerate(np.asarray(m, dtype=np.float64)):
            d = math.sqrt(sum((float(p[j]) - float(origin[j])) ** 2 for j in range(3)))
            if hi > d >= lo:
                res.append((k, i))
    return res
