"""Overlap pruning (Sec. 4.3), FP64 -- TEST INFRASTRUCTURE ONLY.

A Gaussian is removed when the average distance to its three nearest neighbours,
d_avg(i) = (d_i1 + d_i2 + d_i3) / 3, falls below d_OP = s_min / 2 of the level being
trained (Sec. 4.3; run every 1,000 iterations at every level but the last, Sec. 5.1.4).

Readings where the paper is silent: distances are Euclidean distances between the
Gaussians' means; the neighbours are the other Gaussians of the same level (a Gaussian is
not its own neighbour; two Gaussians at the same mean are neighbours at distance 0); a
Gaussian with fewer than three other Gaussians in its level is kept.

``knn3`` is the definition written out: the full distance matrix, block by block, and the
three smallest entries of each row other than the diagonal.
"""
from __future__ import annotations

import math

import numpy as np


def knn3(means: np.ndarray, block: int = 256):
    """(d [N,3] sorted ascending, idx [N,3]) of the three nearest other means, FP64. Rows of a
    level with fewer than four Gaussians are padded with inf / -1."""
    m = np.asarray(means, dtype=np.float64)
    n = m.shape[0]
    d_out = np.full((n, 3), np.inf)
    i_out = np.full((n, 3), -1, dtype=np.int64)
    k = min(3, n - 1)
    if k <= 0:
        return d_out, i_out
    for a in range(0, n, block):
        b = min(n, a + block)
        # squared distances from explicit coordinate differences
        d2 = np.zeros((b - a, n))
        for c in range(3):
            t = m[a:b, None, c] - m[None, :, c]
            d2 += t * t
        d2[np.arange(b - a), np.arange(a, b)] = np.inf        # not its own neighbour
        part = np.argpartition(d2, k - 1, axis=1)[:, :k]
        dd = np.take_along_axis(d2, part, axis=1)
        order = np.argsort(dd, axis=1, kind="stable")
        i_out[a:b, :k] = np.take_along_axis(part, order, axis=1)
        d_out[a:b, :k] = np.sqrt(np.take_along_axis(dd, order, axis=1))
    return d_out, i_out


def d_avg(means: np.ndarray) -> np.ndarray:
    """The average distance of each Gaussian to its three nearest neighbours (inf with fewer
    than three other Gaussians)."""
    d, _ = knn3(means)
    return d.mean(axis=1)


def keep_mask(means: np.ndarray, s_min: float) -> np.ndarray:
    """True for the Gaussians overlap pruning keeps: d_avg >= d_OP = s_min / 2."""
    return ~(d_avg(means) < 0.5 * s_min)


def d_avg_loop(means, i: int) -> float:
    """d_avg of one Gaussian by a plain loop over all others (small inputs, for checks)."""
    m = [tuple(float(v) for v in row) for row in np.asarray(means)]
    ds = sorted(math.dist(m[i], m[j]) for j in range(len(m)) if j != i)
    return sum(ds[:3]) / 3.0 if len(ds) >= 3 else math.inf
