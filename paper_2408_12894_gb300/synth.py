"""Seeded synthetic inputs shaped like the FLoD workloads.

This module only draws random numbers and builds look-at camera poses. It holds none of
the rendering arithmetic, so the CUDA path and the FP64 oracle can both consume what it
returns without sharing any of the method's code.

Recipe (all draws from ``numpy.random.Generator(PCG64(seed))``):

* cluster centres: K points uniform in the ball of radius R;
* Gaussian means: a uniformly chosen centre plus N(0, (0.3 R)^2 I); a draw with
  ||mu|| > R is redrawn;
* s_opt ~ N(-4, 0.5) per axis (the learnable scale parameter of Eq. 4; with s_min = 0 it
  is the 3DGS log-scale);
* rotations: N(0, I_4) normalised to unit length, i.e. uniform on S^3, stored (w, x, y, z);
* opacity logits ~ N(0, 1.5) (opacity = sigmoid(logit));
* colour: the DC coefficient is (u - 0.5) / Y_00 with u ~ U[0, 1] per channel and Y_00 the
  constant zeroth spherical harmonic 1/(2 sqrt(pi)), so a degree-0 render shows u; the
  higher coefficients are N(0, 0.05);
* cameras: pinhole, square pixels, horizontal field of view 60 degrees
  (f = W / (2 tan 30 deg)), principal point at (W/2, H/2), OpenCV axes (x right, y down,
  z forward), world up +y.

Layouts (float32, C-contiguous): means [N,3], quats [N,4], s_opt [N,3], opacity_logit [N],
sh [N,(deg+1)^2,3]. A camera is a dict with viewmat [3,4] (world -> camera, row-major),
fx, fy, cx, cy, width, height and cam_pos [3].
"""
from __future__ import annotations

import math

import numpy as np

Y00 = 0.5 / math.sqrt(math.pi)

#: per-level Gaussian counts of the 5-level scene (levels 1..5)
LEVEL_COUNTS = (20_000, 80_000, 300_000, 1_000_000, 3_000_000)
#: minimum 3D scale of each level of the 5-level benchmark scene (halving from 0.5)
LEVEL_SMIN = (0.5, 0.25, 0.125, 0.0625, 0.03125)
#: camera-distance thresholds of the selective-rendering workload (near -> finest level)
SELECTIVE_THRESHOLDS = (10.0, 25.0, 50.0, 100.0)
#: resolutions mixed in the batched workload
BATCH_RESOLUTIONS = ((640, 480), (1280, 720), (1920, 1080), (3840, 2160))


def _rng(seed: int) -> np.random.Generator:
    return np.random.Generator(np.random.PCG64(seed))


def cluster_centres(rng: np.random.Generator, k: int, radius: float) -> np.ndarray:
    d = rng.standard_normal((k, 3))
    d /= np.linalg.norm(d, axis=1, keepdims=True)
    r = radius * rng.random(k) ** (1.0 / 3.0)
    return d * r[:, None]


def cluster_points(rng: np.random.Generator, centres: np.ndarray, n: int, radius: float,
                   sigma_rel: float = 0.3) -> np.ndarray:
    out = np.empty((n, 3))
    todo = np.arange(n)
    while todo.size:
        c = centres[rng.integers(0, len(centres), todo.size)]
        p = c + rng.standard_normal((todo.size, 3)) * (sigma_rel * radius)
        ok = np.linalg.norm(p, axis=1) <= radius
        out[todo[ok]] = p[ok]
        todo = todo[~ok]
    return out


def gaussian_attributes(rng: np.random.Generator, means: np.ndarray, sh_degree: int,
                        s_mean: float = -4.0, s_std: float = 0.5, logit_std: float = 1.5,
                        sh_std: float = 0.05) -> dict:
    n = means.shape[0]
    k = (sh_degree + 1) ** 2
    q = rng.standard_normal((n, 4))
    q /= np.linalg.norm(q, axis=1, keepdims=True)
    sh = np.zeros((n, k, 3))
    sh[:, 0, :] = (rng.random((n, 3)) - 0.5) / Y00
    if k > 1:
        sh[:, 1:, :] = rng.standard_normal((n, k - 1, 3)) * sh_std
    return {
        "means": np.ascontiguousarray(means, dtype=np.float32),
        "quats": np.ascontiguousarray(q, dtype=np.float32),
        "s_opt": np.ascontiguousarray(s_mean + s_std * rng.standard_normal((n, 3)),
                                      dtype=np.float32),
        "opacity_logit": np.ascontiguousarray(logit_std * rng.standard_normal(n),
                                              dtype=np.float32),
        "sh": np.ascontiguousarray(sh, dtype=np.float32),
        "sh_degree": int(sh_degree),
    }


def gaussian_set(seed: int, n: int, k: int = 8, radius: float = 1.0, sh_degree: int = 0,
                 **kw) -> dict:
    """One Gaussian set drawn from a K-cluster distribution inside a ball of ``radius``."""
    rng = _rng(seed)
    centres = cluster_centres(rng, k, radius)
    means = cluster_points(rng, centres, n, radius)
    return gaussian_attributes(rng, means, sh_degree, **kw)


def look_at(eye, target=(0.0, 0.0, 0.0), up=(0.0, 1.0, 0.0)) -> np.ndarray:
    """World-to-camera [R | t] (3x4) with OpenCV axes: x right, y down, z forward."""
    eye = np.asarray(eye, dtype=np.float64)
    z = np.asarray(target, dtype=np.float64) - eye
    z /= np.linalg.norm(z)
    up = np.asarray(up, dtype=np.float64)
    x = np.cross(z, up)
    if np.linalg.norm(x) < 1e-6:                # looking along the up axis
        x = np.cross(z, np.array([0.0, 0.0, 1.0]))
    x /= np.linalg.norm(x)
    y = np.cross(z, x)
    rot = np.stack([x, y, z])
    return np.concatenate([rot, (-rot @ eye)[:, None]], axis=1)


def camera(eye, width: int, height: int, hfov_deg: float = 60.0, target=(0.0, 0.0, 0.0)) -> dict:
    f = width / (2.0 * math.tan(math.radians(hfov_deg) / 2.0))
    return {
        "viewmat": look_at(eye, target).astype(np.float32),
        "fx": float(np.float32(f)), "fy": float(np.float32(f)),
        "cx": width / 2.0, "cy": height / 2.0,
        "width": int(width), "height": int(height),
        "cam_pos": np.asarray(eye, dtype=np.float32),
    }


# ---------------------------------------------------------------------------------------
# workloads
# ---------------------------------------------------------------------------------------

def scene_single_forward(seed: int = 0, n: int = 10_000):
    """Plain single-level forward render: 10k Gaussians, 8 clusters in the unit ball, SH 0,
    one 128x128 camera at distance 3."""
    g = gaussian_set(seed, n, k=8, radius=1.0, sh_degree=0)
    cam = camera((0.0, 0.0, -3.0), 128, 128)
    return g, [cam]


def scene_multiview_training(seed: int = 1, n: int = 500_000, width: int = 1280,
                             height: int = 720, n_cams: int = 8):
    """Single-level forward+backward: 500k Gaussians, 64 clusters of radius 5, SH 3, eight
    1280x720 cameras on a ring of radius 15 in the xz-plane."""
    g = gaussian_set(seed, n, k=64, radius=5.0, sh_degree=3)
    cams = []
    for i in range(n_cams):
        a = 2.0 * math.pi * i / n_cams
        cams.append(camera((15.0 * math.cos(a), 0.0, 15.0 * math.sin(a)), width, height))
    return g, cams


def upstream_gradient(seed: int, cams, std: float = 1e-3) -> np.ndarray:
    """dL/dimage ~ N(0, std^2) for every pixel and channel of every camera, flattened in the
    planar per-camera layout [sum_c 3*H_c*W_c]."""
    rng = _rng(seed)
    total = sum(3 * c["width"] * c["height"] for c in cams)
    return (std * rng.standard_normal(total)).astype(np.float32)


def level_scene(seed: int = 20, counts=LEVEL_COUNTS, k: int = 64, radius: float = 20.0,
                sh_degree: int = 3):
    """The multi-level scene: level l+1 holds level l's Gaussians (carried, s_opt still the
    level-l value, to be re-parameterised by AdjustScale) followed by fresh draws up to
    counts[l]. Returns a list of (attribute dict, n_carried)."""
    rng = _rng(seed)
    centres = cluster_centres(rng, k, radius)
    levels = []
    prev = None
    for li, n in enumerate(counts):
        lrng = _rng(seed + 1 + li)
        n_new = n - (0 if prev is None else prev["means"].shape[0])
        fresh = gaussian_attributes(lrng, cluster_points(lrng, centres, n_new, radius), sh_degree)
        if prev is None:
            cur = fresh
            carried = 0
        else:
            carried = prev["means"].shape[0]
            cur = {key: (np.concatenate([prev[key], fresh[key]]) if key != "sh_degree"
                         else sh_degree) for key in fresh}
        levels.append((cur, carried))
        prev = cur
    return levels


def level_camera(width: int = 1920, height: int = 1080, distance: float = 40.0):
    return camera((0.0, 0.0, -distance), width, height)


def stretch_levels(levels, factor: float = 5.0):
    """The selective-rendering scene: the level scene with positions scaled by ``factor``."""
    out = []
    for g, carried in levels:
        h = dict(g)
        h["means"] = (g["means"] * np.float32(factor)).astype(np.float32)
        out.append((h, carried))
    return out


def camera_path(seed: int = 3, n_frames: int = 32, width: int = 1920, height: int = 1080,
                radius: float = 30.0, height_y: float = 2.0):
    """A seeded camera path: a quarter circle of ``radius`` at height ``height_y`` with
    N(0,1) positional jitter, looking at the origin."""
    rng = _rng(seed)
    cams = []
    for i in range(n_frames):
        a = 0.5 * math.pi * i / max(n_frames - 1, 1)
        eye = np.array([radius * math.cos(a), height_y, radius * math.sin(a)])
        eye = eye + rng.standard_normal(3)
        cams.append(camera(eye, width, height))
    return cams


def batched_jobs(seed: int = 4, n_cams: int = 64, n_levels: int = 5, radius: float = 40.0,
                 selective_radius: float = 120.0):
    """The batched multi-view mix: for each camera a resolution drawn uniformly from
    BATCH_RESOLUTIONS and a job drawn uniformly from {level 1..n_levels, selective}
    (job index n_levels means selective). Positions uniform on a sphere of ``radius``
    (``selective_radius`` for selective jobs), looking at the origin."""
    rng = _rng(seed)
    res = rng.integers(0, len(BATCH_RESOLUTIONS), n_cams)
    job = rng.integers(0, n_levels + 1, n_cams)
    d = rng.standard_normal((n_cams, 3))
    d /= np.linalg.norm(d, axis=1, keepdims=True)
    cams = []
    for i in range(n_cams):
        w, h = BATCH_RESOLUTIONS[res[i]]
        r = selective_radius if job[i] == n_levels else radius
        cams.append(camera(d[i] * r, w, h))
    return cams, [int(j) for j in job]


def with_jittered_clones(g: dict, frac: float, sigma: float, seed: int = 13) -> dict:
    """A level right after a densification step: a fraction ``frac`` of its Gaussians (drawn
    without replacement) appended again with their means moved by N(0, sigma^2) per axis and
    every other parameter copied (the state overlap pruning is applied to)."""
    rng = _rng(seed)
    n = g["means"].shape[0]
    pick = rng.choice(n, int(round(frac * n)), replace=False)
    out = {}
    for k, v in g.items():
        if k == "sh_degree":
            out[k] = v
            continue
        extra = v[pick].copy()
        if k == "means":
            extra = (extra + sigma * rng.standard_normal(extra.shape)).astype(np.float32)
        out[k] = np.ascontiguousarray(np.concatenate([v, extra]))
    return out
