"""Gaussian parameterisation: Eq. 1, Eq. 3, Eq. 4, Eq. 5 (FP64).

* Eq. 3 (Sec. 4.1): s_min^(l) = lambda * rho^(1-l) for 1 <= l < L_max, 0 at L_max.
* Eq. 4 (Sec. 4.1): s^(l) = exp(s_opt) + s_min^(l), per axis.
* Eq. 5 (Sec. 4.2): s_opt <- log(s^(l) - s_min^(l+1)), so that s^(l+1) = s^(l).
* Eq. 1 (Sec. 3):   Sigma = R S S^T R^T with S = diag(s) and R from the quaternion q.

Quaternion reading (the paper does not fix one): q = (w, x, y, z), normalised before use,
R the standard rotation matrix of the unit quaternion.
"""
from __future__ import annotations

import torch


def s_min_schedule(lam: float = 0.2, rho: float = 4.0, l_max: int = 5) -> list[float]:
    """Eq. 3: the per-level minimum 3D scale for levels 1..l_max."""
    return [lam * rho ** (1 - l) if l < l_max else 0.0 for l in range(1, l_max + 1)]


def constrained_scale(s_opt: torch.Tensor, s_min: float) -> torch.Tensor:
    """Eq. 4."""
    return torch.exp(s_opt) + s_min


def adjust_scale(s_opt: torch.Tensor, s_min_cur: float, s_min_next: float) -> torch.Tensor:
    """Eq. 5: the s_opt that gives level l+1 the same scale that level l had."""
    return torch.log(constrained_scale(s_opt, s_min_cur) - s_min_next)


def rotation(q: torch.Tensor) -> torch.Tensor:
    """[N,4] (w,x,y,z) -> [N,3,3] rotation of the normalised quaternion."""
    q = q / torch.linalg.norm(q, dim=1, keepdim=True)
    w, x, y, z = q[:, 0], q[:, 1], q[:, 2], q[:, 3]
    r = torch.stack([
        1 - 2 * (y * y + z * z), 2 * (x * y - w * z), 2 * (x * z + w * y),
        2 * (x * y + w * z), 1 - 2 * (x * x + z * z), 2 * (y * z - w * x),
        2 * (x * z - w * y), 2 * (y * z + w * x), 1 - 2 * (x * x + y * y),
    ], dim=1)
    return r.reshape(-1, 3, 3)


def covariance(q: torch.Tensor, s: torch.Tensor) -> torch.Tensor:
    """Eq. 1: Sigma = R S S^T R^T, [N,3,3]."""
    rs = rotation(q) * s[:, None, :]          # R @ diag(s)
    return rs @ rs.transpose(1, 2)


def sigmoid(x: torch.Tensor) -> torch.Tensor:
    return 1.0 / (1.0 + torch.exp(-x))
