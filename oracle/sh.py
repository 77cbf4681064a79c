"""Real spherical harmonics up to degree 3, written from the textbook definition.

Sec. 3 gives each Gaussian "spherical harmonic coefficients" for its view-dependent
colour, without fixing a basis. The reading used here: the real orthonormal basis with
the Condon-Shortley phase, index k = l*l + l + m (m = -l..l), built from

    Y_l^0  = K_l^0 P_l(z)
    Y_l^m  = sqrt(2) K_l^m P_l^m(z) cos(m phi)          (m > 0)
    Y_l^-m = sqrt(2) K_l^m P_l^m(z) sin(m phi)          (m > 0)
    K_l^m  = sqrt((2l+1)/(4 pi) * (l-m)!/(l+m)!)
    P_l^m(z) = (-1)^m (1-z^2)^(m/2) d^m/dz^m P_l(z)

and, for a unit direction (x, y, z), (1-z^2)^(m/2) cos(m phi) = Re((x+iy)^m),
(1-z^2)^(m/2) sin(m phi) = Im((x+iy)^m). The Legendre polynomials come from numpy's
Legendre-series conversion; nothing here is a hand-typed table.

Colour (reading of the 3DGS convention the paper builds on): rgb = max(0, sum_k c_k Y_k(d)
+ 0.5) with d the unit vector from the camera centre to the Gaussian mean.
"""
from __future__ import annotations

import math

import numpy as np
import torch
from numpy.polynomial import legendre as npleg
from numpy.polynomial import polynomial as nppoly


def _norm(l: int, m: int) -> float:
    return math.sqrt((2 * l + 1) / (4.0 * math.pi) * math.factorial(l - m) / math.factorial(l + m))


def _dm_legendre(l: int, m: int) -> np.ndarray:
    """Power-series coefficients (ascending) of d^m/dz^m P_l(z)."""
    series = np.zeros(l + 1)
    series[l] = 1.0
    p = npleg.leg2poly(series)
    for _ in range(m):
        p = nppoly.polyder(p)
    return np.atleast_1d(p)


def _polyval(coeffs: np.ndarray, z: torch.Tensor) -> torch.Tensor:
    out = torch.zeros_like(z)
    for c in coeffs[::-1]:
        out = out * z + float(c)
    return out


def basis(dirs: torch.Tensor, degree: int) -> torch.Tensor:
    """Real SH basis [N, (degree+1)^2] at unit directions ``dirs`` [N, 3] (float64)."""
    x, y, z = dirs[:, 0], dirs[:, 1], dirs[:, 2]
    # Re/Im of (x + i y)^m for m = 0..degree
    re = [torch.ones_like(x)]
    im = [torch.zeros_like(x)]
    for _ in range(degree):
        r, i = re[-1], im[-1]
        re.append(r * x - i * y)
        im.append(r * y + i * x)
    cols = []
    for l in range(degree + 1):
        for m in range(-l, l + 1):
            am = abs(m)
            pz = _polyval(_dm_legendre(l, am), z)
            if m == 0:
                cols.append(_norm(l, 0) * pz)
            else:
                k = math.sqrt(2.0) * _norm(l, am) * (-1.0) ** am
                cols.append(k * pz * (re[am] if m > 0 else im[am]))
    return torch.stack(cols, dim=1)


def colour(sh: torch.Tensor, means: torch.Tensor, cam_pos: torch.Tensor, degree: int):
    """rgb [N,3] = max(0, sum_k sh[:, k, :] * Y_k(dir) + 0.5); returns (rgb, pre-clamp)."""
    d = means - cam_pos[None, :]
    d = d / torch.linalg.norm(d, dim=1, keepdim=True)
    y = basis(d, degree)                                   # [N, K]
    k = (degree + 1) ** 2
    raw = torch.einsum("nk,nkc->nc", y, sh[:, :k, :]) + 0.5
    return torch.clamp(raw, min=0.0), raw
