"""The training loss of each level and its gradient, FP64 -- TEST INFRASTRUCTURE ONLY.

Every level is trained with the loss of the backbone it builds on (Sec. 5.1.4,
Implementation: "L1 and SSIM losses ... consistent with the backbone"; the Loss step of
Algorithm 1). Reading of that backbone loss (the paper prints no formula):

* L = (1 - lam) L1 + lam (1 - SSIM), lam = 0.2;
* L1 = mean over channels and pixels of |I - I_hat|;
* SSIM = mean over channels and pixels of the SSIM map of Wang et al. (2004): local means,
  variances and covariance are sums weighted by an 11 x 11 Gaussian window (sigma = 1.5,
  normalised to 1) centred on the pixel, with zero values outside the image, and
  SSIM(p) = ((2 mu_x mu_y + C1)(2 s_xy + C2)) / ((mu_x^2 + mu_y^2 + C1)(s_x^2 + s_y^2 + C2)),
  s_x^2 = E[x^2] - mu_x^2, s_xy = E[xy] - mu_x mu_y, C1 = 0.01^2, C2 = 0.03^2 (unit range);
* images are planar [C, H, W]; for a batch of images the loss is the sum of the images'
  losses (each image's gradient is that of its own loss).

The window sums are written out as a correlation with the window (``torch.nn.functional.
conv2d`` as the library step); the gradient is torch autograd of this forward, with
d|x|/dx = 0 at x = 0.
"""
from __future__ import annotations

import math

import numpy as np
import torch

LAMBDA = 0.2
C1 = 0.01 ** 2
C2 = 0.03 ** 2
WINDOW = 11
SIGMA = 1.5


def window_1d(size: int = WINDOW, sigma: float = SIGMA) -> torch.Tensor:
    """Normalised 1-D Gaussian weights, centred on the middle tap."""
    x = torch.arange(size, dtype=torch.float64) - (size - 1) / 2.0
    w = torch.exp(-x * x / (2.0 * sigma * sigma))
    return w / w.sum()


def window_2d(size: int = WINDOW, sigma: float = SIGMA) -> torch.Tensor:
    """The 2-D window: the outer product of the 1-D weights (sums to 1)."""
    w = window_1d(size, sigma)
    return w[:, None] * w[None, :]


def local_sum(img: torch.Tensor, size: int = WINDOW, sigma: float = SIGMA) -> torch.Tensor:
    """Window-weighted sum around every pixel of each channel of [C, H, W], zeros outside."""
    w = window_2d(size, sigma)[None, None]
    c = img.shape[0]
    return torch.nn.functional.conv2d(img[:, None], w.expand(1, 1, size, size),
                                      padding=size // 2)[:, 0].reshape(c, *img.shape[1:])


def ssim_map(x: torch.Tensor, y: torch.Tensor) -> torch.Tensor:
    """The SSIM of every pixel and channel of two [C, H, W] images."""
    mx, my = local_sum(x), local_sum(y)
    exx, eyy, exy = local_sum(x * x), local_sum(y * y), local_sum(x * y)
    sxx, syy, sxy = exx - mx * mx, eyy - my * my, exy - mx * my
    num = (2.0 * mx * my + C1) * (2.0 * sxy + C2)
    den = (mx * mx + my * my + C1) * (sxx + syy + C2)
    return num / den


def l1(x: torch.Tensor, y: torch.Tensor) -> torch.Tensor:
    return torch.abs(x - y).mean()


def loss(x: torch.Tensor, y: torch.Tensor, lam: float = LAMBDA) -> torch.Tensor:
    """(1 - lam) L1 + lam (1 - SSIM) of one [C, H, W] image against its target."""
    return (1.0 - lam) * l1(x, y) + lam * (1.0 - ssim_map(x, y).mean())


def loss_and_grad(img: np.ndarray, target: np.ndarray, lam: float = LAMBDA):
    """(loss, dL/dimg) in FP64 for one [C, H, W] image."""
    x = torch.as_tensor(np.asarray(img, dtype=np.float64)).clone().requires_grad_(True)
    y = torch.as_tensor(np.asarray(target, dtype=np.float64))
    L = loss(x, y, lam)
    L.backward()
    return float(L.detach()), x.grad.numpy()


def ssim_pixel_loop(x: np.ndarray, y: np.ndarray, c: int, i: int, j: int,
                    size: int = WINDOW, sigma: float = SIGMA) -> float:
    """SSIM of one pixel (row i, column j) of channel c by explicit loops over the window
    (pixels outside the image contribute zeros): the definition, for small checks."""
    r = size // 2
    wsum = 0.0
    w = {}
    for a in range(-r, r + 1):
        for b in range(-r, r + 1):
            w[a, b] = math.exp(-(a * a + b * b) / (2.0 * sigma * sigma))
            wsum += w[a, b]
    mx = my = exx = eyy = exy = 0.0
    H, W = x.shape[1], x.shape[2]
    for a in range(-r, r + 1):
        for b in range(-r, r + 1):
            ii, jj = i + a, j + b
            if 0 <= ii < H and 0 <= jj < W:
                k = w[a, b] / wsum
                xv, yv = float(x[c, ii, jj]), float(y[c, ii, jj])
                mx += k * xv
                my += k * yv
                exx += k * xv * xv
                eyy += k * yv * yv
                exy += k * xv * yv
    sxx, syy, sxy = exx - mx * mx, eyy - my * my, exy - mx * my
    return ((2 * mx * my + C1) * (2 * sxy + C2)) / ((mx * mx + my * my + C1) * (sxx + syy + C2))
