"""Pins of the oracle's training loss (L1 + D-SSIM, Sec. 5.1.4 and the Loss step of
Algorithm 1) -- CPU only."""
import numpy as np
import pytest
import torch
from scipy.signal import windows

from oracle import loss as LS


def _imgs(seed, c=3, h=17, w=23):
    rng = np.random.default_rng(seed)
    return rng.random((c, h, w)), rng.random((c, h, w))


def test_window_is_the_normalised_gaussian():
    w = LS.window_1d().numpy()
    ref = windows.gaussian(11, std=1.5)          # library routine, independent of the oracle
    np.testing.assert_allclose(w, ref / ref.sum(), rtol=1e-14)
    w2 = LS.window_2d().numpy()
    assert abs(w2.sum() - 1.0) < 1e-14 and np.allclose(w2, w2.T) and np.allclose(w2, w2[::-1, ::-1])


def test_ssim_map_equals_the_per_pixel_definition_everywhere():
    x, y = _imgs(0, c=2, h=9, w=13)
    m = LS.ssim_map(torch.as_tensor(x), torch.as_tensor(y)).numpy()
    for c in range(2):
        for i in range(9):
            for j in range(13):
                assert abs(m[c, i, j] - LS.ssim_pixel_loop(x, y, c, i, j)) < 1e-12, (c, i, j)


def test_ssim_of_an_image_with_itself_is_one_and_the_loss_zero():
    x, _ = _imgs(1)
    t = torch.as_tensor(x)
    np.testing.assert_allclose(LS.ssim_map(t, t).numpy(), 1.0, atol=1e-12)
    L, g = LS.loss_and_grad(x, x)
    assert abs(L) < 1e-12
    assert np.abs(g).max() < 1e-9      # the maximum of SSIM, and |0| has subgradient 0


def test_ssim_of_constant_images_interior_closed_form():
    a, b = 0.3, 0.7
    x = np.full((1, 21, 21), a)
    y = np.full((1, 21, 21), b)
    m = LS.ssim_map(torch.as_tensor(x), torch.as_tensor(y)).numpy()
    want = (2 * a * b + LS.C1) / (a * a + b * b + LS.C1)   # variances and covariance vanish
    np.testing.assert_allclose(m[0, 5:-5, 5:-5], want, rtol=1e-12)
    # on the border the zero padding lowers the local means: not the closed form
    assert abs(m[0, 0, 0] - want) > 1e-6


def test_l1_part_and_lambda():
    x, y = _imgs(2)
    L, g = LS.loss_and_grad(x, y, lam=0.0)
    np.testing.assert_allclose(L, np.abs(x - y).mean(), rtol=1e-14)
    np.testing.assert_allclose(g, np.sign(x - y) / x.size, rtol=1e-14)
    L2, _ = LS.loss_and_grad(x, y, lam=1.0)
    ssim = LS.ssim_map(torch.as_tensor(x), torch.as_tensor(y)).mean().item()
    np.testing.assert_allclose(L2, 1.0 - ssim, rtol=1e-14)


@pytest.mark.parametrize("seed", [3, 4])
def test_gradient_matches_central_finite_differences(seed):
    x, y = _imgs(seed, c=2, h=12, w=15)
    # keep |x - y| away from 0 so that the L1 kink is not crossed by the perturbation
    x = np.where(np.abs(x - y) < 0.05, y + 0.1, x)
    _, g = LS.loss_and_grad(x, y)
    rng = np.random.default_rng(seed)
    h = 1e-6
    for _ in range(60):
        c, i, j = rng.integers(0, 2), rng.integers(0, 12), rng.integers(0, 15)
        xp, xm = x.copy(), x.copy()
        xp[c, i, j] += h
        xm[c, i, j] -= h
        fd = (LS.loss_and_grad(xp, y)[0] - LS.loss_and_grad(xm, y)[0]) / (2 * h)
        assert abs(fd - g[c, i, j]) <= 1e-6 * max(abs(g[c, i, j]), 1e-4), (c, i, j, fd, g[c, i, j])
