"""Pins of the oracle's spherical-harmonic colour -- CPU only."""
import math

import numpy as np
import pytest
import torch

from oracle import sh as SH
from paper_2408_12894_gb300 import synth


def _quadrature(n_z=8, n_phi=16):
    """Gauss-Legendre in z times uniform phi: exact for the degree <= 6 products of two
    degree <= 3 harmonics."""
    z, wz = np.polynomial.legendre.leggauss(n_z)
    phi = 2 * math.pi * np.arange(n_phi) / n_phi
    zz, pp = np.meshgrid(z, phi, indexing="ij")
    s = np.sqrt(1 - zz ** 2)
    dirs = np.stack([s * np.cos(pp), s * np.sin(pp), zz], -1).reshape(-1, 3)
    w = (wz[:, None] * np.full(n_phi, 2 * math.pi / n_phi)[None, :]).ravel()
    return dirs, w


def test_orthonormal_by_exact_quadrature():
    dirs, w = _quadrature()
    y = SH.basis(torch.as_tensor(dirs), 3).numpy()
    gram = (y * w[:, None]).T @ y
    np.testing.assert_allclose(gram, np.eye(16), atol=1e-12)


def test_matches_scipy_complex_harmonics():
    from scipy import special
    if not hasattr(special, "sph_harm_y"):
        pytest.skip("scipy without sph_harm_y")
    rng = np.random.default_rng(0)
    d = rng.normal(size=(500, 3))
    d /= np.linalg.norm(d, axis=1, keepdims=True)
    theta = np.arccos(np.clip(d[:, 2], -1, 1))
    phi = np.arctan2(d[:, 1], d[:, 0])
    y = SH.basis(torch.as_tensor(d), 3).numpy()
    for l in range(4):
        for m in range(-l, l + 1):
            c = special.sph_harm_y(l, abs(m), theta, phi)      # Condon-Shortley phase included
            if m == 0:
                ref = c.real
            elif m > 0:
                ref = math.sqrt(2) * c.real
            else:
                ref = math.sqrt(2) * c.imag
            np.testing.assert_allclose(y[:, l * l + l + m], ref, atol=1e-12,
                                       err_msg=f"l={l} m={m}")


def test_addition_theorem_band_energy():
    rng = np.random.default_rng(1)
    d = rng.normal(size=(300, 3))
    d /= np.linalg.norm(d, axis=1, keepdims=True)
    y = SH.basis(torch.as_tensor(d), 3).numpy()
    for l in range(4):
        band = (y[:, l * l:(l + 1) ** 2] ** 2).sum(1)
        np.testing.assert_allclose(band, (2 * l + 1) / (4 * math.pi), rtol=1e-12)


def test_first_bands_closed_form():
    # Y_00 = 1/(2 sqrt(pi)); band 1 = sqrt(3/(4 pi)) * (-y, z, -x) with the CS phase
    rng = np.random.default_rng(2)
    d = rng.normal(size=(50, 3))
    d /= np.linalg.norm(d, axis=1, keepdims=True)
    y = SH.basis(torch.as_tensor(d), 1).numpy()
    c1 = math.sqrt(3 / (4 * math.pi))
    np.testing.assert_allclose(y[:, 0], 0.5 / math.sqrt(math.pi), rtol=1e-15)
    np.testing.assert_allclose(y[:, 1:], c1 * np.stack([-d[:, 1], d[:, 2], -d[:, 0]], 1), atol=1e-15)


def test_degree0_colour_is_the_drawn_colour():
    g = synth.gaussian_set(5, 200, sh_degree=0)
    rgb, _ = SH.colour(torch.as_tensor(g["sh"].astype(np.float64)),
                       torch.as_tensor(g["means"].astype(np.float64)),
                       torch.tensor([0.0, 0.0, -3.0], dtype=torch.float64), 0)
    u = g["sh"][:, 0, :].astype(np.float64) * synth.Y00 + 0.5
    np.testing.assert_allclose(rgb.numpy(), u, atol=1e-7)
    assert rgb.min() >= 0 and rgb.max() <= 1


def test_colour_clamps_at_zero():
    sh = torch.zeros((2, 1, 3), dtype=torch.float64)
    sh[0, 0, :] = -10.0
    rgb, raw = SH.colour(sh, torch.zeros((2, 3), dtype=torch.float64) + 1,
                         torch.zeros(3, dtype=torch.float64), 0)
    assert torch.all(rgb[0] == 0) and torch.all(raw[0] < 0)
    np.testing.assert_allclose(rgb[1].numpy(), 0.5)
