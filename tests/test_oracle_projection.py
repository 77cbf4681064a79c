"""Pins of the oracle's projection, extent and rectangles (Eq. 2) -- CPU only."""
import math

import numpy as np
import torch

from oracle import gaussians as G
from oracle import projection as P
from oracle import raster as R
from paper_2408_12894_gb300 import synth


def _pinhole(t, cam):
    return np.array([cam["fx"] * t[0] / t[2] + cam["cx"], cam["fy"] * t[1] / t[2] + cam["cy"]])


def test_covariance_projection_matches_finite_difference_jacobian():
    rng = np.random.default_rng(0)
    cam = synth.camera((1.0, 2.0, -6.0), 640, 480)
    n = 200
    means = rng.normal(0, 1.0, (n, 3))
    q = torch.as_tensor(rng.normal(size=(n, 4)))
    s = torch.as_tensor(np.exp(rng.normal(-2, 0.5, (n, 3))))
    cov3 = G.covariance(q, s)
    dil = 0.3
    t, mean2d, cov2d, front = P.project(torch.as_tensor(means), cov3, cam, dil, 0.2)
    rw = np.asarray(cam["viewmat"], np.float64)[:, :3]
    lim = 1.3 * 0.5 * cam["width"] / cam["fx"]
    checked = 0
    for i in range(n):
        ti = t[i].numpy()
        if not front[i] or abs(ti[0] / ti[2]) > lim or abs(ti[1] / ti[2]) > 1.3 * 0.5 * 480 / cam["fy"]:
            continue
        h = 1e-6 * ti[2]
        jac = np.stack([(_pinhole(ti + h * e, cam) - _pinhole(ti - h * e, cam)) / (2 * h)
                        for e in np.eye(3)], 1)
        want = jac @ rw @ cov3[i].numpy() @ rw.T @ jac.T + dil * np.eye(2)
        np.testing.assert_allclose(cov2d[i].numpy(), want, rtol=1e-8, atol=1e-12)
        np.testing.assert_allclose(mean2d[i].numpy(), _pinhole(ti, cam), rtol=1e-13)
        checked += 1
    assert checked > 150


def test_isotropic_gaussian_on_optical_axis():
    for z0, s, dil in ((3.0, 0.05, 0.3), (10.0, 0.2, 0.0), (40.0, 0.03125, 0.3)):
        cam = synth.camera((0.0, 0.0, -z0), 1920, 1080)
        cov3 = G.covariance(torch.tensor([[1.0, 0, 0, 0]], dtype=torch.float64),
                            torch.full((1, 3), s, dtype=torch.float64))
        _, m2, c2, _ = P.project(torch.zeros((1, 3), dtype=torch.float64), cov3, cam, dil, 0.2)
        sig = cam["fx"] * s / z0
        np.testing.assert_allclose(c2[0].numpy(), (sig * sig + dil) * np.eye(2), rtol=1e-6)
        np.testing.assert_allclose(m2[0].numpy(), [960.0, 540.0], atol=1e-9)


def test_projected_covariance_is_positive_definite():
    rng = np.random.default_rng(1)
    cam = synth.camera((0.0, 0.0, -5.0), 256, 256)
    q = torch.as_tensor(rng.normal(size=(500, 4)))
    s = torch.as_tensor(np.exp(rng.normal(-3, 1.5, (500, 3))))
    _, _, c2, front = P.project(torch.as_tensor(rng.normal(0, 1, (500, 3))), G.covariance(q, s),
                                cam, 0.3, 0.2)
    ev = np.linalg.eigvalsh(c2.numpy())
    assert np.all(ev[front.numpy()] >= 0.3 - 1e-9)


def test_opacity_aware_extent_is_exact_support():
    rng = np.random.default_rng(2)
    for trial in range(40):
        a = rng.uniform(0.5, 30)
        c = rng.uniform(0.5, 30)
        b = rng.uniform(-0.9, 0.9) * math.sqrt(a * c)
        cov = torch.tensor([[[a, b], [b, c]]], dtype=torch.float64)
        o = torch.tensor([rng.uniform(0.01, 1.0)], dtype=torch.float64)
        r, ok = P.radius(cov, o, 0)
        assert ok[0]
        con, _ = P.conic(cov)
        # tight: on the major axis at distance r the opacity is exactly 1/255
        w, v = np.linalg.eigh(cov[0].numpy())
        d = v[:, 1] * float(r[0])
        qv = con[0, 0] * d[0] ** 2 + 2 * con[0, 1] * d[0] * d[1] + con[0, 2] * d[1] ** 2
        assert math.isclose(float(o[0]) * math.exp(-0.5 * float(qv)), 1 / 255, rel_tol=1e-10)
        # sound: any offset with opacity >= 1/255 lies within r
        pts = rng.uniform(-1.2, 1.2, (4000, 2)) * float(r[0])
        qq = con[0, 0].item() * pts[:, 0] ** 2 + 2 * con[0, 1].item() * pts[:, 0] * pts[:, 1] \
            + con[0, 2].item() * pts[:, 1] ** 2
        inside = float(o[0]) * np.exp(-0.5 * qq) >= 1 / 255
        assert np.all(np.linalg.norm(pts[inside], axis=1) <= float(r[0]) * (1 + 1e-12))
    r, ok = P.radius(torch.eye(2, dtype=torch.float64)[None], torch.tensor([0.5 / 255], dtype=torch.float64), 0)
    assert not ok[0]


def test_pixel_rect_brute_force():
    rng = np.random.default_rng(3)
    W, H = 50, 37
    u = rng.uniform(-20, 70, 3000)
    v = rng.uniform(-20, 60, 3000)
    r = rng.uniform(0.01, 15, 3000)
    x0, x1, y0, y1 = P.pixel_rect(u, v, r, W, H)
    cols = np.arange(W) + 0.5
    rows = np.arange(H) + 0.5
    for i in range(3000):
        cx = np.nonzero(np.abs(cols - u[i]) <= r[i])[0]
        cy = np.nonzero(np.abs(rows - v[i]) <= r[i])[0]
        if cx.size == 0 or cy.size == 0:
            assert x0[i] > x1[i] or y0[i] > y1[i]
        else:
            assert (x0[i], x1[i], y0[i], y1[i]) == (cx[0], cx[-1], cy[0], cy[-1])


def test_pixel_rect_f32_agrees_away_from_boundaries():
    rng = np.random.default_rng(4)
    u = rng.uniform(-20, 1000, 20000).astype(np.float32)
    v = rng.uniform(-20, 600, 20000).astype(np.float32)
    r = rng.uniform(0.01, 50, 20000).astype(np.float32)
    a = P.pixel_rect(u, v, r, 960, 540)
    b = P.pixel_rect_f32(u, v, r, 960, 540)
    d = np.minimum.reduce([np.abs(((u.astype(np.float64) + s * r) - 0.5) - np.round((u.astype(np.float64) + s * r) - 0.5)) for s in (-1, 1)] +
                          [np.abs(((v.astype(np.float64) + s * r) - 0.5) - np.round((v.astype(np.float64) + s * r) - 0.5)) for s in (-1, 1)])
    far = d > 1e-4
    for x, y in zip(a, b):
        assert np.array_equal(x[far], y[far])


def test_tile_rect_counts():
    px = (np.array([0, 17, 5, 40]), np.array([15, 40, 4, 63]), np.array([0, 3, 0, 0]),
          np.array([31, 3, 9, 15]))
    tx0, tx1, ty0, ty1, n = P.tile_rect(px, 16, 16, np.array([True, True, True, False]))
    assert list(n) == [2, 2, 0, 0]
    assert (tx0[1], tx1[1], ty0[1], ty1[1]) == (1, 2, 0, 0)


def test_near_plane_culls():
    cam = synth.camera((0.0, 0.0, -3.0), 64, 64)
    means = torch.tensor([[0.0, 0.0, -2.85], [0.0, 0.0, -2.81], [0.0, 0.0, 0.0]], dtype=torch.float64)
    g = {"means": means.numpy(), "quats": np.tile([1.0, 0, 0, 0], (3, 1)),
         "s_opt": np.full((3, 3), -3.0), "opacity_logit": np.zeros(3), "sh": np.zeros((3, 1, 3))}
    pre = R.preprocess(R.params(g), 0, 0.0, cam, R.Config())
    assert list(pre["valid"].numpy()) == [False, False, True]
