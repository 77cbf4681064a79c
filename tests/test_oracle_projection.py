"""Pins of the oracle's projection, extent and rectangles (Eq. 2) -- CPU only."""
import math

import numpy as np
import pytest
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


# ---------------------------------------------------------------------------------------
# rule 2: ellipse rows
# ---------------------------------------------------------------------------------------
def _random_splats(seed, n, W, H):
    """Random 2D Gaussians: anisotropy up to 1:40, any orientation, partly off-screen."""
    rng = np.random.default_rng(seed)
    th = rng.uniform(0, np.pi, n)
    s1 = np.exp(rng.uniform(np.log(0.3), np.log(25.0), n))
    s2 = s1 / np.exp(rng.uniform(0, np.log(40.0), n))
    R_ = np.stack([np.cos(th), -np.sin(th), np.sin(th), np.cos(th)], 1).reshape(n, 2, 2)
    D = np.zeros((n, 2, 2))
    D[:, 0, 0], D[:, 1, 1] = s1 ** 2, s2 ** 2
    cov = R_ @ D @ R_.transpose(0, 2, 1) + 0.3 * np.eye(2)[None]
    u = rng.uniform(-30, W + 30, n)
    v = rng.uniform(-30, H + 30, n)
    o = rng.uniform(0.003, 1.0, n)
    return u, v, cov, o


def _alpha(u, v, cov, o, W, H):
    """o exp(-q/2) at every pixel centre, FP64 [n, H, W] (conic from numpy's inverse)."""
    inv = np.linalg.inv(cov)
    xs = np.arange(W) + 0.5
    ys = np.arange(H) + 0.5
    dx = xs[None, None, :] - u[:, None, None]
    dy = ys[None, :, None] - v[:, None, None]
    q = inv[:, 0, 0, None, None] * dx * dx + 2 * inv[:, 0, 1, None, None] * dx * dy \
        + inv[:, 1, 1, None, None] * dy * dy
    return o[:, None, None] * np.exp(-0.5 * q)


def _listed(segs, n, tiles_x, tiles_y):
    out = np.zeros((n, tiles_y, tiles_x), bool)
    for j, ty, a, b in zip(*segs):
        out[j, ty, a:b + 1] = True
    return out


def _rule2(u, v, cov, o, W, H, tile, dtype=np.float64):
    ext, ok = P.ellipse_extent(torch.as_tensor(cov), torch.as_tensor(o))
    e = ext.numpy()
    if dtype == np.float32:
        u, v, e = u.astype(np.float32), v.astype(np.float32), e.astype(np.float32)
    px = P.pixel_rect_xy(u, v, e[:, 2], e[:, 3], W, H, dtype)
    return P.ellipse_segments(u, v, e, px, tile, tile, ok.numpy(), dtype), e, ok.numpy()


def test_ellipse_extent_closed_forms():
    # axis-aligned: m = 0, h = sx / sy, rx = sqrt(tau) sx, ry = sqrt(tau) sy
    cov = torch.tensor([[[9.0, 0.0], [0.0, 4.0]]], dtype=torch.float64)
    o = torch.tensor([0.5], dtype=torch.float64)
    e, ok = P.ellipse_extent(cov, o)
    tau = 2 * math.log(255 * 0.5) * (1 + 2.0 ** -10)
    np.testing.assert_allclose(e[0].numpy(), [0.0, 1.5, 3 * math.sqrt(tau), 2 * math.sqrt(tau)],
                               rtol=1e-14)
    assert bool(ok[0])
    # rotated: the boundary, sampled from the eigen-decomposition, has x extremes +-rx,
    # y extremes +-ry, and every boundary point satisfies x = m dy +- h sqrt(ry^2 - dy^2)
    u, v, covs, oo = _random_splats(11, 50, 100, 100)
    e, ok = P.ellipse_extent(torch.as_tensor(covs), torch.as_tensor(oo))
    e = e.numpy()
    t = np.linspace(0, 2 * np.pi, 20001)
    for i in np.nonzero(ok.numpy())[0]:
        lam, V = np.linalg.eigh(covs[i])
        tau = 2 * math.log(255 * oo[i]) * (1 + 2.0 ** -10)
        pts = (V @ (np.sqrt(tau * lam)[:, None] * np.stack([np.cos(t), np.sin(t)])))
        m, h, rx, ry = e[i]
        assert abs(pts[0].max() - rx) <= 1e-6 * rx and abs(pts[1].max() - ry) <= 1e-6 * ry
        w = h * np.sqrt(np.maximum(ry * ry - pts[1] ** 2, 0))
        off = np.minimum(np.abs(pts[0] - (m * pts[1] + w)), np.abs(pts[0] - (m * pts[1] - w)))
        assert off.max() <= 1e-6 * rx + 1e-3 * h * ry * np.sqrt(2 * np.pi / 20001)
    # culled below 1/255 and for a singular covariance
    e, ok = P.ellipse_extent(torch.tensor([[[1.0, 0.0], [0.0, 1.0]], [[1.0, 1.0], [1.0, 1.0]]],
                                          dtype=torch.float64),
                             torch.tensor([0.5 / 255, 0.5], dtype=torch.float64))
    assert not ok.any() and float(e.abs().max()) == 0.0


@pytest.mark.parametrize("seed,tile", [(0, 16), (1, 8)])
def test_ellipse_rows_cover_every_supported_pixel(seed, tile):
    W, H = 120, 90
    u, v, cov, o = _random_splats(seed, 400, W, H)
    a = _alpha(u, v, cov, o, W, H)
    tx, ty = -(-W // tile), -(-H // tile)
    for dtype, thr in ((np.float64, 1 / 255), (np.float32, (1 / 255) * (1 + 1e-4))):
        (segs, touched), _, ok = _rule2(u, v, cov, o, W, H, tile, dtype)
        lst = _listed(segs, u.size, tx, ty)
        assert np.array_equal(touched, lst.reshape(u.size, -1).sum(1))
        need = a >= thr
        cov_tiles = np.zeros((u.size, ty, tx), bool)
        jj, yy, xx = np.nonzero(need)
        cov_tiles[jj, yy // tile, xx // tile] = True
        assert not np.any(cov_tiles & ~lst), dtype


@pytest.mark.parametrize("seed,tile", [(2, 16), (3, 8)])
def test_ellipse_rows_are_tight(seed, tile):
    # every listed tile's pixel-centre rectangle meets the ellipse q <= tau: the minimum of
    # the convex q over the rectangle, taken on its edges (1D closed form), is <= tau
    W, H = 120, 90
    u, v, cov, o = _random_splats(seed, 300, W, H)
    (segs, touched), e, ok = _rule2(u, v, cov, o, W, H, tile)
    inv = np.linalg.inv(cov)
    tau = np.where(ok, 2 * np.log(255 * o) * (1 + 2.0 ** -10), 0)

    def qmin(j, xa, xb, ya, yb):
        a, b, c = inv[j, 0, 0], inv[j, 0, 1], inv[j, 1, 1]
        if xa <= u[j] <= xb and ya <= v[j] <= yb:
            return 0.0
        best = np.inf
        for xe in (xa, xb):
            dx = xe - u[j]
            dy = np.clip(-b * dx / c, ya - v[j], yb - v[j])
            best = min(best, a * dx * dx + 2 * b * dx * dy + c * dy * dy)
        for ye in (ya, yb):
            dy = ye - v[j]
            dx = np.clip(-b * dy / a, xa - u[j], xb - u[j])
            best = min(best, a * dx * dx + 2 * b * dx * dy + c * dy * dy)
        return best

    n_tiles = 0
    for j, tyi, c0, c1 in zip(*segs):
        ya = max(tyi * tile, 0) + 0.5
        yb = min(tyi * tile + tile - 1, H - 1) + 0.5
        for txi in range(c0, c1 + 1):
            xa = txi * tile + 0.5
            xb = min(txi * tile + tile - 1, W - 1) + 0.5
            assert qmin(j, xa, xb, ya, yb) <= tau[j] * (1 + 1e-9) + 1e-12
            n_tiles += 1
    assert n_tiles == touched.sum() > 500


def test_ellipse_rows_f32_mirror_matches_f64_rule_almost_everywhere():
    W, H = 1920, 1080
    u, v, cov, o = _random_splats(7, 20000, W, H)
    (s64, t64), _, _ = _rule2(u, v, cov, o, W, H, 16)
    (s32, t32), _, _ = _rule2(u, v, cov, o, W, H, 16, np.float32)
    assert np.mean(t64 != t32) < 2e-3
    assert abs(int(t64.sum()) - int(t32.sum())) <= 1e-4 * t64.sum()
