"""Density control on the GPU (Densification and Pruning of Algorithm 1) against the
oracle: the 2D-gradient statistics after a backward, and the clone / split / prune step
(the new set, its order and the Adam moments)."""
import numpy as np
import pytest
import torch

from gpu_helpers import assert_grad_close, rasterizer
from oracle import densify as D
from oracle import raster as R
from paper_2408_12894_gb300 import flod, synth

pytestmark = pytest.mark.gpu


def test_statistics_match_the_oracle_2d_gradient_norms():
    g = synth.gaussian_set(40, 3000, k=8, radius=1.0, sh_degree=3, s_mean=-3.0)
    cams = [synth.camera((0.3, -0.2, -3.0), 96, 64), synth.camera((1.4, 0.3, -2.6), 80, 72)]
    dL = synth.upstream_gradient(41, cams)
    rast = rasterizer([g], cams, [0.01])
    rgb, T, nc = rast.forward()
    rast.blend_bwd(torch.as_tensor(dL, device="cuda"), T, nc)
    acc = torch.zeros(g["means"].shape[0], device="cuda")
    den = torch.zeros_like(acc)
    rast.densify_stats([acc], [den])
    rast.densify_stats([acc], [den])      # twice: the statistics add up
    torch.cuda.synchronize()
    tt = rast.region("tiles_touched", torch.int32, rast.layout.units).cpu().numpy()
    ra, rd = np.zeros(acc.numel()), np.zeros(acc.numel())
    vis_all = np.ones(acc.numel(), bool)
    off = 0
    for v, c in enumerate(cams):
        n = 3 * c["width"] * c["height"]
        p = R.params(g, requires_grad=False)
        with torch.no_grad():
            pre = R.preprocess(p, 3, 0.01, c, R.Config())
        _, _, _, g2 = R.render_tiled(pre, c, R.Config(), grad_out=dL[off:off + n].reshape(3, c["height"], c["width"]))
        off += n
        vis = pre["tiles_touched"] > 0
        u0 = rast.unit_off[v]
        gpu_vis = tt[u0:u0 + acc.numel()] > 0
        vis_all &= vis == gpu_vis
        for _ in range(2):
            ra, rd = D.stats_update(ra, rd, g2["mean2d"].numpy(), vis, c["width"], c["height"])
    got_a, got_d = acc.cpu().numpy(), den.cpu().numpy()
    assert vis_all.mean() > 0.99
    assert np.array_equal(got_d[vis_all], rd[vis_all])
    assert_grad_close({"accum": got_a[vis_all]}, {"accum": ra[vis_all]}, "densify statistics")


def _inputs(n=4000, seed=42):
    rng = np.random.default_rng(seed)
    g = synth.gaussian_set(seed, n, k=8, radius=1.0, sh_degree=3, s_mean=-3.0)
    # scales clear of the clone/split threshold 0.05, opacities clear of 0.005, statistics
    # clear of tau: no decision within rounding of its threshold
    g["s_opt"] = np.where(rng.random((n, 1)) < 0.5, np.log(0.02), np.log(0.2)).astype(np.float32) \
        + rng.normal(0, 0.1, (n, 3)).astype(np.float32)
    g["opacity_logit"] = np.where(rng.random(n) < 0.1, -8.0, 1.0).astype(np.float32)
    denom = rng.integers(0, 5, n).astype(np.float32)
    accum = (denom * np.where(rng.random(n) < 0.4, 5e-4, 5e-5)).astype(np.float32)
    normals = rng.standard_normal((2 * n, 3)).astype(np.float32)
    return g, accum, denom, normals


def test_densify_step_matches_the_oracle_with_moments():
    g, accum, denom, normals = _inputs()
    s_min = 0.01
    gs = flod.GaussianSet.from_numpy(g, s_min)
    rng = np.random.default_rng(43)
    m = [torch.as_tensor(rng.normal(size=np.shape(g[f])).astype(np.float32), device="cuda")
         for f in flod.GaussianSet.FIELDS]
    v = [torch.as_tensor(rng.random(np.shape(g[f])).astype(np.float32), device="cuda")
         for f in flod.GaussianSet.FIELDS]
    dev = lambda a: torch.as_tensor(a, device="cuda")
    new, mo, vo, counts = flod.densify(gs, dev(accum), dev(denom), dev(normals), tau=2e-4,
                                       max_clone_scale=0.05, min_opacity=0.005, m=m, v=v)
    torch.cuda.synchronize()
    mn = {f: t.cpu().numpy() for f, t in zip(flod.GaussianSet.FIELDS, m)}
    vn = {f: t.cpu().numpy() for f, t in zip(flod.GaussianSet.FIELDS, v)}
    ref, rm, rv = D.densify(g, s_min, accum, denom, normals, 2e-4, 0.05, 0.005, mn, vn)
    surv, clone, split = D.decisions(g, s_min, accum, denom, 2e-4, 0.05, 0.005)
    assert counts == (surv.sum(), clone.sum(), split.sum())
    assert clone.sum() > 50 and split.sum() > 50 and (~surv & ~split).sum() > 50
    assert new.n == ref["means"].shape[0]
    nc = surv.sum() + clone.sum()
    for f in flod.GaussianSet.FIELDS:
        a = getattr(new, f).cpu().numpy().astype(np.float64)
        b = ref[f]
        if f in ("means", "s_opt"):
            np.testing.assert_array_equal(a[:nc], b[:nc])           # copies
            np.testing.assert_allclose(a[nc:], b[nc:], rtol=2e-6, atol=2e-6)
        else:
            np.testing.assert_array_equal(a, b)
    for got, want in ((mo, rm), (vo, rv)):
        for f, t in zip(flod.GaussianSet.FIELDS, got):
            np.testing.assert_array_equal(t.cpu().numpy(), want[f])


def test_densify_capacity_and_empty():
    g, accum, denom, normals = _inputs(n=600, seed=44)
    gs = flod.GaussianSet.from_numpy(g, 0.0)
    dev = lambda a: torch.as_tensor(a, device="cuda")
    new, _, _, counts = flod.densify(gs, dev(accum), dev(denom), dev(normals), max_clone_scale=0.05)
    assert new.n == counts[0] + counts[1] + 2 * counts[2]
    # nothing reaches tau: the set is the survivors only (low-opacity ones removed)
    new2, _, _, c2 = flod.densify(gs, dev(accum * 0), dev(denom), dev(normals), max_clone_scale=0.05)
    assert c2[1] == c2[2] == 0 and new2.n == c2[0]
    keep = ~(1 / (1 + np.exp(-g["opacity_logit"])) < 0.005)
    np.testing.assert_array_equal(new2.means.cpu().numpy(), g["means"][keep])
