"""Parity at the full benchmark sizes, in the launch configuration bench.py times (16x16
tiles, batch 128, one CTA per tile): sampled pixels against the oracle's per-pixel render
over every Gaussian, sampled Gaussians' gradients against the oracle's exact per-footprint
gradient, and invariants that hold at any size."""
import numpy as np
import pytest
import torch

from gpu_helpers import GRAD_REL, IMG_MAX_ABS, rasterizer
from oracle import gaussians as OG
from oracle import raster as R
from paper_2408_12894_gb300 import flod, synth

pytestmark = pytest.mark.gpu


def _level5():
    """Level 5 of the 5-level scene, with Eq. 5 applied level by level in FP64 (both sides
    then take the same float32 parameters)."""
    levels = synth.level_scene()
    g = dict(levels[-1][0])
    s = torch.as_tensor(g["s_opt"].astype(np.float64))
    for l in range(4):
        n = synth.LEVEL_COUNTS[l]
        s[:n] = OG.adjust_scale(s[:n], synth.LEVEL_SMIN[l], synth.LEVEL_SMIN[l + 1])
    g["s_opt"] = s.numpy().astype(np.float32)
    return g


def _invariants(rast, rgb, T, nc):
    torch.cuda.synchronize()
    assert flod.flod_read_status(rast.ws) == 0
    P = int(rast.pair_count.item())
    U = rast.layout.units
    tt = rast.region("tiles_touched", torch.int32, U).to(torch.int64)
    assert int(tt.sum().item()) == P
    plan = rast.region("plan", torch.int32, 64)
    fin = int(plan[63].item())
    tiles = rast.region("keys", torch.int32, rast.pair_capacity, fin)[:P].to(torch.int64)
    vals = rast.region("vals", torch.int32, rast.pair_capacity, fin)[:P].to(torch.int64)
    assert bool((tiles[1:] >= tiles[:-1]).all())
    same = tiles[1:] == tiles[:-1]
    depth = rast.region("depth", torch.float32, U)[vals]
    assert bool((depth[1:][same] >= depth[:-1][same]).all())
    rg = rast.region("ranges", torch.int32, 2 * rast.layout.tiles).view(-1, 2).to(torch.int64)
    nz = rg[rg[:, 1] > rg[:, 0]]
    assert int(nz[0, 0]) == 0 and int(nz[-1, 1]) == P and bool((nz[1:, 0] == nz[:-1, 1]).all())
    assert float(T.min()) >= float(np.float32(1e-4)) and float(T.max()) <= 1.0
    assert bool(torch.isfinite(rgb).all())


def _pixels_vs_oracle(g, s_min, cam, img, n=48, seed=0):
    rng = np.random.default_rng(seed)
    pix = np.stack([rng.integers(0, cam["width"], n), rng.integers(0, cam["height"], n)], 1)
    with torch.no_grad():
        pre = R.preprocess(R.params(g), g["sh_degree"], s_min, cam, R.Config())
        errs = []
        for k in range(0, n, 4):
            col, _ = R.render_brute(pre, cam, R.Config(), pixels=pix[k:k + 4])
            want = col.numpy()
            got = img[:, pix[k:k + 4, 1], pix[k:k + 4, 0]].T
            errs.append(np.abs(got - want).max(axis=1))
    errs = np.concatenate(errs)
    assert (errs <= IMG_MAX_ABS).mean() >= 1 - 1.5 / n, errs
    assert errs.mean() <= 2e-5, errs.mean()
    return pre


def _sampled_grad_check(g, s_min, cam, dL_img, got, pre, sample):
    ref = R.sampled_gradients(g, g["sh_degree"], s_min, cam, R.Config(), dL_img, sample, pre=pre)
    for k in ref:
        a = got[k][sample].reshape(len(sample), -1).astype(np.float64)
        b = ref[k].reshape(len(sample), -1)
        scale = np.abs(b).max() + 1e-30
        for i in range(len(sample)):
            err = np.linalg.norm(a[i] - b[i])
            assert err <= GRAD_REL * np.linalg.norm(b[i]) + 1e-5 * scale, (k, sample[i], err)


def test_level5_3M_1080p():
    g = _level5()
    cam = synth.level_camera()
    s_min = synth.LEVEL_SMIN[-1]
    rast = rasterizer([g], [cam], [s_min])
    for f in flod.GaussianSet.FIELDS:
        getattr(rast.sets[0], f).requires_grad_(True)
    rgb, T, nc = flod.rasterize(rast)
    dL = synth.upstream_gradient(11, [cam])
    (rgb * torch.as_tensor(dL, device="cuda")).sum().backward()
    _invariants(rast, rgb, T, nc)
    img = rgb.detach().view(3, 1080, 1920).cpu().numpy()
    pre = _pixels_vs_oracle(g, s_min, cam, img)
    got = {f: getattr(rast.sets[0], f).grad.cpu().numpy() for f in flod.GaussianSet.FIELDS}
    vis = np.nonzero(pre["tiles_touched"] > 0)[0]
    rng = np.random.default_rng(1)
    # a few of each size class: carried level-1 Gaussians (largest) to fresh level-5 ones
    sample = np.concatenate([rng.choice(vis[vis < 20_000], 3), rng.choice(vis[vis >= 1_000_000], 5)])
    _sampled_grad_check(g, s_min, cam, dL.reshape(3, 1080, 1920), got, pre, sample)


def test_multiview_500k_720p_eight_views():
    g, cams = synth.scene_multiview_training()
    rast = rasterizer([g], cams, [0.0])
    for f in flod.GaussianSet.FIELDS:
        getattr(rast.sets[0], f).requires_grad_(True)
    rgb, T, nc = flod.rasterize(rast)
    dL = synth.upstream_gradient(11, cams)
    (rgb * torch.as_tensor(dL, device="cuda")).sum().backward()
    _invariants(rast, rgb, T, nc)
    imgs = flod.image_views(rgb.detach(), rast.views, 3)
    got = {f: getattr(rast.sets[0], f).grad.cpu().numpy() for f in flod.GaussianSet.FIELDS}
    rng = np.random.default_rng(2)
    pres = []
    for v in (0, 5):
        pres.append(_pixels_vs_oracle(g, 0.0, cams[v], imgs[v].cpu().numpy(), n=24, seed=v))
    # gradients sum over all eight views: per-view exact footprint gradients, summed
    vis = np.nonzero(pres[0]["tiles_touched"] > 0)[0]
    sample = rng.choice(vis, 6, replace=False)
    ref = None
    off = 0
    for c in cams:
        n = 3 * c["width"] * c["height"]
        r = R.sampled_gradients(g, 3, 0.0, c, R.Config(), dL[off:off + n].reshape(3, c["height"], c["width"]), sample)
        off += n
        ref = r if ref is None else {k: ref[k] + r[k] for k in ref}
    for k in ref:
        a = got[k][sample].reshape(len(sample), -1).astype(np.float64)
        b = ref[k].reshape(len(sample), -1)
        scale = np.abs(b).max() + 1e-30
        for i in range(len(sample)):
            assert np.linalg.norm(a[i] - b[i]) <= GRAD_REL * np.linalg.norm(b[i]) + 1e-5 * scale, (k, i)
