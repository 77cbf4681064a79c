"""GPU blending vs the FP64 oracle: stage-wise (oracle-made splats and sorted lists written
into the workspace, GPU render only) and end to end (each side from its own preprocess)."""
import numpy as np
import pytest
import torch

from gpu_helpers import (DECISION_MARGIN, IMG_FRAC, IMG_MAX_ABS, assert_image_close,
                         assert_tiles_close, blend_decision_margin, clear_units, gpu_view_lists,
                         inject_units, oracle_cfg, oracle_pre, oracle_units_f32, rasterizer)
from oracle import raster as R
from paper_2408_12894_gb300 import flod, synth

pytestmark = pytest.mark.gpu


def _inject_lists(rast, keys, vals, ranges):
    P = keys.size
    dev = rast.ws.device
    rast.region("plan", torch.int32, 64)[63] = 0
    rast.region("vals", torch.int32, rast.pair_capacity, 0)[:P] = torch.as_tensor(vals.view(np.int32), device=dev)
    rast.region("ranges", torch.int32, 2 * rast.layout.tiles).view(-1, 2)[:] = \
        torch.as_tensor(ranges.astype(np.int32), device=dev)


def _stage_render(g, cam, cfg, s_min=0.0):
    """Render oracle float32 splats on the GPU; returns (gpu img, T, nc, oracle img, T, nc)."""
    ocfg = oracle_cfg(cfg)
    pre = oracle_pre(g, s_min, cam, ocfg)
    f = oracle_units_f32(pre, cam, ocfg)
    tx = -(-cam["width"] // cfg.tile_w)
    ty = -(-cam["height"] // cfg.tile_h)
    segs = tuple(np.asarray(a)[f["valid"][np.asarray(f["segments"][0])]] for a in f["segments"])
    k, v = R.bin_segments(segs, f["depth"], tx, tx * ty)
    k, v = R.sort_pairs(k, v)
    rg = R.tile_ranges(k, tx * ty)
    rast = rasterizer([g], [cam], [s_min], cfg=cfg, pair_capacity=max(k.size, 1024))
    clear_units(rast)
    inject_units(rast, 0, f)
    _inject_lists(rast, k, v, rg)
    rgb, T, nc = rast.new_outputs()
    rast.render_fwd(rgb, T, nc)
    torch.cuda.synchronize()
    # oracle blend of exactly the same float32 splats, in float64
    o_pre = {"mean2d": torch.as_tensor(np.stack([f["u"], f["v"]], 1).astype(np.float64)),
             "conic": torch.as_tensor(f["conic"].astype(np.float64)),
             "opacity": torch.as_tensor(f["opacity"].astype(np.float64)),
             "rgb": torch.as_tensor(f["rgb"].astype(np.float64))}
    img, tf, last = R.render_tiled(o_pre, cam, ocfg, lists=(k, v, rg, tx, ty))
    H, W = cam["height"], cam["width"]
    clear = _unambiguous(o_pre, (k, v, rg, tx, ty), cam, ocfg)
    return (rgb.view(3, H, W).cpu().numpy(), T.view(H, W).cpu().numpy(),
            nc.view(H, W).cpu().numpy(), img, tf, last, clear)


def _unambiguous(pre, lists, cam, ocfg):
    """[H, W] mask of the pixels whose blending decisions lie clear of their thresholds
    (n_contrib then has one right answer in any precision)."""
    keys, vals, ranges, tx, ty = lists
    H, W = cam["height"], cam["width"]
    clear = np.ones((H, W), dtype=bool)
    for t in range(tx * ty):
        x0, y0, x1, y1 = R.tile_pixels(t, tx, cam, ocfg)
        s, e = ranges[t]
        g = torch.as_tensor(vals[s:e].astype(np.int64))
        gx, gy = np.meshgrid(np.arange(x0, x1), np.arange(y0, y1))
        pix = torch.as_tensor(np.stack([gx.ravel() + 0.5, gy.ravel() + 0.5], 1).astype(np.float64))
        m = blend_decision_margin(pix, pre["mean2d"].detach()[g], pre["conic"].detach()[g],
                                  pre["opacity"].detach()[g])
        clear[y0:y1, x0:x1] = (m > DECISION_MARGIN).reshape(y1 - y0, x1 - x0)
    return clear


def _assert_nc(gnc, onc, clear):
    assert (~clear).mean() < 0.05, f"{(~clear).mean():.4f} of pixels ambiguous"
    bad = clear & (gnc != onc)
    assert not bad.any(), f"n_contrib differs on {int(bad.sum())} unambiguous pixels"


@pytest.mark.parametrize("tile,batch", [((16, 16), 256), ((8, 8), 32), ((32, 8), 64), ((16, 16), 128)])
def test_render_stage_matches_oracle(tile, batch):
    g, cams = synth.scene_single_forward()
    cfg = flod.default_config(tile_w=tile[0], tile_h=tile[1], batch=batch)
    gi, gT, gnc, oi, oT, onc, clear = _stage_render(g, cams[0], cfg)
    assert_image_close(gi, oi)
    np.testing.assert_allclose(gT, oT, atol=2e-4)
    _assert_nc(gnc, onc, clear)


def test_render_stage_dense_sh3_background():
    g = synth.gaussian_set(4, 20000, k=8, radius=1.0, sh_degree=3, s_mean=-3.0)
    cam = synth.camera((0.4, -0.3, -3.0), 200, 150)
    cfg = flod.default_config(bg=(0.2, 0.5, 0.9))
    gi, gT, gnc, oi, oT, onc, clear = _stage_render(g, cam, cfg)
    assert_image_close(gi, oi)
    np.testing.assert_allclose(gT, oT, atol=2e-4)
    _assert_nc(gnc, onc, clear)
    assert (oT < 1e-3).mean() > 0.05          # early termination is exercised


def test_render_end_to_end_single_forward_scene():
    g, cams = synth.scene_single_forward()
    rast = rasterizer([g], cams, [0.0])
    rgb, T, nc = rast.forward()
    torch.cuda.synchronize()
    ocfg = R.Config()
    pre = oracle_pre(g, 0.0, cams[0], ocfg)
    lists = R.tile_lists(pre, cams[0], ocfg)
    img, tf, last = R.render_tiled(pre, cams[0], ocfg, lists=lists)
    assert_image_close(rgb.view(3, 128, 128).cpu().numpy(), img)
    # T like an image channel; n_contrib names a position in each side's own tile list (the
    # lists may differ by Gaussians at the edge of their tile sets): the Gaussian it names is
    # compared, wherever the decisions are unambiguous
    tiles = list(range(lists[3] * lists[4]))
    ref = R.render_tiles(pre, cams[0], ocfg, lists, tiles)
    n = assert_tiles_close(rgb.view(3, 128, 128).cpu().numpy(), T.view(128, 128).cpu().numpy(),
                           nc.view(128, 128).cpu().numpy(), ref, pre, lists, cams[0], ocfg,
                           "single forward", gpu_view_lists(rast, 0))
    assert n == 128 * 128
    assert flod.flod_read_status(rast.ws) == 0


def test_render_end_to_end_batched_views():
    g = synth.gaussian_set(5, 30000, k=16, radius=5.0, sh_degree=3)
    cams = [synth.camera((15.0 * np.cos(a), 1.5, 15.0 * np.sin(a)), w, h)
            for a, (w, h) in zip((0.2, 2.0, 4.1), ((160, 90), (96, 96), (123, 77)))]
    rast = rasterizer([g], cams, [0.02])
    rgb, T, nc = rast.forward()
    torch.cuda.synchronize()
    imgs = flod.image_views(rgb, rast.views, 3)
    for i, c in enumerate(cams):
        img, tf, _ = R.render(g, 3, 0.02, c, R.Config())
        assert_image_close(imgs[i].cpu().numpy(), img)


def test_render_empty_view_is_background():
    g, cams = synth.scene_single_forward(n=100)
    g["means"][:, 2] = -10.0
    rast = rasterizer([g], cams, [0.0], cfg=flod.default_config(bg=(0.1, 0.2, 0.3)))
    rgb, T, nc = rast.forward()
    torch.cuda.synchronize()
    assert torch.all(T == 1) and torch.all(nc == 0)
    im = rgb.view(3, -1)
    for c, want in enumerate((0.1, 0.2, 0.3)):
        assert torch.allclose(im[c], torch.full_like(im[c], want))
