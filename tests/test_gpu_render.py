"""GPU blending vs the FP64 oracle: stage-wise (oracle-made splats and sorted lists written
into the workspace, GPU render only) and end to end (each side from its own preprocess)."""
import numpy as np
import pytest
import torch

from gpu_helpers import (assert_image_close, clear_units, image_compare, inject_units,
                         oracle_cfg, oracle_pre, oracle_units_f32, rasterizer)
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
    return (rgb.view(3, H, W).cpu().numpy(), T.view(H, W).cpu().numpy(),
            nc.view(H, W).cpu().numpy(), img, tf, last)


@pytest.mark.parametrize("tile,batch", [((16, 16), 256), ((8, 8), 32), ((32, 8), 64), ((16, 16), 128)])
def test_render_stage_matches_oracle(tile, batch):
    g, cams = synth.scene_single_forward()
    cfg = flod.default_config(tile_w=tile[0], tile_h=tile[1], batch=batch)
    gi, gT, gnc, oi, oT, onc = _stage_render(g, cams[0], cfg)
    assert_image_close(gi, oi)
    np.testing.assert_allclose(gT, oT, atol=2e-4)
    assert (gnc == onc).mean() >= 0.999


def test_render_stage_dense_sh3_background():
    g = synth.gaussian_set(4, 20000, k=8, radius=1.0, sh_degree=3, s_mean=-3.0)
    cam = synth.camera((0.4, -0.3, -3.0), 200, 150)
    cfg = flod.default_config(bg=(0.2, 0.5, 0.9))
    gi, gT, gnc, oi, oT, onc = _stage_render(g, cam, cfg)
    assert_image_close(gi, oi)
    assert (gnc == onc).mean() >= 0.999
    assert (oT < 1e-3).mean() > 0.05          # early termination is exercised


def test_render_end_to_end_single_forward_scene():
    g, cams = synth.scene_single_forward()
    rast = rasterizer([g], cams, [0.0])
    rgb, T, nc = rast.forward()
    torch.cuda.synchronize()
    img, tf, _ = R.render(g, 0, 0.0, cams[0], R.Config())
    assert_image_close(rgb.view(3, 128, 128).cpu().numpy(), img)
    np.testing.assert_allclose(T.view(128, 128).cpu().numpy(), tf, atol=2e-3)
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
