"""GPU binning + radix sort + tile ranges, bit-exact against the oracle.

The oracle's own preprocess (rounded to float32, with the rectangle decided in float32) is
written into the workspace; the GPU then runs flod_bin_sort alone. Keys, values, the pair
count and every tile range must match the oracle's stable sort of the same pairs exactly."""
import numpy as np
import pytest
import torch

from gpu_helpers import (clear_units, inject_units, oracle_cfg, oracle_pre, oracle_units_f32,
                         rasterizer, sorted_pairs)
from oracle import projection as OP
from oracle import raster as R
from paper_2408_12894_gb300 import flod, synth

pytestmark = pytest.mark.gpu


def _oracle_lists(rast, fs, cams, ocfg):
    keys, vals = [], []
    for i, (f, cam) in enumerate(zip(fs, cams)):
        tx = -(-cam["width"] // ocfg.tile_w)
        ty = -(-cam["height"] // ocfg.tile_h)
        tt = np.where(f["valid"], f["tiles_touched"], 0)
        k, v = R.bin_pairs(f["tile_rect"], tt, f["depth"], tx, tx * ty,
                           tile_offset=rast.tile_off[i], unit_offset=rast.unit_off[i])
        keys.append(k)
        vals.append(v)
    k, v = R.sort_pairs(np.concatenate(keys), np.concatenate(vals))
    return k, v, R.tile_ranges(k, rast.layout.tiles)


def _run(rast, fs, cams):
    ocfg = oracle_cfg(rast.cfg)
    clear_units(rast)
    for i, f in enumerate(fs):
        inject_units(rast, i, f)
    rast.bin_sort()
    keys, vals, ranges, P, status = sorted_pairs(rast)
    k, v, rg = _oracle_lists(rast, fs, cams, ocfg)
    assert status == 0
    assert P == k.size
    assert np.array_equal(keys, k)
    assert np.array_equal(vals, v)
    assert np.array_equal(ranges, rg)
    return P


def _scene_units(g, s_min, cams, cfg):
    ocfg = oracle_cfg(cfg)
    return [oracle_units_f32(oracle_pre(g, s_min, c, ocfg), c, ocfg) for c in cams]


@pytest.mark.parametrize("tile", [(16, 16), (8, 8), (32, 8)])
def test_binning_single_view(tile):
    g, cams = synth.scene_single_forward()
    cfg = flod.default_config(tile_w=tile[0], tile_h=tile[1])
    rast = rasterizer([g], cams, [0.0], cfg=cfg)
    P = _run(rast, _scene_units(g, 0.0, cams, cfg), cams)
    assert P > 0


def test_binning_batched_views_ragged_sizes():
    g = synth.gaussian_set(2, 5003, k=16, radius=5.0, sh_degree=0, s_mean=-2.5)
    cams = [synth.camera((15.0 * np.cos(a), 1.0, 15.0 * np.sin(a)), w, h)
            for a, (w, h) in zip((0.0, 1.3, 2.9, 4.4), ((333, 201), (128, 128), (97, 250), (640, 360)))]
    cfg = flod.default_config()
    rast = rasterizer([g], cams, [0.0], cfg=cfg)
    _run(rast, _scene_units(g, 0.0, cams, cfg), cams)


def test_binning_ties_in_depth_keep_unit_order():
    # 3000 Gaussians on 7 distinct depths: the stable sort must keep unit order inside a tie
    rng = np.random.default_rng(0)
    n = 3000
    cam = synth.camera((0.0, 0.0, -3.0), 256, 256)
    f = {"u": rng.uniform(-20, 280, n).astype(np.float32),
         "v": rng.uniform(-20, 280, n).astype(np.float32),
         "r": rng.uniform(0.5, 40, n).astype(np.float32),
         "depth": rng.choice(np.float32([1.0, 2.0, 2.5, 3.0, 7.25, 11.0, 100.0]), n),
         "valid": rng.random(n) > 0.1}
    px = OP.pixel_rect_f32(f["u"], f["v"], f["r"], 256, 256)
    tr = OP.tile_rect(px, 16, 16, f["valid"])
    f["tile_rect"], f["tiles_touched"] = tr[:4], tr[4]
    f["valid"] = f["valid"] & (tr[4] > 0)
    g = synth.gaussian_set(0, n, sh_degree=0)
    rast = rasterizer([g], [cam], [0.0])
    _run(rast, [f], [cam])


def test_binning_many_partitions_and_passes():
    # about 6M pairs over 4 views of 1080p: > 1400 sort partitions, 6 digit passes
    rng = np.random.default_rng(1)
    n = 400_000
    cams = [synth.camera((0.0, 0.0, -40.0 - i), 1920, 1080) for i in range(4)]
    fs = []
    for c in cams:
        f = {"u": rng.uniform(-50, 1970, n).astype(np.float32),
             "v": rng.uniform(-50, 1130, n).astype(np.float32),
             "r": rng.gamma(2.0, 4.0, n).astype(np.float32),
             "depth": rng.uniform(20, 60, n).astype(np.float32),
             "valid": np.ones(n, bool)}
        px = OP.pixel_rect_f32(f["u"], f["v"], f["r"], 1920, 1080)
        tr = OP.tile_rect(px, 16, 16, f["valid"])
        f["tile_rect"], f["tiles_touched"] = tr[:4], tr[4]
        f["valid"] = tr[4] > 0
        fs.append(f)
    g = synth.gaussian_set(0, n, sh_degree=0)
    rast = rasterizer([g], cams, [0.0], pair_capacity=12_000_000)
    P = _run(rast, fs, cams)
    assert P > 4_000_000


def test_binning_empty():
    g, cams = synth.scene_single_forward(n=500)
    rast = rasterizer([g], cams, [0.0])
    clear_units(rast)
    rast.bin_sort()
    keys, vals, ranges, P, status = sorted_pairs(rast)
    assert P == 0 and keys.size == 0 and status == 0
    assert np.all(ranges == 0)


def test_capacity_overflow_is_reported_not_faulted():
    g, cams = synth.scene_single_forward()
    cfg = flod.default_config()
    fs = _scene_units(g, 0.0, cams, cfg)
    need = int(np.where(fs[0]["valid"], fs[0]["tiles_touched"], 0).sum())
    rast = rasterizer([g], cams, [0.0], cfg=cfg, pair_capacity=need // 2)
    clear_units(rast)
    inject_units(rast, 0, fs[0])
    rast.bin_sort()
    torch.cuda.synchronize()
    assert int(rast.pair_count.item()) == need
    assert flod.flod_read_status(rast.ws) & flod.DEV_CAPACITY
    # the sorted prefix that fitted is still ordered
    keys, _, _, _, _ = sorted_pairs(rast)
    assert keys.size == need // 2 and np.all(keys[1:] >= keys[:-1])
    assert not rast.ensure_capacity() and rast.pair_capacity >= need
