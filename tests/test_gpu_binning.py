"""GPU binning + radix sort + tile ranges, bit-exact against the oracle.

The oracle's own preprocess (rounded to float32, with the rectangle decided in float32) is
written into the workspace; the GPU then runs flod_bin_sort alone. Keys, values, the pair
count and every tile range must match the oracle's stable sort of the same pairs exactly."""
import numpy as np
import pytest
import torch

from gpu_helpers import (clear_units, inject_units, oracle_cfg, oracle_pre, oracle_units_f32,
                         random_units_f32, rasterizer, sorted_pairs)
from oracle import projection as OP
from oracle import raster as R
from paper_2408_12894_gb300 import flod, synth

pytestmark = pytest.mark.gpu


def _oracle_lists(rast, fs, cams, ocfg):
    keys, vals = [], []
    for i, (f, cam) in enumerate(zip(fs, cams)):
        tx = -(-cam["width"] // ocfg.tile_w)
        ty = -(-cam["height"] // ocfg.tile_h)
        segs = tuple(np.asarray(a)[f["valid"][np.asarray(f["segments"][0])]] for a in f["segments"])
        k, v = R.bin_segments(segs, f["depth"], tx, tx * ty, tile_offset=rast.tile_off[i],
                              unit_offset=rast.unit_off[i])
        keys.append(k)
        vals.append(v)
    k, v = R.sort_pairs(np.concatenate(keys), np.concatenate(vals))
    return k, v, R.tile_ranges(k, rast.layout.tiles)


def _run(rast, fs, cams, phased=False):
    ocfg = oracle_cfg(rast.cfg)
    clear_units(rast)
    for i, f in enumerate(fs):
        inject_units(rast, i, f)
    if phased:   # the four parts of flod_bin_sort_phase, in order
        for ph in (flod.BIN_PHASE_DEPTH, flod.BIN_PHASE_EMIT, flod.BIN_PHASE_TILES,
                   flod.BIN_PHASE_RANGES):
            rast.bin_sort_phase(ph)
    else:
        rast.bin_sort()
    keys, vals, ranges, P, status = sorted_pairs(rast)
    k, v, rg = _oracle_lists(rast, fs, cams, ocfg)
    assert status == 0, status
    assert P == k.size
    assert np.array_equal(keys, k)
    assert np.array_equal(vals, v)
    assert np.array_equal(ranges, rg)
    return P


def _scene_units(g, s_min, cams, cfg):
    ocfg = oracle_cfg(cfg)
    return [oracle_units_f32(oracle_pre(g, s_min, c, ocfg), c, ocfg) for c in cams]


@pytest.mark.parametrize("tile,rule", [((16, 16), 2), ((8, 8), 2), ((32, 8), 2), ((16, 16), 0)])
def test_binning_single_view(tile, rule):
    g, cams = synth.scene_single_forward()
    cfg = flod.default_config(tile_w=tile[0], tile_h=tile[1], extent_rule=rule)
    rast = rasterizer([g], cams, [0.0], cfg=cfg)
    P = _run(rast, _scene_units(g, 0.0, cams, cfg), cams)
    assert P > 0


@pytest.mark.parametrize("phased", [False, True])
def test_binning_batched_views_ragged_sizes(phased):
    g = synth.gaussian_set(2, 5003, k=16, radius=5.0, sh_degree=0, s_mean=-2.5)
    cams = [synth.camera((15.0 * np.cos(a), 1.0, 15.0 * np.sin(a)), w, h)
            for a, (w, h) in zip((0.0, 1.3, 2.9, 4.4), ((333, 201), (128, 128), (97, 250), (640, 360)))]
    cfg = flod.default_config(persistent=1 if phased else 0)
    rast = rasterizer([g], cams, [0.0], cfg=cfg)
    _run(rast, _scene_units(g, 0.0, cams, cfg), cams, phased)


@pytest.mark.parametrize("rule", [2, 0])
def test_binning_ties_in_depth_keep_unit_order(rule):
    # 3000 Gaussians on 7 distinct depths: the stable sort must keep unit order inside a tie
    rng = np.random.default_rng(0)
    n = 3000
    cam = synth.camera((0.0, 0.0, -3.0), 256, 256)
    cfg = flod.default_config(extent_rule=rule)
    depth = rng.choice(np.float32([1.0, 2.0, 2.5, 3.0, 7.25, 11.0, 100.0]), n)
    f = random_units_f32(rng, n, cam, oracle_cfg(cfg), r_scale=6.0, depth=depth)
    g = synth.gaussian_set(0, n, sh_degree=0)
    rast = rasterizer([g], [cam], [0.0], cfg=cfg)
    _run(rast, [f], [cam])


def test_binning_many_partitions_and_passes():
    # millions of pairs over 4 views of 1080p: > 1000 sort partitions in both stages
    rng = np.random.default_rng(1)
    n = 400_000
    cams = [synth.camera((0.0, 0.0, -40.0 - i), 1920, 1080) for i in range(4)]
    cfg = flod.default_config()
    fs = [random_units_f32(rng, n, c, oracle_cfg(cfg), r_scale=5.0) for c in cams]
    g = synth.gaussian_set(0, n, sh_degree=0)
    rast = rasterizer([g], cams, [0.0], cfg=cfg, pair_capacity=12_000_000)
    P = _run(rast, fs, cams)
    assert P > 4_000_000


def test_binning_huge_splats_span_many_slices():
    # a few hundred splats that each cover hundreds of tiles, over 8x8 tiles
    rng = np.random.default_rng(2)
    n = 600
    cam = synth.camera((0.0, 0.0, -3.0), 1280, 720)
    cfg = flod.default_config(tile_w=8, tile_h=8)
    f = random_units_f32(rng, n, cam, oracle_cfg(cfg), r_scale=60.0, aniso=8.0)
    g = synth.gaussian_set(0, n, sh_degree=0)
    rast = rasterizer([g], [cam], [0.0], cfg=cfg, pair_capacity=4_000_000)
    P = _run(rast, [f], [cam])
    assert P > 100_000


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
    assert need > 2048
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
