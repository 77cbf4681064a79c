"""flod_gather and the modes built on it: the predetermined selective set of Sec. 5.2 made
resident on its own, and per-view selection streamed from levels kept in pinned host memory
(the Limitation section), against the oracle."""
import ctypes as C

import numpy as np
import pytest
import torch

from gpu_helpers import assert_image_close
from oracle import raster as R
from oracle import select as S
from paper_2408_12894_gb300 import flod, multiview, selective, synth

pytestmark = pytest.mark.gpu

COUNTS = (2_000, 6_000, 15_000, 30_000, 60_000)
TH = [100.0, 50.0, 25.0, 10.0]


def _levels():
    base = synth.level_scene(counts=COUNTS, radius=20.0, sh_degree=3)
    np_sets = [g for g, _ in synth.stretch_levels(base, 5.0)]
    sets = [flod.GaussianSet.from_numpy(g, 5.0 * s) for g, s in zip(np_sets, synth.LEVEL_SMIN)]
    return sets, np_sets


def _oracle_selective(np_sets, origin, cam):
    ent = S.select([g["means"] for g in np_sets], origin, TH)
    lv, idx = ent >> S.LEVEL_SHIFT, ent & ((1 << S.LEVEL_SHIFT) - 1)
    g = {k: np.concatenate([np_sets[l][k][i:i + 1] for l, i in zip(lv, idx)])
         for k in ("means", "quats", "s_opt", "opacity_logit", "sh")}
    smin = torch.as_tensor(np.array([5.0 * synth.LEVEL_SMIN[l] for l in lv])[:, None])
    img, _, _ = R.render(g, 3, smin, cam, R.Config())
    return img, ent


def test_gather_copies_entries_folds_s_min_and_skips_bad_entries():
    sets, _ = _levels()
    rng = np.random.default_rng(0)
    ent = np.concatenate([(np.uint32(l) << np.uint32(28)) | rng.choice(COUNTS[l], 50).astype(np.uint32)
                          for l in (4, 0, 2)])
    ent = np.concatenate([ent, np.array([(7 << 28) | 1, (1 << 28) | 999_999], np.uint32)])  # bad
    e = torch.as_tensor(ent.view(np.int32), device="cuda")
    cnt = torch.tensor([ent.size], dtype=torch.int32, device="cuda")
    out = flod.gather_set(sets, e, cnt, ent.size + 4, 3, fold_s_min=False)
    fold = flod.gather_set(sets, e, cnt, ent.size + 4, 3, fold_s_min=True)
    torch.cuda.synchronize()
    for k, en in enumerate(ent[:150]):
        l, i = int(en >> 28), int(en & 0x0fffffff)
        for f in flod.GaussianSet.FIELDS:
            assert torch.equal(getattr(out, f)[k], getattr(sets[l], f)[i]), (k, f)
        want = np.log(np.exp(sets[l].s_opt[i].cpu().numpy().astype(np.float64)) + sets[l].s_min)
        np.testing.assert_allclose(fold.s_opt[k].cpu().numpy(), want, rtol=2e-6)
    for f in flod.GaussianSet.FIELDS:   # bad entries and the rows past the count stay zero
        assert not bool(getattr(out, f)[150:].any())


def test_gather_from_pinned_host_memory_and_refuses_pageable():
    sets, _ = _levels()
    s = sets[3]
    host = [getattr(s, f).cpu().pin_memory() for f in flod.GaussianSet.FIELDS]
    g = selective._host_struct(host, s.n, 3, s.s_min)
    cnt = torch.tensor([s.n], dtype=torch.int32, device="cuda")
    out = flod.gather_set([g], None, cnt, s.n, 3, fold_s_min=False)
    torch.cuda.synchronize()
    for f in flod.GaussianSet.FIELDS:
        assert torch.equal(getattr(out, f), getattr(s, f))
    pageable = [getattr(s, f).cpu() for f in flod.GaussianSet.FIELDS]
    gp = selective._host_struct(pageable, s.n, 3, s.s_min)
    with pytest.raises(flod.FlodError):
        flod.gather_set([gp], None, cnt, s.n, 3)


def test_predetermined_set_renders_like_the_oracle():
    sets, np_sets = _levels()
    train_cams = synth.camera_path(width=160, height=90)
    origin = selective.mean_camera_position(train_cams)
    compact, n = selective.predetermined_set(sets, origin, TH)
    cam = synth.camera_path(seed=9, width=160, height=90)[5]
    r = flod.Rasterizer([compact], [flod.view_struct(cam)])
    rgb, T, nc = r.forward()
    torch.cuda.synchronize()
    img, ent = _oracle_selective(np_sets, origin, cam)
    assert n == ent.size and 0 < n < sum(COUNTS)
    assert_image_close(rgb.view(3, 90, 160).cpu().numpy(), img)


def test_streamed_per_view_frames_render_like_the_oracle_and_the_resident_path():
    sets, np_sets = _levels()
    path = synth.camera_path(width=160, height=90)
    most = max(S.select([g["means"] for g in np_sets], c["cam_pos"], TH).size for c in path[:8])
    sl = selective.StreamedLevels(sets, TH, capacity=most + 256)
    sl.size_capacity(path[:8])
    st = multiview.BatchedStep(sets, [multiview.Job(path[0], levels=[0, 1, 2, 3, 4], thresholds=TH)],
                               flod.default_config())
    for fr in (0, 7):
        cam = path[fr]
        rgb, T, nc = sl.frame(cam)
        st.set_camera(0, cam)
        st.size_capacity()
        torch.cuda.synchronize()
        img, ent = _oracle_selective(np_sets, cam["cam_pos"], cam)
        assert int(sl.cnt.item()) == ent.size
        assert_image_close(rgb.view(3, 90, 160).cpu().numpy(), img)
        # the device-resident per-view selective frame (s_min not folded) agrees too
        assert_image_close(rgb.view(3, -1).cpu().numpy(), st.out[0].view(3, -1).cpu().numpy().astype(np.float64))
        assert flod.flod_read_status(sl.rast.ws) == 0
    assert sl.device_bytes() < sum(s.n for s in sets) * 236
