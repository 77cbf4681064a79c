"""GPU level selection (Eq. 6 / Eq. 7) and AdjustScale (Eq. 5) vs the oracle."""
import math

import numpy as np
import pytest
import torch

from oracle import gaussians as OG
from oracle import select as S
from paper_2408_12894_gb300 import flod, synth

pytestmark = pytest.mark.gpu


def _levels(scale=5.0, counts=(3000, 9000, 20000, 41000, 77777)):
    lv = synth.stretch_levels(synth.level_scene(counts=counts, radius=20.0, sh_degree=0), scale)
    s_min = [s * scale for s in synth.LEVEL_SMIN]
    return [flod.GaussianSet.from_numpy(g, s) for (g, _), s in zip(lv, s_min)], lv


def _gpu_select(sets, origin, d_thresh=None, gamma=1.0, focal=0.0, cap=None):
    cap = cap or sum(s.n for s in sets)
    out = torch.zeros(max(cap, 1), dtype=torch.int32, device="cuda")
    cnt = torch.zeros(1, dtype=torch.int32, device="cuda")
    scr = torch.zeros(flod.flod_select_scratch_size(sets), dtype=torch.uint8, device="cuda")
    flod.flod_select_levels(sets, origin, out, cnt, scr, d_thresh=d_thresh, gamma=gamma, focal=focal)
    torch.cuda.synchronize()
    n = int(cnt.item())
    return out[:min(n, cap)].cpu().numpy().view(np.uint32), n


@pytest.mark.parametrize("frame", [0, 9, 31])
def test_select_explicit_thresholds_bit_exact(frame):
    sets, lv = _levels()
    origin = synth.camera_path()[frame]["cam_pos"]
    th = list(synth.SELECTIVE_THRESHOLDS[::-1])         # coarse -> fine: 100, 50, 25, 10
    got, n = _gpu_select(sets, origin, d_thresh=th)
    want = S.select([g["means"] for g, _ in lv], origin, th)
    assert n == want.size
    assert np.array_equal(got, want)
    # against exact arithmetic only threshold-rounding cases may differ
    exact = S.select_exact([g["means"] for g, _ in lv], origin, th)
    assert abs(exact.size - want.size) <= 2


def test_select_eq7_thresholds_bit_exact():
    sets, lv = _levels(scale=1.0)
    focal = np.float32(synth.camera((0, 0, -1), 1920, 1080)["fx"])
    origin = np.array([3.0, 1.0, -35.0], np.float32)
    got, n = _gpu_select(sets, origin, gamma=1.0, focal=float(focal))
    s_min32 = [float(np.float32(s.s_min)) for s in sets]
    th = [float(np.float32(t)) for t in S.d_proj(s_min32, float(focal), 1.0)]
    want = S.select([g["means"] for g, _ in lv], origin, th)
    assert n == want.size and np.array_equal(got, want)


def test_select_partition_when_levels_are_equal():
    g = synth.gaussian_set(3, 50000, k=16, radius=100.0, sh_degree=0)
    sets = [flod.GaussianSet.from_numpy(g, 0.1 * (5 - k)) for k in range(5)]
    got, n = _gpu_select(sets, np.zeros(3, np.float32), d_thresh=[100.0, 50.0, 25.0, 10.0])
    idx = got & ((1 << flod.SEL_SHIFT) - 1)
    assert n == 50000 and np.array_equal(np.sort(idx), np.arange(50000))


def test_select_capacity_clamps_writes():
    sets, lv = _levels()
    origin = synth.camera_path()[0]["cam_pos"]
    th = [100.0, 50.0, 25.0, 10.0]
    want = S.select([g["means"] for g, _ in lv], origin, th)
    got, n = _gpu_select(sets, origin, d_thresh=th, cap=want.size // 3)
    assert n == want.size and np.array_equal(got, want[:want.size // 3])


def test_adjust_scale_eq5():
    rng = np.random.default_rng(0)
    s = rng.normal(-4, 0.8, (100_003, 3)).astype(np.float32)
    sched = list(synth.LEVEL_SMIN)
    for l in range(4):
        t = torch.as_tensor(s, device="cuda")
        flod.flod_adjust_scale(t, sched[l], sched[l + 1])
        got = t.cpu().numpy().astype(np.float64)
        ref = OG.adjust_scale(torch.as_tensor(s.astype(np.float64)), sched[l], sched[l + 1]).numpy()
        np.testing.assert_allclose(got, ref, rtol=0, atol=4e-6)
        before = np.exp(s.astype(np.float64)) + sched[l]
        after = np.exp(got) + sched[l + 1]
        np.testing.assert_allclose(after, before, rtol=2e-6)
