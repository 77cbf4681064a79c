"""The allocation-free selection entry point (flod_select_levels_noalloc).

It exists for callers that cannot allocate device memory (an engine plugin whose host owns
every device allocation, a real-time loop that must not take cudaMalloc's synchronisation).
It must return exactly what flod_select_levels returns with caller scratch, call after call,
although its scratch is one fixed array shared by every call.

This file sorts last on purpose, so that a failure here comes after every other test has
run; it also passes when run alone in a fresh process."""
import ctypes as C

import numpy as np
import pytest
import torch

from paper_2408_12894_gb300 import flod, synth

pytestmark = pytest.mark.gpu


def _levels():
    lv = synth.stretch_levels(synth.level_scene(counts=(3000, 9000, 20000, 41000, 77777),
                                                radius=20.0, sh_degree=0), 5.0)
    return [flod.GaussianSet.from_numpy(g, 5.0 * s) for (g, _), s in zip(lv, synth.LEVEL_SMIN)]


def _with_scratch(sets, origin, th):
    cap = sum(s.n for s in sets)
    out = torch.zeros(cap, dtype=torch.int32, device="cuda")
    cnt = torch.zeros(1, dtype=torch.int32, device="cuda")
    scr = torch.zeros(flod.flod_select_scratch_size(sets), dtype=torch.uint8, device="cuda")
    flod.flod_select_levels(sets, origin, out, cnt, scr, d_thresh=th)
    torch.cuda.synchronize()
    n = int(cnt.item())
    return out[:n].cpu().numpy(), n


def _no_alloc(sets, origin, th):
    cap = sum(s.n for s in sets)
    out = torch.full((cap,), -1, dtype=torch.int32, device="cuda")
    cnt = torch.zeros(1, dtype=torch.int32, device="cuda")
    flod.flod_select_levels_noalloc(sets, origin, out, cnt, d_thresh=th)
    torch.cuda.synchronize()
    n = int(cnt.item())
    return out[:n].cpu().numpy(), n


def test_no_alloc_selection_matches_the_scratch_entry_point_twice():
    sets = _levels()
    th = [100.0, 50.0, 25.0, 10.0]
    path = synth.camera_path()
    # two calls in a row with different cameras: the second must not see the first's scratch
    for frame in (0, 31):
        origin = path[frame]["cam_pos"]
        want, n_want = _with_scratch(sets, origin, th)
        got, n_got = _no_alloc(sets, origin, th)
        assert n_got == n_want and n_want > 0
        assert np.array_equal(got, want)


def test_no_alloc_selection_eq7_thresholds():
    sets = _levels()
    origin = np.array([10.0, 2.0, -60.0], np.float32)
    focal = float(np.float32(synth.camera((0, 0, -1), 1920, 1080)["fx"]))
    cap = sum(s.n for s in sets)
    ref = torch.zeros(cap, dtype=torch.int32, device="cuda")
    rc = torch.zeros(1, dtype=torch.int32, device="cuda")
    scr = torch.zeros(flod.flod_select_scratch_size(sets), dtype=torch.uint8, device="cuda")
    flod.flod_select_levels(sets, origin, ref, rc, scr, gamma=1.0, focal=focal)
    out = torch.zeros(cap, dtype=torch.int32, device="cuda")
    oc = torch.zeros(1, dtype=torch.int32, device="cuda")
    flod.flod_select_levels_noalloc(sets, origin, out, oc, gamma=1.0, focal=focal)
    torch.cuda.synchronize()
    n = int(rc.item())
    assert int(oc.item()) == n
    assert torch.equal(out[:n], ref[:n])


def test_no_alloc_selection_rejects_inputs_beyond_its_scratch():
    # described sizes only: the call is refused on the host, no device memory is touched
    means = torch.zeros(3, dtype=torch.float32, device="cuda")
    g = flod.Gaussians()
    g.means = means.data_ptr()
    g.n, g.sh_degree, g.s_min = (1 << 25) + 1, 0, 0.0
    arr = (flod.Gaussians * 1)(g)
    org = (C.c_float * 3)(0.0, 0.0, 0.0)
    out = torch.zeros(1, dtype=torch.int32, device="cuda")
    rc = flod.lib().flod_select_levels_noalloc(arr, 1, None, 1.0, 100.0, org, out.data_ptr(), 1,
                                               out.data_ptr(), None)
    assert rc == 1   # FLOD_ERR_INVALID_ARG
