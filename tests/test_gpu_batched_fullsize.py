"""Parity of the 64-view batch that the benchmark times, at full size: mixed 640x480 ..
3840x2160 views over the five levels of the 5-level scene (20k .. 3M Gaussians) and the
per-view selective mix of the stretched scene, one autotuned persistent launch per stage,
replayed from a captured CUDA graph.

Three views are compared with the oracle: a 3840x2160 view of level 1, a 1920x1080 view of
level 5 and a 3840x2160 selective view (Eq. 6 selection from the camera, each Gaussian with
its own level's s_min). Images on sampled whole tiles; gradients of sampled Gaussians, with
the upstream gradient of every other view set to zero (the gradient is linear in it, so the
batch then returns that view's gradient alone, through the same launches)."""
import numpy as np
import pytest
import torch

from gpu_helpers import (assert_grad_close, assert_nonvacuous, assert_tiles_close,
                         blended_gaussians, gpu_view_lists, oracle_cfg, tile_sample)
from oracle import gaussians as OG
from oracle import raster as R
from oracle import select as S
from paper_2408_12894_gb300 import flod, multiview, synth

pytestmark = pytest.mark.gpu

TH = list(synth.SELECTIVE_THRESHOLDS[::-1])
VIEW_L1_4K, VIEW_L5_1080P, VIEW_SEL_4K = 4, 16, 1


def _chain(g, li, smin):
    """Eq. 5 in FP64 for the Gaussians carried into level li (level by level)."""
    g = dict(g)
    s = torch.as_tensor(g["s_opt"].astype(np.float64))
    for l in range(li):
        n = synth.LEVEL_COUNTS[l]
        s[:n] = OG.adjust_scale(s[:n], smin[l], smin[l + 1])
    g["s_opt"] = s.numpy().astype(np.float32)
    return g


@pytest.fixture(scope="module")
def c4():
    levels = synth.level_scene()
    stretched = synth.stretch_levels(levels, 5.0)
    smin5 = [5.0 * s for s in synth.LEVEL_SMIN]
    np_sel = [_chain(g, li, smin5) for li, (g, _) in enumerate(stretched)]
    np_lvl = [_chain(g, li, synth.LEVEL_SMIN) for li, (g, _) in enumerate(levels)]
    sets = ([flod.GaussianSet.from_numpy(g, s) for g, s in zip(np_sel, smin5)] +
            [flod.GaussianSet.from_numpy(g, s) for g, s in zip(np_lvl, synth.LEVEL_SMIN)])
    cams, job_ids = synth.batched_jobs(n_cams=64)
    jobs = [multiview.Job(c, levels=[0, 1, 2, 3, 4], thresholds=TH) if j == 5
            else multiview.Job(c, set_index=5 + j) for c, j in zip(cams, job_ids)]
    assert job_ids[VIEW_L1_4K] == 0 and cams[VIEW_L1_4K]["width"] == 3840
    assert job_ids[VIEW_L5_1080P] == 4 and cams[VIEW_L5_1080P]["width"] == 1920
    assert job_ids[VIEW_SEL_4K] == 5 and cams[VIEW_SEL_4K]["width"] == 3840
    dL_np = synth.upstream_gradient(11, cams)
    dL = torch.as_tensor(dL_np, device="cuda")
    cfg, _ = multiview.autotune(sets, jobs, backward=True, dL=dL, steps=2)
    st = multiview.BatchedStep(sets, jobs, cfg, backward=True, dL=dL)
    st.size_capacity()
    st.capture()
    st.replay()
    torch.cuda.synchronize()
    assert flod.flod_read_status(st.rast.ws) == 0
    offs = np.cumsum([0] + [c["width"] * c["height"] for c in cams])
    return {"sets": sets, "np_sel": np_sel, "np_lvl": np_lvl, "smin5": smin5, "cams": cams,
            "jobs": jobs, "dL_np": dL_np, "dL": dL, "cfg": cfg, "st": st, "offs": offs}


def _outputs(c, v):
    st, o = c["st"], c["offs"]
    cam = c["cams"][v]
    H, W = cam["height"], cam["width"]
    rgb = st.out[0][3 * o[v]:3 * o[v + 1]].view(3, H, W).cpu().numpy()
    T = st.out[1][o[v]:o[v + 1]].view(H, W).cpu().numpy()
    nc = st.out[2][o[v]:o[v + 1]].view(H, W).cpu().numpy()
    return rgb, T, nc


def _view_grads(c, v):
    """Replay the captured batch with the upstream gradient of view v only."""
    o, dL = c["offs"], c["dL"]
    full = torch.as_tensor(c["dL_np"], device="cuda")
    dL.zero_()
    dL[3 * o[v]:3 * o[v + 1]] = full[3 * o[v]:3 * o[v + 1]]
    c["st"].replay()
    torch.cuda.synchronize()
    assert flod.flod_read_status(c["st"].rast.ws) == 0
    out = [{f: t.cpu().numpy() for f, t in zip(flod.GaussianSet.FIELDS, per)} for per in c["st"].grads]
    dL.copy_(full)
    return out


def _selection(c, v):
    cam = c["cams"][v]
    ent = S.select([c["np_sel"][i]["means"] for i in range(5)], cam["cam_pos"], TH)
    lv, idx = ent >> S.LEVEL_SHIFT, ent & ((1 << S.LEVEL_SHIFT) - 1)
    g = {k: np.concatenate([c["np_sel"][l][k][i:i + 1] for l, i in zip(lv, idx)])
         for k in ("means", "quats", "s_opt", "opacity_logit", "sh")}
    g["sh_degree"] = 3
    smin = torch.as_tensor(np.array([c["smin5"][l] for l in lv])[:, None])
    return g, smin, lv, idx


def _check_view(c, v, g, s_min, set_of, sample_fn, seed):
    cam = c["cams"][v]
    ocfg = oracle_cfg(c["cfg"])
    with torch.no_grad():
        pre = R.preprocess(R.params(g), 3, s_min, cam, ocfg)
    lists = R.tile_lists(pre, cam, ocfg)
    rng = np.random.default_rng(seed)
    tiles = tile_sample(lists[2], lists[3], lists[4], 24, rng)
    ref = R.render_tiles(pre, cam, ocfg, lists, tiles)
    rgb, T, nc = _outputs(c, v)
    assert_tiles_close(rgb, T, nc, ref, pre, lists, cam, ocfg, f"batched view {v}",
                       gpu_view_lists(c["st"].rast, v))
    grads = _view_grads(c, v)
    # Gaussians the oracle blends in the sampled tiles (a fully occluded one has a zero
    # gradient and would make the comparison vacuous)
    sample = sample_fn(blended_gaussians(lists, ref), rng)
    H, W = cam["height"], cam["width"]
    o = c["offs"]
    dL_img = c["dL_np"][3 * o[v]:3 * o[v + 1]].reshape(3, H, W)
    want = R.sampled_gradients(g, 3, s_min, cam, ocfg, dL_img, sample, lists=lists, pre=pre)
    got = {k: np.stack([grads[set_of(j)[0]][k][set_of(j)[1]] for j in sample]) for k in want}
    assert_nonvacuous(want, f"batched view {v}")
    assert_grad_close(got, want, f"batched view {v}")


def test_c4_level1_4k_view(c4):
    _check_view(c4, VIEW_L1_4K, c4["np_lvl"][0], synth.LEVEL_SMIN[0], lambda j: (5, j),
                lambda vis, rng: rng.choice(vis, 6, replace=False), 40)


def test_c4_level5_1080p_view(c4):
    def pick(vis, rng):
        return np.concatenate([rng.choice(vis[vis < 20_000], 2, replace=False),
                               rng.choice(vis[vis >= 1_000_000], 4, replace=False)])
    _check_view(c4, VIEW_L5_1080P, c4["np_lvl"][4], synth.LEVEL_SMIN[4], lambda j: (9, j), pick, 41)


def test_c4_selective_4k_view(c4):
    g, smin, lv, idx = _selection(c4, VIEW_SEL_4K)
    # the selection the batch rendered is the oracle's, entry for entry
    st = c4["st"]
    k = VIEW_SEL_4K
    jobs_sel = [i for i, s in enumerate(st.sel) if s is not None]
    assert k in jobs_sel
    _, buf, cnt, _ = st.sel[k]
    n = int(cnt.item())
    assert n == lv.size and n > 0
    ent = buf[:n].cpu().numpy().astype(np.int64)
    assert np.array_equal(ent >> S.LEVEL_SHIFT, lv) and np.array_equal(ent & ((1 << S.LEVEL_SHIFT) - 1), idx)
    _check_view(c4, k, g, smin, lambda j: (int(lv[j]), int(idx[j])),
                lambda vis, rng: rng.choice(vis, 6, replace=False), 42)
