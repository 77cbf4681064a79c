"""The training step of a level (Loss and Adam of Algorithm 1) on the GPU against the FP64
oracle: the L1 + D-SSIM loss and its gradient (ragged multi-image batches and a full
1920x1080 image), the Adam step (several sets, several steps, the device step counter), the
preprocess backward fused with Adam, and a whole iteration."""
import numpy as np
import pytest
import torch

from gpu_helpers import GRAD_REL, assert_grad_close, rasterizer
from oracle import adam as AD
from oracle import loss as LS
from oracle import raster as R
from paper_2408_12894_gb300 import flod, synth, train

pytestmark = pytest.mark.gpu

LRS = {"means": 3.2e-3, "quats": 1e-3, "s_opt": 5e-3, "opacity_logit": 0.05, "sh_dc": 2.5e-3,
       "sh_rest": 1.25e-4}


def _gpu_loss(imgs, tgts):
    sizes = [(a.shape[2], a.shape[1]) for a in imgs]
    x = torch.as_tensor(np.concatenate([a.ravel() for a in imgs]).astype(np.float32), device="cuda")
    y = torch.as_tensor(np.concatenate([a.ravel() for a in tgts]).astype(np.float32), device="cuda")
    dL = torch.full_like(x, 7.0)
    loss = torch.full((len(imgs),), -1.0, device="cuda")
    scr = train._aligned_bytes(flod.flod_loss_scratch_size(sizes), "cuda")
    flod.flod_loss(x, y, sizes, dL, scr, loss)
    torch.cuda.synchronize()
    out, off = [], 0
    for a in imgs:
        out.append(dL[off:off + a.size].view(a.shape).cpu().numpy())
        off += a.size
    return loss.cpu().numpy(), out


def _check_loss(imgs, tgts):
    gl, gd = _gpu_loss(imgs, tgts)
    for i, (a, b) in enumerate(zip(imgs, tgts)):
        L, g = LS.loss_and_grad(a.astype(np.float32).astype(np.float64),
                                b.astype(np.float32).astype(np.float64))
        assert abs(gl[i] - L) <= 1e-5 * abs(L) + 1e-7, (i, gl[i], L)
        # the SSIM gradient is assembled from window sums of terms of size about
        # lambda / (N C2) (C2 = 9e-4) that cancel down to lambda / N or less; float32 leaves an
        # absolute error of about 1e-4 lambda / N there, so the elementwise floor is
        # 1e-3 lambda / N (N = 3 H W)
        floor = 1e-3 * LS.LAMBDA / a.size
        assert_grad_close({"dL": gd[i]}, {"dL": g}, f"loss gradient, image {i}", floor_abs=floor)


def test_loss_ragged_batch_matches_oracle():
    rng = np.random.default_rng(0)
    sizes = [(200, 120), (37, 53), (64, 64), (31, 5)]
    imgs = [rng.random((3, h, w)) for w, h in sizes]
    # targets: partly near the image (small differences, L1 kink nearby), partly far
    tgts = [np.clip(a + rng.normal(0, 0.05, a.shape), 0, 1) if i % 2 else rng.random(a.shape)
            for i, a in enumerate(imgs)]
    _check_loss(imgs, tgts)


def test_loss_full_hd_rendered_image_matches_oracle():
    # a rendered-looking image (smooth blobs, dark background) against a noisy target
    rng = np.random.default_rng(1)
    H, W = 1080, 1920
    yy, xx = np.mgrid[0:H, 0:W]
    img = np.zeros((3, H, W))
    for _ in range(40):
        cx, cy, s = rng.uniform(0, W), rng.uniform(0, H), rng.uniform(20, 200)
        img += rng.random(3)[:, None, None] * np.exp(-((xx - cx) ** 2 + (yy - cy) ** 2) / (2 * s * s))
    tgt = np.clip(img + rng.normal(0, 0.1, img.shape), 0, None)
    _check_loss([img], [tgt])


def test_loss_of_target_itself_is_zero():
    rng = np.random.default_rng(2)
    a = rng.random((3, 70, 90))
    gl, gd = _gpu_loss([a], [a])
    assert abs(gl[0]) < 1e-6
    assert np.abs(gd[0]).max() < 1e-9


def _rand_set(rng, n, deg):
    k = (deg + 1) ** 2
    return {"means": rng.normal(size=(n, 3)), "quats": rng.normal(size=(n, 4)),
            "s_opt": rng.normal(size=(n, 3)), "opacity_logit": rng.normal(size=n),
            "sh": rng.normal(size=(n, k, 3))}


def _dev(d):
    return [torch.as_tensor(d[f].astype(np.float32), device="cuda").contiguous()
            for f in flod.GaussianSet.FIELDS]


def _assert_adam_close(gpu, ora, lrs, what):
    for f, a in zip(flod.GaussianSet.FIELDS, gpu):
        a = a.cpu().numpy().astype(np.float64)
        b = ora[f]
        lr = AD.lr_of(f, b.shape, lrs)
        # float32 rounding of the new value plus a relative 1e-5 of the step (at most lr)
        tol = 2.0 ** -23 * np.abs(b) * 2 + 1e-5 * lr
        bad = np.abs(a - b) > tol
        assert not bad.any(), (what, f, np.abs(a - b)[bad].max())


def test_adam_step_two_sets_three_steps_matches_oracle():
    rng = np.random.default_rng(3)
    sets = [_rand_set(rng, 1003, 3), _rand_set(rng, 517, 1)]
    par = [_dev(s) for s in sets]
    m = [[torch.zeros_like(t) for t in p] for p in par]
    v = [[torch.zeros_like(t) for t in p] for p in par]
    step = torch.zeros(1, dtype=torch.int32, device="cuda")
    cfg = flod.adam_config(LRS, step, betas=(AD.BETA1, AD.BETA2), eps=AD.EPS)
    # the oracle starts from the same float32 values
    cur = [{f: s[f].astype(np.float32).astype(np.float64) for f in s} for s in sets]
    om = [{f: np.zeros_like(x) for f, x in c.items()} for c in cur]
    ov = [{f: np.zeros_like(x) for f, x in c.items()} for c in cur]
    for t in range(1, 4):
        grads_np = [_rand_set(rng, 1003, 3), _rand_set(rng, 517, 1)]
        for g in grads_np:
            g["means"][:5] = 0.0          # zero gradients take the step with g = 0
        grads = [_dev(g) for g in grads_np]
        flod.flod_adam_step(par, grads, m, v, [1003, 517], [3, 1], cfg)
        torch.cuda.synchronize()
        for k in range(2):
            gk = {f: grads_np[k][f].astype(np.float32).astype(np.float64) for f in grads_np[k]}
            cur[k], om[k], ov[k] = AD.adam_set(cur[k], gk, om[k], ov[k], t, LRS)
            _assert_adam_close(par[k], cur[k], LRS, f"set {k} step {t}")
            for f, a in zip(flod.GaussianSet.FIELDS, m[k]):
                # m = b1 m + (1 - b1) g cancels where m and g differ in sign: float32 leaves an
                # error of a few ulp of the terms, not of the result
                np.testing.assert_allclose(a.cpu().numpy(), om[k][f], rtol=1e-5,
                                           atol=4e-7 * np.abs(om[k][f]).max())
            for f, a in zip(flod.GaussianSet.FIELDS, v[k]):
                np.testing.assert_allclose(a.cpu().numpy(), ov[k][f], rtol=1e-5, atol=1e-12)
    assert int(step.item()) == 3


def _small_scene():
    g = synth.gaussian_set(21, 2500, k=8, radius=1.0, sh_degree=3, s_mean=-3.0)
    cam = synth.camera((0.4, 0.2, -3.0), 96, 72)
    return g, cam


def test_fused_backward_adam_equals_gradient_then_adam():
    # flod_preprocess_bwd_adam against flod_preprocess_bwd (overwrite) + flod_adam_step on the
    # same per-unit 2D gradients: two steps
    g, cam = _small_scene()
    dL = torch.as_tensor(synth.upstream_gradient(22, [cam]), device="cuda")
    ra = rasterizer([g], [cam], [0.01])
    rb = rasterizer([g], [cam], [0.01])
    step_a = torch.zeros(1, dtype=torch.int32, device="cuda")
    step_b = torch.zeros(1, dtype=torch.int32, device="cuda")
    ma = [torch.zeros_like(getattr(ra.sets[0], f)) for f in flod.GaussianSet.FIELDS]
    va = [torch.zeros_like(t) for t in ma]
    mb = [torch.zeros_like(t) for t in ma]
    vb = [torch.zeros_like(t) for t in ma]
    pa = [getattr(ra.sets[0], f) for f in flod.GaussianSet.FIELDS]
    pb = [getattr(rb.sets[0], f) for f in flod.GaussianSet.FIELDS]
    states = flod.adam_states([(pa, ma, va)])
    gb = [torch.empty_like(t) for t in pb]
    for t in range(2):
        rgb, T, nc = ra.forward()
        ra.blend_bwd(dL, T, nc)
        ra.preprocess_bwd_adam(states, flod.adam_config(LRS, step_a))
        rgb2, T2, nc2 = rb.forward()
        rb.blend_bwd(dL, T2, nc2)
        rb.preprocess_bwd(flod.grads_struct([gb], overwrite=True))
        flod.flod_adam_step([pb], [gb], [mb], [vb], [rb.sets[0].n], [3], flod.adam_config(LRS, step_b))
        torch.cuda.synchronize()
        # the moments hold the gradients: equal up to the blending backward's atomics order
        for a, b in zip(ma, mb):
            assert torch.allclose(a, b, rtol=1e-4, atol=1e-7 * float(b.abs().max()) + 1e-30)
        # parameters: entries whose step direction is settled agree to float32 rounding
        for f, a, b, mbv in zip(flod.GaussianSet.FIELDS, pa, pb, mb):
            settled = mbv.abs() > 1e-3 * mbv.abs().max()
            lr = torch.as_tensor(AD.lr_of(f, tuple(b.shape), LRS), device="cuda", dtype=torch.float32)
            d = (a - b).abs()
            tol = 4e-7 * b.abs() + 1e-3 * lr
            assert bool((d <= tol)[settled].all()), (f, t)
    assert int(step_a.item()) == 2 and int(step_b.item()) == 2


def test_fused_backward_adam_two_sets_ragged_and_many_chunks_per_cta():
    # two sets, each rendered by its own view: 200,003 Gaussians at SH degree 3 (about five
    # 128-Gaussian chunks per persistent CTA, so both shared buffers are reused) and 1,333 at
    # degree 1 (a last chunk of 53: the scalar tails); the fused step against gradient then
    # Adam, two steps
    g1 = synth.gaussian_set(31, 200_003, k=16, radius=1.0, sh_degree=3, s_mean=-4.0)
    g2 = synth.gaussian_set(32, 1_333, k=4, radius=1.0, sh_degree=1, s_mean=-3.0)
    cams = [synth.camera((0.4, 0.2, -3.0), 96, 72), synth.camera((-0.3, 0.1, -2.5), 128, 96)]
    dL = torch.as_tensor(synth.upstream_gradient(24, cams), device="cuda")
    ra = rasterizer([g1, g2], cams, [0.01, 0.02], view_sets=[0, 1])
    rb = rasterizer([g1, g2], cams, [0.01, 0.02], view_sets=[0, 1])
    step_a = torch.zeros(1, dtype=torch.int32, device="cuda")
    step_b = torch.zeros(1, dtype=torch.int32, device="cuda")
    fa, fb, ga = [], [], []
    for k in range(2):
        pa = [getattr(ra.sets[k], f) for f in flod.GaussianSet.FIELDS]
        pb = [getattr(rb.sets[k], f) for f in flod.GaussianSet.FIELDS]
        fa.append((pa, [torch.zeros_like(t) for t in pa], [torch.zeros_like(t) for t in pa]))
        fb.append((pb, [torch.zeros_like(t) for t in pb], [torch.zeros_like(t) for t in pb]))
        ga.append([torch.empty_like(t) for t in pb])
    states = flod.adam_states(fa)
    for t in range(2):
        rgb, T, nc = ra.forward()
        ra.blend_bwd(dL, T, nc)
        ra.preprocess_bwd_adam(states, flod.adam_config(LRS, step_a))
        rgb2, T2, nc2 = rb.forward()
        rb.blend_bwd(dL, T2, nc2)
        rb.preprocess_bwd(flod.grads_struct(ga, overwrite=True))
        flod.flod_adam_step([x[0] for x in fb], ga, [x[1] for x in fb], [x[2] for x in fb],
                            [s.n for s in rb.sets], [s.sh_degree for s in rb.sets],
                            flod.adam_config(LRS, step_b))
        torch.cuda.synchronize()
        for k in range(2):
            for a, b in zip(fa[k][1], fb[k][1]):
                assert torch.allclose(a, b, rtol=1e-4, atol=1e-7 * float(b.abs().max()) + 1e-30), (k, t)
            for a, b in zip(fa[k][2], fb[k][2]):
                assert torch.allclose(a, b, rtol=1e-4, atol=1e-7 * float(b.abs().max()) + 1e-30), (k, t)
            for f, a, b, mbv in zip(flod.GaussianSet.FIELDS, fa[k][0], fb[k][0], fb[k][1]):
                settled = mbv.abs() > 1e-3 * mbv.abs().max()
                lr = torch.as_tensor(AD.lr_of(f, tuple(b.shape), LRS), device="cuda", dtype=torch.float32)
                d = (a - b).abs()
                tol = 4e-7 * b.abs() + 1e-3 * lr
                assert bool((d <= tol)[settled].all()), (k, f, t)
                # untouched entries (zero moments) keep their value on both paths
                assert torch.equal(a[mbv == 0], b[mbv == 0]), (k, f, t)
    assert int(step_a.item()) == 2 and int(step_b.item()) == 2


def test_fused_backward_adam_first_step_matches_oracle():
    # one fused step from zero moments: m = (1 - beta1) g must hold the oracle's gradient, and
    # every parameter whose gradient is clear of zero moves by exactly lr against its sign
    g, cam = _small_scene()
    s_min = 0.01
    dL_np = synth.upstream_gradient(23, [cam])
    dL = torch.as_tensor(dL_np, device="cuda")
    rast = rasterizer([g], [cam], [s_min])
    p0 = {f: getattr(rast.sets[0], f).clone() for f in flod.GaussianSet.FIELDS}
    pa = [getattr(rast.sets[0], f) for f in flod.GaussianSet.FIELDS]
    ma = [torch.zeros_like(t) for t in pa]
    va = [torch.zeros_like(t) for t in pa]
    step = torch.zeros(1, dtype=torch.int32, device="cuda")
    rgb, T, nc = rast.forward()
    rast.blend_bwd(dL, T, nc)
    rast.preprocess_bwd_adam(flod.adam_states([(pa, ma, va)]),
                             flod.adam_config(LRS, step, betas=(AD.BETA1, AD.BETA2), eps=AD.EPS))
    torch.cuda.synchronize()
    _, _, _, ref = R.forward_backward(g, 3, s_min, cam, R.Config(),
                                      dL_np.reshape(3, cam["height"], cam["width"]).astype(np.float64))
    got = {f: a.cpu().numpy() / (1.0 - AD.BETA1) for f, a in zip(flod.GaussianSet.FIELDS, ma)}
    assert_grad_close(got, ref, "fused backward gradient")
    for f, a in zip(flod.GaussianSet.FIELDS, pa):
        gr = ref[f]
        clear = np.abs(gr) > 10 * GRAD_REL * np.abs(gr).max()
        lr = AD.lr_of(f, gr.shape, LRS)
        want = p0[f].cpu().numpy().astype(np.float64) - lr * np.sign(gr)
        d = np.abs(a.cpu().numpy() - want)
        assert np.all((d <= 4e-7 * np.abs(want) + 1e-5 * lr)[clear]), f
        assert clear.sum() > 0


def test_train_step_iteration_matches_oracle_loss_and_reduces_it():
    # whole iterations through TrainStep: the first iteration's loss equals the oracle's loss
    # of the oracle render; over 30 iterations towards a target rendered from perturbed
    # colours the loss goes down
    g, cam = _small_scene()
    gt = dict(g)
    rng = np.random.default_rng(24)
    gt["sh"] = g["sh"].copy()
    gt["sh"][:, 0, :] += rng.normal(0, 0.6, gt["sh"][:, 0, :].shape).astype(np.float32)
    tgt_img, _, _ = R.render(gt, 3, 0.01, cam, R.Config())
    target = torch.as_tensor(tgt_img.astype(np.float32).ravel(), device="cuda")
    sets = [flod.GaussianSet.from_numpy(g, 0.01)]
    lrs = {"means": 1e-4, "quats": 1e-3, "s_opt": 1e-3, "opacity_logit": 1e-2, "sh_dc": 5e-2,
           "sh_rest": 1e-3}
    st = train.TrainStep(sets, [flod.view_struct(cam)], target, lrs=lrs)
    assert st.fused
    st.size_capacity()
    st.run()
    torch.cuda.synchronize()
    img, _, _ = R.render(g, 3, 0.01, cam, R.Config())
    L0, _ = LS.loss_and_grad(img, tgt_img.astype(np.float32).astype(np.float64))
    assert abs(float(st.loss[0]) - L0) <= 2e-4 * L0
    first = float(st.loss[0])
    for _ in range(29):
        st.run()
    torch.cuda.synchronize()
    assert float(st.loss[0]) < 0.9 * first
    assert int(st.d_step.item()) == 30
    assert flod.flod_read_status(st.rast.ws) == 0


def test_train_step_two_views_uses_gradient_then_adam_and_graph_replay():
    g, cam = _small_scene()
    cam2 = synth.camera((-1.5, 0.4, -2.6), 80, 64)
    rng = np.random.default_rng(25)
    target = torch.as_tensor(rng.random(3 * (96 * 72 + 80 * 64)).astype(np.float32), device="cuda")
    sets = [flod.GaussianSet.from_numpy(g, 0.01)]
    st = train.TrainStep(sets, [flod.view_struct(cam), flod.view_struct(cam2)], target, lrs=LRS)
    assert not st.fused
    st.size_capacity()
    st.capture()
    for _ in range(3):
        st.replay()
    torch.cuda.synchronize()
    assert int(st.d_step.item()) == 3
    assert torch.isfinite(st.loss).all() and bool((st.loss > 0).all())
    assert flod.flod_read_status(st.rast.ws) == 0
