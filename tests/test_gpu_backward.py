"""GPU backward (blend backward + preprocess backward, behind torch.autograd) vs the
oracle's analytic gradient (autograd of the FP64 forward, itself pinned to central finite
differences in test_oracle_raster)."""
import numpy as np
import pytest
import torch

from gpu_helpers import assert_grad_close, rasterizer
from oracle import raster as R
from paper_2408_12894_gb300 import flod, synth

pytestmark = pytest.mark.gpu


def _gpu_grads(g, cams, s_min, dL, cfg=None):
    rast = rasterizer([g], cams, [s_min], cfg=cfg)
    for f in flod.GaussianSet.FIELDS:
        getattr(rast.sets[0], f).requires_grad_(True)
    rgb, T, nc = flod.rasterize(rast)
    (rgb * torch.as_tensor(dL, device=rgb.device)).sum().backward()
    out = {f: getattr(rast.sets[0], f).grad.cpu().numpy().astype(np.float64)
           for f in flod.GaussianSet.FIELDS}
    assert flod.flod_read_status(rast.ws) == 0
    return out, rgb.detach().cpu().numpy()


def _oracle_grads(g, cams, s_min, dL, cfg=R.Config()):
    tot = None
    off = 0
    for c in cams:
        n = 3 * c["width"] * c["height"]
        go = dL[off:off + n].reshape(3, c["height"], c["width"]).astype(np.float64)
        off += n
        _, _, _, gr = R.forward_backward(g, g["sh_degree"], s_min, c, cfg, go)
        tot = gr if tot is None else {k: tot[k] + gr[k] for k in tot}
    return tot


def _compare(got, ref):
    assert_grad_close(got, ref)


@pytest.mark.parametrize("views", [1, 2])
def test_backward_matches_oracle(views):
    g = synth.gaussian_set(9, 2500, k=8, radius=1.0, sh_degree=3, s_mean=-3.0)
    cams = [synth.camera((0.4, 0.2, -3.0), 96, 72), synth.camera((-2.0, 0.5, -2.2), 80, 80)][:views]
    s_min = 0.01
    dL = synth.upstream_gradient(11, cams)
    got, _ = _gpu_grads(g, cams, s_min, dL)
    ref = _oracle_grads(g, cams, s_min, dL)
    _compare(got, ref)


def test_backward_small_tiles_and_batches():
    g = synth.gaussian_set(10, 1500, k=4, radius=1.0, sh_degree=2, s_mean=-2.7)
    cams = [synth.camera((0.1, -0.3, -2.8), 72, 56)]
    dL = synth.upstream_gradient(12, cams)
    cfg = flod.default_config(tile_w=8, tile_h=8, batch=32)
    got, _ = _gpu_grads(g, cams, 0.0, dL, cfg)
    ref = _oracle_grads(g, cams, 0.0, dL, R.Config(tile_w=8, tile_h=8))
    _compare(got, ref)


def test_backward_zero_upstream_gives_zero():
    g = synth.gaussian_set(11, 500, sh_degree=1)
    cams = [synth.camera((0.0, 0.0, -3.0), 64, 64)]
    got, _ = _gpu_grads(g, cams, 0.0, np.zeros(3 * 64 * 64, np.float32))
    for v in got.values():
        assert np.all(v == 0)


def test_overwrite_mode_equals_accumulate_into_zeros():
    g = synth.gaussian_set(12, 3000, k=8, radius=1.0, sh_degree=3, s_mean=-3.0)
    cam = synth.camera((0.3, -0.2, -3.0), 96, 64)
    dL = torch.as_tensor(synth.upstream_gradient(13, [cam]), device="cuda")
    rast = rasterizer([g], [cam], [0.02])
    rgb, T, nc = rast.forward()
    # one blend backward (its float atomics make the per-unit sums order-dependent), then
    # both write modes of the preprocess backward over the same per-unit gradients
    rast.blend_bwd(dL, T, nc)
    acc = [[torch.zeros_like(getattr(rast.sets[0], f)) for f in flod.GaussianSet.FIELDS]]
    rast.preprocess_bwd(flod.grads_struct(acc))
    over = [[torch.full_like(getattr(rast.sets[0], f), 7.5) for f in flod.GaussianSet.FIELDS]]
    rast.preprocess_bwd(flod.grads_struct(over, overwrite=True))
    torch.cuda.synchronize()
    for a, b in zip(acc[0], over[0]):
        assert torch.equal(a, b)
    # a set that two views render cannot be overwritten
    rast2 = rasterizer([g], [cam, cam], [0.02])
    rgb2, T2, nc2 = rast2.forward()
    dL2 = torch.zeros(2 * dL.numel(), device="cuda")
    rast2.blend_bwd(dL2, T2, nc2)
    with pytest.raises(flod.FlodError):
        rast2.preprocess_bwd(flod.grads_struct(over, overwrite=True))


@pytest.mark.parametrize("shape", [(16, 16), (32, 8)])
def test_persistent_backward_matches_oracle(shape):
    # the persistent launch (largest-first tile queue, CTAs taking tiles by ticket) of the
    # batched path, checked against the oracle directly: two views of one set, atomics
    g = synth.gaussian_set(14, 2500, k=8, radius=1.0, sh_degree=3, s_mean=-3.0)
    cams = [synth.camera((0.4, 0.2, -3.0), 96, 72), synth.camera((-2.0, 0.5, -2.2), 80, 80)]
    s_min = 0.01
    dL = synth.upstream_gradient(15, cams)
    cfg = flod.default_config(tile_w=shape[0], tile_h=shape[1], persistent=1)
    got, _ = _gpu_grads(g, cams, s_min, dL, cfg)
    ref = _oracle_grads(g, cams, s_min, dL, R.Config(tile_w=shape[0], tile_h=shape[1]))
    _compare(got, ref)


def test_backward_into_uninitialised_buffers_zero_first_mode():
    # flod_grads.overwrite = 2: the library zero-fills the buffers, then accumulates; two
    # views of one set (atomic path) from garbage-filled buffers equal accumulation into zeros
    g = synth.gaussian_set(16, 2000, k=8, radius=1.0, sh_degree=3, s_mean=-3.0)
    cams = [synth.camera((0.3, -0.2, -3.0), 96, 64), synth.camera((1.5, 0.2, -2.5), 64, 64)]
    dL = torch.as_tensor(synth.upstream_gradient(17, cams), device="cuda")
    rast = rasterizer([g], cams, [0.02])
    rgb, T, nc = rast.forward()
    rast.blend_bwd(dL, T, nc)
    acc = [[torch.zeros_like(getattr(rast.sets[0], f)) for f in flod.GaussianSet.FIELDS]]
    rast.preprocess_bwd(flod.grads_struct(acc))
    torch.cuda.synchronize()
    zf = [[torch.full_like(getattr(rast.sets[0], f), -3.25) for f in flod.GaussianSet.FIELDS]]
    rast.preprocess_bwd(flod.grads_struct(zf, flod.GRAD_ZERO_FIRST))
    torch.cuda.synchronize()
    for a, b in zip(acc[0], zf[0]):
        # atomics add in another order: equal up to float32 rounding of the sums
        assert torch.allclose(a, b, rtol=1e-5, atol=1e-12)
    assert rast.grad_modes() == [flod.GRAD_ZERO_FIRST]
    with pytest.raises(flod.FlodError):
        rast.preprocess_bwd(flod.grads_struct(zf, 3))


def test_autograd_backward_needs_its_own_forward():
    # a second forward on the same Rasterizer re-sorts the workspace: the first render's
    # backward must refuse instead of using the other sort
    g = synth.gaussian_set(18, 800, k=4, radius=1.0, sh_degree=1, s_mean=-3.0)
    cam = synth.camera((0.0, 0.1, -3.0), 64, 48)
    rast = rasterizer([g], [cam], [0.0])
    for f in flod.GaussianSet.FIELDS:
        getattr(rast.sets[0], f).requires_grad_(True)
    rgb1, _, _ = flod.rasterize(rast)
    rgb2, _, _ = flod.rasterize(rast)
    with pytest.raises(flod.FlodError):
        rgb1.sum().backward()
    rgb2.sum().backward()      # the latest forward's backward is fine
    assert rast.grad_modes() == [flod.GRAD_OVERWRITE]
