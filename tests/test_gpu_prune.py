"""Overlap pruning (Sec. 4.3) on the GPU against the oracle's brute-force three nearest
neighbours: the keep mask bit for bit away from ties, d_avg where it is exact, the kept
index list, closed forms, and a full-size level."""
import numpy as np
import pytest
import torch

from oracle import prune as PR
from paper_2408_12894_gb300 import flod, synth

pytestmark = pytest.mark.gpu

TIE = 1e-5   # relative distance of d_avg to d_OP within which float32 may decide otherwise


def _run(means, d_op, s_min=0.0):
    n = means.shape[0]
    g = {"means": means.astype(np.float32), "quats": np.tile([1, 0, 0, 0], (n, 1)).astype(np.float32),
         "s_opt": np.zeros((n, 3), np.float32), "opacity_logit": np.zeros(n, np.float32),
         "sh": np.zeros((n, 1, 3), np.float32), "sh_degree": 0}
    gs = flod.GaussianSet.from_numpy(g, s_min)
    keep = torch.empty(max(n, 1), dtype=torch.uint8, device="cuda")
    davg = torch.empty(max(n, 1), dtype=torch.float32, device="cuda")
    kept = torch.full((max(n, 1),), -1, dtype=torch.int32, device="cuda")
    cnt = torch.zeros(1, dtype=torch.int32, device="cuda")
    status = torch.full((1,), 77, dtype=torch.int32, device="cuda")
    nb = flod.flod_prune_scratch_size(n)
    scr = torch.empty(nb + 256, dtype=torch.uint8, device="cuda")
    scr = scr[(-scr.data_ptr()) % 256:][:nb]
    flod.flod_overlap_prune(gs, d_op, keep, cnt, scr, d_avg=davg, out_kept=kept, d_status=status)
    torch.cuda.synchronize()
    k = keep[:n].cpu().numpy().astype(bool)
    m = int(cnt.item())
    assert int(status.item()) == 0
    assert m == int(k.sum())
    assert np.array_equal(kept[:m].cpu().numpy(), np.nonzero(k)[0])
    return k, davg[:n].cpu().numpy()


def _check(means, d_op):
    k, da = _run(means, d_op)
    d, _ = PR.knn3(means.astype(np.float32).astype(np.float64))
    ref_avg = d.mean(axis=1)
    ref_keep = ~(ref_avg < d_op)
    tie = np.abs(ref_avg - d_op) <= TIE * d_op
    assert np.array_equal(k[~tie], ref_keep[~tie]), np.nonzero(k[~tie] != ref_keep[~tie])[0][:10]
    exact = d[:, 2] < 3 * d_op * (1 - 1e-5)          # three neighbours within 3 d_OP
    np.testing.assert_allclose(da[exact], ref_avg[exact], rtol=2e-6, atol=1e-7 * d_op)
    assert np.all(np.isinf(da[d[:, 2] > 3 * d_op * (1 + 1e-5)]))
    return k, tie


@pytest.mark.parametrize("s_min", [0.05, 0.2])
def test_prune_mask_matches_oracle_on_a_clustered_level(s_min):
    g = synth.gaussian_set(31, 20000, k=16, radius=2.0)
    k, tie = _check(g["means"], 0.5 * s_min)
    assert 0 < (~k).sum() < k.size and tie.sum() < 10


def test_prune_lattice_duplicates_and_tiny_sets():
    a = 0.25
    lat = (np.stack(np.meshgrid(*[np.arange(12)] * 3, indexing="ij"), -1).reshape(-1, 3) * a)
    k, _ = _run(lat, a * 1.001)
    assert not k.any()                      # d_avg = a < d_OP: every point pruned
    k, _ = _run(lat, a * 0.999)
    assert k.all()
    rng = np.random.default_rng(5)
    m = rng.normal(size=(500, 3))
    m[10] = m[20] = m[30] = m[40]           # four Gaussians at one mean: d_avg 0
    k, da = _run(m, 1e-3)
    assert not k[[10, 20, 30, 40]].any() and np.all(da[[10, 20, 30, 40]] == 0)
    k, da = _run(m[:3], 1e6)                # fewer than three others: kept
    assert k.all()
    k, da = _run(np.zeros((0, 3)), 0.1)


def test_prune_full_level_four_sample():
    # level 4 of the 5-level scene (1M Gaussians, s_min 0.0625 -> d_OP 0.03125) right after a
    # densification step (10% clones moved by N(0, d_OP^2)): the mask and d_avg of a sample of
    # Gaussians, clones included, against brute force over the whole level
    levels = synth.level_scene(counts=synth.LEVEL_COUNTS[:4])
    d_op = 0.5 * synth.LEVEL_SMIN[3]
    means = synth.with_jittered_clones(levels[3][0], 0.1, d_op)["means"]
    k, da = _run(means, d_op)
    rng = np.random.default_rng(6)
    n0 = synth.LEVEL_COUNTS[3]
    # random Gaussians (nearly all kept) and every Gaussian the kernel pruned (up to 100)
    sample = np.concatenate([rng.choice(n0, 150, replace=False),
                             n0 + rng.choice(means.shape[0] - n0, 150, replace=False),
                             np.nonzero(~k)[0][:100]])
    m64 = means.astype(np.float64)
    for i in sample:
        dd = np.sqrt(((m64 - m64[i]) ** 2).sum(axis=1))
        dd[i] = np.inf
        d3 = np.sort(np.partition(dd, 3)[:3])
        avg = d3.mean()
        if abs(avg - d_op) <= TIE * d_op:
            continue
        assert k[i] == (not avg < d_op), i
        if d3[2] < 3 * d_op * (1 - 1e-5):
            assert abs(da[i] - avg) <= 2e-6 * avg + 1e-7 * d_op, (i, da[i], avg)
    assert 0 < (~k).sum()
