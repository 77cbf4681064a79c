"""Pins of the oracle's selective-rendering set (Eq. 6, Eq. 7) -- CPU only."""
import math
import os

import numpy as np
import pytest

from oracle import gaussians as G
from oracle import select as S
from paper_2408_12894_gb300 import synth

GOLD = os.path.join(os.path.dirname(__file__), "golden")


def _table(name):
    out = []
    for line in open(os.path.join(GOLD, name)):
        line = line.split("#")[0].strip()
        if line:
            out.append(line.split())
    return out


def test_eq7_thresholds_worked_values():
    par = {r[0]: float(r[1]) for r in _table("paper_parameters.txt")}
    sched = G.s_min_schedule(par["lambda"], par["rho"], int(par["L_max"]))
    f = 960.0 * math.sqrt(3.0)
    assert f == pytest.approx(synth.camera((0, 0, -1), 1920, 1080)["fx"], rel=1e-7)
    th = S.d_proj(sched, f, par["gamma"])
    want = [float(r[1]) for r in _table("eq7_dproj_worked.txt")]
    np.testing.assert_allclose(th, want[:-1], rtol=1e-12)
    # the band of the finest level ends at 0 and that of the coarsest at infinity
    assert S.band(4, th) == (0.0, th[3])
    assert S.band(0, th) == (th[0], math.inf)


def test_partition_every_distance_maps_to_one_level():
    rng = np.random.default_rng(0)
    means = rng.uniform(-150, 150, (5000, 3)).astype(np.float32)
    th = list(synth.SELECTIVE_THRESHOLDS[::-1])           # 100, 50, 25, 10: coarse -> fine
    sel = S.select([means] * 5, np.zeros(3), th)
    idx = sel & ((1 << S.LEVEL_SHIFT) - 1)
    assert np.array_equal(np.sort(idx), np.arange(5000))   # each Gaussian exactly once
    lev = sel >> S.LEVEL_SHIFT
    d = np.linalg.norm(means.astype(np.float64), axis=1)
    for k in range(5):
        lo, hi = S.band(k, th)
        dk = d[idx[lev == k]]
        assert np.all((dk >= lo - 1e-4) & (dk < hi + 1e-4))


def test_select_matches_brute_force_loop():
    rng = np.random.default_rng(1)
    levels = [rng.uniform(-60, 60, (n, 3)).astype(np.float32) for n in (50, 120, 300, 500, 800)]
    origin = np.array([3.0, -2.0, 7.5], dtype=np.float32)
    th = [100.0, 50.0, 25.0, 10.0]
    got = S.select(levels, origin, th)
    loop = S.select_loop(levels, origin, th)
    assert [(int(e) >> S.LEVEL_SHIFT, int(e) & ((1 << S.LEVEL_SHIFT) - 1)) for e in got] == loop
    np.testing.assert_array_equal(S.select_exact(levels, origin, th), got)


def test_selected_count_monotone_in_gamma_for_nested_levels():
    # nested levels (each level holds the previous one's Gaussians): a larger gamma moves
    # every distance band towards coarser levels, so |G_sel| never grows (Sec. 5.2)
    rng = np.random.default_rng(2)
    base = rng.uniform(-100, 100, (4000, 3)).astype(np.float32)
    counts = (200, 500, 1000, 2000, 4000)
    levels = [base[:n] for n in counts]
    sched = [0.5, 0.25, 0.125, 0.0625, 0.03125]
    prev = None
    for gamma in (0.25, 0.5, 1.0, 2.0, 4.0, 8.0):
        th = S.d_proj(sched, 200.0, gamma)
        n = S.select(levels, np.zeros(3), th).size
        if prev is not None:
            assert n <= prev
        prev = n


def test_threshold_ties_go_to_the_level_whose_band_starts_there():
    means = np.array([[10.0, 0, 0], [0, 25.0, 0], [0, 0, 9.999999]], dtype=np.float32)
    th = [100.0, 50.0, 25.0, 10.0]
    sel = S.select([means] * 5, np.zeros(3), th)
    got = {int(e) & 0xFFFFFFF: int(e) >> S.LEVEL_SHIFT for e in sel}
    assert got == {0: 3, 1: 2, 2: 4}     # d = 10 -> level index 3 (band [10, 25))
