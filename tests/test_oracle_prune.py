"""Pins of the oracle's overlap pruning (Sec. 4.3) -- CPU only."""
import numpy as np
import pytest
from scipy.spatial import cKDTree

from oracle import prune as PR
from paper_2408_12894_gb300 import synth


def test_knn3_equals_a_kd_tree():
    # scipy's k-d tree, a library routine independent of the oracle
    g = synth.gaussian_set(0, 3000, k=8, radius=2.0)
    m = g["means"].astype(np.float64)
    d, idx = PR.knn3(m)
    dt, it = cKDTree(m).query(m, k=4)
    np.testing.assert_allclose(d, dt[:, 1:], rtol=1e-12, atol=1e-15)
    np.testing.assert_allclose(PR.d_avg(m), dt[:, 1:].mean(axis=1), rtol=1e-12)


def test_lattice_closed_form():
    # on a cubic lattice of spacing a every point has neighbours at exactly a (6 inside, at
    # least 3 on a corner): d_avg = a, pruned exactly when a < s_min / 2
    a = 0.3
    g = np.stack(np.meshgrid(*[np.arange(5) * a] * 3, indexing="ij"), -1).reshape(-1, 3)
    np.testing.assert_allclose(PR.d_avg(g), a, rtol=1e-12)
    assert PR.keep_mask(g, 2 * a - 1e-9).all()            # d_OP just below a: kept
    assert not PR.keep_mask(g, 2 * a + 1e-9).any()        # d_OP just above a: all pruned


def test_equals_a_plain_loop_with_duplicates_and_tiny_sets():
    rng = np.random.default_rng(1)
    m = rng.normal(size=(40, 3))
    m[7] = m[3]                          # a duplicate: neighbour at distance 0
    da = PR.d_avg(m)
    for i in range(40):
        assert abs(da[i] - PR.d_avg_loop(m, i)) < 1e-12
    assert PR.knn3(m)[0][3, 0] == 0.0 and PR.knn3(m)[1][3, 0] == 7
    # fewer than three other Gaussians: kept
    assert PR.keep_mask(m[:3], 1e9).all() and np.isinf(PR.d_avg(m[:3])).all()
    assert PR.keep_mask(m[:1], 1e9).all()


@pytest.mark.parametrize("s_min", [0.05, 0.2])
def test_prune_fraction_grows_with_the_constraint(s_min):
    g = synth.gaussian_set(2, 5000, k=8, radius=1.0)
    keep = PR.keep_mask(g["means"], s_min)
    keep2 = PR.keep_mask(g["means"], 2 * s_min)
    assert keep.sum() > keep2.sum() and (keep2 <= keep).all()   # monotone in d_OP
