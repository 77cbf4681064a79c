"""Pins of the oracle's density control (Densification and Pruning of Algorithm 1) -- CPU
only."""
import numpy as np
import torch

from oracle import densify as D
from oracle import gaussians as G


def _set(n=6, seed=0):
    rng = np.random.default_rng(seed)
    q = rng.normal(size=(n, 4))
    return {"means": rng.normal(size=(n, 3)), "quats": q / np.linalg.norm(q, axis=1, keepdims=True),
            "s_opt": np.log(np.full((n, 3), 0.05)), "opacity_logit": np.zeros(n),
            "sh": rng.normal(size=(n, 16, 3)), "sh_degree": 3}


def test_statistics_are_the_ndc_gradient_norm_of_visible_gaussians():
    acc, den = np.zeros(3), np.zeros(3)
    g = np.array([[3.0, 4.0], [1.0, 0.0], [5.0, 5.0]])
    acc, den = D.stats_update(acc, den, g, np.array([True, True, False]), 2, 4)
    # NDC gradient = pixel gradient x (W/2, H/2) = (1, 2)
    np.testing.assert_allclose(acc, [np.hypot(3.0, 8.0), 1.0, 0.0])
    np.testing.assert_allclose(den, [1, 1, 0])
    acc, den = D.stats_update(acc, den, g, np.array([True, False, True]), 2, 4)
    np.testing.assert_allclose(den, [2, 1, 1])


def test_each_branch_and_the_new_set_order():
    g = _set(6)
    s_min = 0.01
    # sizes: 0, 1, 2 small (0.06 <= 0.1), 3, 4, 5 large; 4 transparent
    g["s_opt"][3:] = np.log(0.5)
    g["opacity_logit"][4] = -10.0
    accum = np.array([5e-4, 1e-4, 2e-4, 5e-4, 5e-4, 0.0])
    denom = np.array([1, 1, 1, 1, 1, 0])
    surv, clone, split = D.decisions(g, s_min, accum, denom, 2e-4, 0.1, 0.005)
    assert list(surv) == [True, True, True, False, False, True]
    assert list(clone) == [True, False, True, False, False, False]   # 2: g == tau clones
    assert list(split) == [False, False, False, True, False, False]
    normals = np.random.default_rng(1).normal(size=(12, 3))
    out = D.densify(g, s_min, accum, denom, normals, 2e-4, 0.1, 0.005)
    assert out["means"].shape[0] == 4 + 2 + 2
    np.testing.assert_array_equal(out["sh"][:4], g["sh"][[0, 1, 2, 5]])
    np.testing.assert_array_equal(out["sh"][4:6], g["sh"][[0, 2]])
    np.testing.assert_array_equal(out["sh"][6:], g["sh"][[3, 3]])
    # children: the learnable part of the scale over 1.6, s_min kept as the lower bound
    np.testing.assert_allclose(np.exp(out["s_opt"][6:]) + s_min, 0.5 / 1.6 + s_min, rtol=1e-12)


def test_split_children_sample_the_gaussian():
    # the children's offsets R (s * eps) have the covariance of Eq. 1 (Sigma = R S S^T R^T)
    g = _set(1, seed=3)
    g["s_opt"][:] = np.log([0.3, 0.1, 0.05])
    n = 100_000
    rng = np.random.default_rng(4)
    big = {k: (np.repeat(v, n, axis=0) if k != "sh_degree" else v) for k, v in g.items()}
    normals = rng.normal(size=(2 * n, 3))
    out = D.densify(big, 0.0, np.ones(n), np.ones(n), normals, 0.5, 0.01, 0.005)
    offs = out["means"] - g["means"][0]
    cov = np.cov(offs.T)
    sigma = G.covariance(torch.as_tensor(g["quats"]), torch.as_tensor(np.exp(g["s_opt"]))).numpy()[0]
    np.testing.assert_allclose(cov, sigma, atol=0.01 * np.abs(sigma).max())


def test_adam_moments_follow_the_survivors():
    g = _set(5)
    g["s_opt"][2] = np.log(0.5)
    m = {k: np.full(np.shape(g[k]), 3.0) for k in D.FIELDS}
    v = {k: np.full(np.shape(g[k]), 7.0) for k in D.FIELDS}
    out, m2, v2 = D.densify(g, 0.0, np.array([1, 1, 1, 0, 0.0]), np.ones(5),
                            np.zeros((10, 3)), 0.5, 0.1, 0.005, m, v)
    # 0, 1 cloned, 2 split, 3, 4 kept: 4 survivors, 2 clones, 2 children
    assert out["means"].shape[0] == 8
    for k in D.FIELDS:
        assert np.all(m2[k][:4] == 3.0) and np.all(m2[k][4:] == 0.0)
        assert np.all(v2[k][:4] == 7.0) and np.all(v2[k][4:] == 0.0)
    # zero draws: the children sit on the parent's mean
    np.testing.assert_array_equal(out["means"][6:], g["means"][[2, 2]])
