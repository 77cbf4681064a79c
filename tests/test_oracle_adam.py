"""Pins of the oracle's Adam step (the Adam step of Algorithm 1) -- CPU only."""
import numpy as np
import torch

from oracle import adam as AD

LRS = {"means": 3.2e-3, "quats": 1e-3, "s_opt": 5e-3, "opacity_logit": 0.05,
       "sh_dc": 2.5e-3, "sh_rest": 1.25e-4}


def _set(rng, n=37, k=16):
    return {"means": rng.normal(size=(n, 3)), "quats": rng.normal(size=(n, 4)),
            "s_opt": rng.normal(size=(n, 3)), "opacity_logit": rng.normal(size=n),
            "sh": rng.normal(size=(n, k, 3))}


def test_first_step_moves_by_lr_times_sign():
    rng = np.random.default_rng(0)
    p, g = _set(rng), _set(rng)
    z = {k: np.zeros_like(v) for k, v in p.items()}
    p1, m1, v1 = AD.adam_set(p, g, z, z, 1, LRS)
    for k in p:
        lr = AD.lr_of(k, p[k].shape, LRS)
        # m_hat = g and v_hat = g^2 at t = 1: the step is lr g / (|g| + eps)
        np.testing.assert_allclose(p1[k], p[k] - lr * g[k] / (np.abs(g[k]) + AD.EPS), rtol=1e-13)
        np.testing.assert_allclose(m1[k], 0.1 * g[k], rtol=1e-14)
        np.testing.assert_allclose(v1[k], 0.001 * g[k] ** 2, rtol=1e-14)
    # the SH DC coefficient takes its own rate
    d = p[k] - p1[k]
    np.testing.assert_allclose(np.abs(d[:, 0, :]), LRS["sh_dc"], rtol=1e-9)
    np.testing.assert_allclose(np.abs(d[:, 1:, :]), LRS["sh_rest"], rtol=1e-9)


def test_matches_torch_adam_over_several_steps():
    # torch.optim.Adam (a library implementation) with one parameter group per rate
    rng = np.random.default_rng(1)
    p = _set(rng)
    tp = {k: torch.tensor(v, dtype=torch.float64, requires_grad=True) for k, v in p.items()}
    dc = torch.tensor(p["sh"][:, :1, :], dtype=torch.float64, requires_grad=True)
    rest = torch.tensor(p["sh"][:, 1:, :], dtype=torch.float64, requires_grad=True)
    groups = [{"params": [tp[k]], "lr": LRS[k]} for k in ("means", "quats", "s_opt", "opacity_logit")]
    groups += [{"params": [dc], "lr": LRS["sh_dc"]}, {"params": [rest], "lr": LRS["sh_rest"]}]
    opt = torch.optim.Adam(groups, betas=(AD.BETA1, AD.BETA2), eps=AD.EPS)
    m = {k: np.zeros_like(v) for k, v in p.items()}
    v = {k: np.zeros_like(x) for k, x in p.items()}
    cur = {k: x.copy() for k, x in p.items()}
    for t in range(1, 8):
        g = _set(rng)
        for k in ("means", "quats", "s_opt", "opacity_logit"):
            tp[k].grad = torch.tensor(g[k])
        dc.grad = torch.tensor(g["sh"][:, :1, :])
        rest.grad = torch.tensor(g["sh"][:, 1:, :])
        opt.step()
        cur, m, v = AD.adam_set(cur, g, m, v, t, LRS)
    for k in ("means", "quats", "s_opt", "opacity_logit"):
        np.testing.assert_allclose(cur[k], tp[k].detach().numpy(), rtol=1e-12, atol=1e-15)
    np.testing.assert_allclose(cur["sh"][:, :1, :], dc.detach().numpy(), rtol=1e-12, atol=1e-15)
    np.testing.assert_allclose(cur["sh"][:, 1:, :], rest.detach().numpy(), rtol=1e-12, atol=1e-15)


def test_zero_gradient_from_zero_state_leaves_parameters():
    rng = np.random.default_rng(2)
    p = _set(rng)
    z = {k: np.zeros_like(v) for k, v in p.items()}
    p1, m1, v1 = AD.adam_set(p, z, z, z, 1, LRS)
    for k in p:
        np.testing.assert_array_equal(p1[k], p[k])
