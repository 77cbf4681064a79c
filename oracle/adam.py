"""The optimiser step of each training iteration, FP64 -- TEST INFRASTRUCTURE ONLY.

Algorithm 1 updates the means, the scale parameters s_opt, the rotations, the colours and
the opacities with Adam on the loss gradient after every rasterization (the Adam /
Backpropagation step). Adam (Kingma and Ba, 2015), per parameter entry, at step t >= 1:

    m <- beta1 m + (1 - beta1) g
    v <- beta2 v + (1 - beta2) g^2
    p <- p - lr (m / (1 - beta1^t)) / (sqrt(v / (1 - beta2^t)) + eps)

Reading of the hyper-parameters (those of the 3DGS backbone, which the paper keeps for
everything it does not state, Sec. 5.1.4): beta1 = 0.9, beta2 = 0.999, eps = 1e-15, one
learning rate per parameter group -- means, rotations, s_opt, opacity logits, the SH DC
coefficient and the higher SH coefficients (the last two are one [N, K, 3] array here,
coefficient 0 and coefficients 1..K-1).
"""
from __future__ import annotations

import numpy as np

BETA1, BETA2, EPS = 0.9, 0.999, 1e-15
GROUPS = ("means", "quats", "s_opt", "opacity_logit", "sh_dc", "sh_rest")


def adam_entry(p, g, m, v, t: int, lr, beta1=BETA1, beta2=BETA2, eps=EPS):
    """One Adam step of arrays of entries (FP64); returns (p, m, v) new."""
    p, g, m, v = (np.asarray(a, dtype=np.float64) for a in (p, g, m, v))
    m = beta1 * m + (1.0 - beta1) * g
    v = beta2 * v + (1.0 - beta2) * g * g
    mh = m / (1.0 - beta1 ** t)
    vh = v / (1.0 - beta2 ** t)
    return p - lr * mh / (np.sqrt(vh) + eps), m, v


def lr_of(name: str, shape, lrs: dict):
    """Per-entry learning rate of a parameter array: the SH array takes the DC rate on
    coefficient 0 and the higher-order rate on the others."""
    if name != "sh":
        return lrs[name]
    lr = np.full(shape, lrs["sh_rest"], dtype=np.float64)
    lr[:, 0, :] = lrs["sh_dc"]
    return lr


def adam_set(params: dict, grads: dict, m: dict, v: dict, t: int, lrs: dict,
             beta1=BETA1, beta2=BETA2, eps=EPS):
    """Adam on every parameter array of one Gaussian set (dicts of arrays keyed means,
    quats, s_opt, opacity_logit, sh); returns new (params, m, v) dicts."""
    out_p, out_m, out_v = {}, {}, {}
    for k in ("means", "quats", "s_opt", "opacity_logit", "sh"):
        lr = lr_of(k, np.shape(params[k]), lrs)
        out_p[k], out_m[k], out_v[k] = adam_entry(params[k], grads[k], m[k], v[k], t, lr,
                                                  beta1, beta2, eps)
    return out_p, out_m, out_v
