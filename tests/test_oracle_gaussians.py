"""Pins of the oracle's Gaussian parameterisation (Eq. 1, 3, 4, 5) -- CPU only."""
import math
import os

import numpy as np
import pytest
import torch

from oracle import gaussians as G

GOLD = os.path.join(os.path.dirname(__file__), "golden")


def _table(name):
    rows = []
    for line in open(os.path.join(GOLD, name)):
        line = line.split("#")[0].strip()
        if line:
            rows.append(line.split())
    return rows


def test_eq3_schedule_matches_worked_values():
    par = {r[0]: float(r[1]) for r in _table("paper_parameters.txt")}
    sched = G.s_min_schedule(par["lambda"], par["rho"], int(par["L_max"]))
    want = [float(r[1]) for r in _table("eq3_smin_worked.txt")]
    assert len(sched) == 5
    np.testing.assert_allclose(sched, want, rtol=0, atol=1e-15)
    # levels below L_max shrink by rho each step
    for a, b in zip(sched[:3], sched[1:4]):
        assert a / b == pytest.approx(par["rho"], rel=1e-14)


def test_eq4_lower_bound_and_plain_3dgs_limit():
    rng = np.random.default_rng(0)
    s_opt = torch.as_tensor(rng.normal(-4, 3, (1000, 3)))
    for s_min in (0.0, 0.003125, 0.5):
        s = G.constrained_scale(s_opt, s_min)
        assert torch.all(s >= s_min)
    # with s_min = 0, Eq. 4 is the plain exponential parameterisation of 3DGS
    assert torch.equal(G.constrained_scale(s_opt, 0.0), torch.exp(s_opt))


def test_eq5_adjust_scale_keeps_scale():
    rng = np.random.default_rng(1)
    s_opt = torch.as_tensor(rng.normal(-4, 0.5, (1000, 3)))
    sched = G.s_min_schedule()
    for l in range(4):
        nxt = G.adjust_scale(s_opt, sched[l], sched[l + 1])
        before = G.constrained_scale(s_opt, sched[l])
        after = G.constrained_scale(nxt, sched[l + 1])
        np.testing.assert_allclose(after.numpy(), before.numpy(), rtol=1e-12, atol=0)


def test_rotation_matches_scipy_and_sign_invariance():
    from scipy.spatial.transform import Rotation
    rng = np.random.default_rng(2)
    q = rng.normal(size=(200, 4)) * rng.uniform(0.2, 3.0, (200, 1))   # unnormalised
    r = G.rotation(torch.as_tensor(q)).numpy()
    ref = Rotation.from_quat(np.concatenate([q[:, 1:], q[:, :1]], 1)).as_matrix()  # x,y,z,w
    np.testing.assert_allclose(r, ref, atol=1e-12)
    np.testing.assert_allclose(G.rotation(torch.as_tensor(-q)).numpy(), r, atol=1e-14)
    eye = np.einsum("nij,nkj->nik", r, r)
    np.testing.assert_allclose(eye, np.broadcast_to(np.eye(3), eye.shape), atol=1e-12)
    np.testing.assert_allclose(np.linalg.det(r), 1.0, atol=1e-12)


def test_eq1_covariance_spectrum():
    rng = np.random.default_rng(3)
    q = torch.as_tensor(rng.normal(size=(300, 4)))
    s = torch.as_tensor(np.exp(rng.normal(-2, 1, (300, 3))))
    cov = G.covariance(q, s).numpy()
    np.testing.assert_allclose(cov, np.transpose(cov, (0, 2, 1)), atol=1e-15)
    ev = np.sort(np.linalg.eigvalsh(cov), axis=1)
    np.testing.assert_allclose(ev, np.sort(s.numpy() ** 2, axis=1), rtol=1e-9, atol=1e-15)
    # eigenvectors are the columns of R: Sigma R e_k = s_k^2 R e_k
    rot = G.rotation(q).numpy()
    for k in range(3):
        v = rot[:, :, k]
        np.testing.assert_allclose(np.einsum("nij,nj->ni", cov, v),
                                   v * (s.numpy()[:, k:k + 1] ** 2), atol=1e-12)


def test_sigmoid_closed_form():
    x = torch.linspace(-20, 20, 101, dtype=torch.float64)
    np.testing.assert_allclose(G.sigmoid(x).numpy(), 0.5 * (1 + np.tanh(x.numpy() / 2)), atol=1e-15)
    assert float(G.sigmoid(torch.tensor(0.0, dtype=torch.float64))) == 0.5
    assert math.isclose(float(G.sigmoid(torch.tensor(math.log(3.0), dtype=torch.float64))), 0.75)
