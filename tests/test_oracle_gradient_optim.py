"""Oracle pins: the hand-written adjoint against FP64 central differences of the
total loss (Sec. MUSTER overview), adjoint identities of the nonlinear pieces,
and the optimiser (Sec. Implementation Details)."""
import json
import os

import numpy as np
import pytest
import scipy.ndimage
import torch

import oracle

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


def _smooth(rng, shape, sigma, scale):
    x = scipy.ndimage.gaussian_filter(rng.normal(size=shape), sigma)
    return x * (scale / x.std())


def _problem(N, ni, seed, phi_scale=0.6):
    rng = np.random.default_rng(seed)
    base = _smooth(rng, ni, 1.5, 0.2) + 0.5
    imgs = np.stack([base + 0.05 * _smooth(rng, ni, 1.0, 1.0) for _ in range(N)])
    nf = tuple((a + 1) // 2 for a in ni)
    phi = np.stack([np.stack([_smooth(rng, nf, 1.0, phi_scale) for _ in range(3)]) for _ in range(N - 1)])
    return imgs, phi


@pytest.mark.parametrize(
    "N,kind,K,w",
    [(2, oracle.SILNCC, 3, 3), (3, oracle.SILNCC, 3, 3), (4, oracle.LNCC, 2, 3), (3, oracle.LNCC, 4, 5)],
)
def test_total_gradient_central_differences(N, kind, K, w):
    ni = (12, 13, 11)
    imgs, phi = _problem(N, ni, seed=20 + N + K)
    p = oracle.params(K=K, window=w, sim_kind=kind, alpha_ss=0.05, alpha_l2=0.01, alpha_ts=0.02)
    t = np.array([0.0, 1.0, 2.5, 3.0][:N])
    tot, split, g = oracle.loss_grad(imgs, phi, p, t)
    assert abs(tot - (split[0] + 0.05 * split[1] + 0.01 * split[2] + 0.02 * split[3])) < 1e-14
    rng = np.random.default_rng(30 + N)
    h = 1e-6
    scale = np.abs(g).max()
    for _ in range(24):
        idx = tuple(rng.integers(0, a) for a in phi.shape)
        pp, pm = phi.copy(), phi.copy()
        pp[idx] += h
        pm[idx] -= h
        fd = (oracle.loss_grad(imgs, pp, p, t, grad=False)[0] - oracle.loss_grad(imgs, pm, p, t, grad=False)[0]) / (2 * h)
        assert abs(fd - g[idx]) < 1e-6 * scale + 1e-6 * abs(fd), (idx, fd, g[idx], scale)


def test_exp_adjoint_matches_directional_derivative():
    rng = np.random.default_rng(40)
    n = (7, 8, 6)
    phi = _smooth(rng, (3,) + n, 1.0, 0.8)
    gu = rng.normal(size=phi.shape)
    d = rng.normal(size=phi.shape)
    h = 1e-6
    for sign in (1.0, -1.0):
        fd = ((oracle.exp(phi + h * d, 4, sign) - oracle.exp(phi - h * d, 4, sign)) * gu).sum() / (2 * h)
        adj = (oracle.exp_adjoint(phi, 4, sign, gu) * d).sum()
        assert abs(fd - adj) < 1e-6 * max(1.0, abs(fd)), (sign, fd, adj)


def test_compose_adjoint_matches_directional_derivative():
    rng = np.random.default_rng(41)
    N, n = 4, (6, 7, 5)
    up = _smooth(rng, (N - 1, 3) + n, 1.0, 0.7)
    um = _smooth(rng, (N - 1, 3) + n, 1.0, 0.7)
    gU = rng.normal(size=(N, N, 3) + n)
    for i in range(N):
        gU[i, i] = 0
    dp, dm = rng.normal(size=up.shape), rng.normal(size=um.shape)
    h = 1e-6
    fd = ((oracle.compose(up + h * dp, um + h * dm) - oracle.compose(up - h * dp, um - h * dm)) * gU).sum() / (2 * h)
    g_up, g_um = oracle.compose_adjoint(up, um, gU)
    adj = (g_up * dp).sum() + (g_um * dm).sum()
    assert abs(fd - adj) < 1e-6 * max(1.0, abs(fd)), (fd, adj)


def test_adam_matches_torch_optim():
    rng = np.random.default_rng(42)
    theta = rng.normal(size=1000)
    m, v = np.zeros_like(theta), np.zeros_like(theta)
    tt = torch.tensor(theta.copy(), dtype=torch.float64, requires_grad=True)
    opt = torch.optim.Adam([tt], lr=0.05, betas=(0.9, 0.999), eps=1e-8)
    for step in range(1, 8):
        g = rng.normal(size=theta.shape) * 10.0 ** rng.uniform(-9, 0, size=theta.shape)
        oracle.adam_step(theta, m, v, g, step, 0.05)
        tt.grad = torch.tensor(g, dtype=torch.float64)
        opt.step()
    assert np.abs(theta - tt.detach().numpy()).max() < 1e-12


def test_lr_schedule_closed_form():
    sch = json.load(open(os.path.join(GOLDEN, "paper_schedule.json")))
    T = 100
    Wu = int(np.ceil(sch["warmup_frac"] * T))
    assert Wu == 20
    assert abs(oracle.lr_at(1, T, 0.1) - 0.1 / 20) < 1e-15
    assert abs(oracle.lr_at(20, T, 0.1) - 0.1) < 1e-15
    assert abs(oracle.lr_at(60, T, 0.1) - 0.05) < 1e-15  # half-way through the cosine
    assert abs(oracle.lr_at(T, T, 0.1)) < 1e-15
    lrs = [oracle.lr_at(s, T, 0.1) for s in range(1, T + 1)]
    assert np.all(np.diff(lrs[:20]) > 0) and np.all(np.diff(lrs[19:]) < 0)
