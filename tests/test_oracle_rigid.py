"""Pins of the oracle's rigid registration in parallel (Sec. Rigid Registration)."""
import numpy as np
import pytest

import oracle


def test_rotation_matrix_and_derivatives():
    a = np.array([0.3, -0.2, 0.7])
    R, dR = oracle.rotation(a)

    def rot(k, t):
        c, s = np.cos(t), np.sin(t)
        M = np.eye(3)
        u, w = (k + 1) % 3, (k + 2) % 3
        M[u, u], M[u, w], M[w, u], M[w, w] = c, -s, s, c
        return M

    np.testing.assert_allclose(R, rot(0, a[0]) @ rot(1, a[1]) @ rot(2, a[2]), atol=1e-14)
    np.testing.assert_allclose(R @ R.T, np.eye(3), atol=1e-14)
    assert np.linalg.det(R) == pytest.approx(1.0, abs=1e-14)
    h = 1e-6
    for k in range(3):
        ap, am = a.copy(), a.copy()
        ap[k] += h
        am[k] -= h
        fd = (oracle.rotation(ap)[0] - oracle.rotation(am)[0]) / (2 * h)
        np.testing.assert_allclose(dR[k], fd, atol=1e-8)


def setup(shape=(12, 10, 14), N=3, seed=1):
    rng = np.random.default_rng(seed)
    imgs = np.stack([np.fromfunction(lambda z, y, x: np.sin(0.4 * z + 0.3 * y) + np.cos(0.35 * x - 0.2 * z), shape)
                     for _ in range(N)]) + 0.05 * rng.normal(size=(N,) + shape)
    nf = tuple((a + 1) // 2 for a in shape)
    theta = rng.normal(scale=0.2, size=(N - 1, 3) + nf)
    p = oracle.params(K=3, window=3, alpha_ss=0.1, alpha_l2=0.01, alpha_ts=0.02, rigid=1)
    return imgs, theta, p


def test_zero_rigid_parameters_give_the_plain_loss():
    imgs, theta, p = setup()
    L0, _, g0 = oracle.loss_grad(imgs, theta, p)
    L1, _, g1, gr = oracle.loss_grad_rigid(imgs, theta, np.zeros((2, 6)), p)
    # (p - c) + c - p rounds to 0 only up to the last bits
    assert L1 == pytest.approx(L0, rel=1e-12)
    np.testing.assert_allclose(g1, g0, rtol=1e-9, atol=1e-15)
    assert np.all(np.isfinite(gr))


def test_translation_equals_constant_displacement():
    imgs, _, p = setup(N=2)
    shape = imgs.shape[1:]
    nf = tuple((a + 1) // 2 for a in shape)
    zero = np.zeros((1, 3) + nf)
    t = np.array([0.7, -0.4, 1.3])
    rho = np.zeros((1, 6))
    rho[0, 3:] = t
    L, split, _, _ = oracle.loss_grad_rigid(imgs, zero, rho, p)
    # the same pair terms by hand: session 0 pulled onto grid 1 shifted by t, session 1 onto grid 0 as is
    W = oracle.warp(imgs[0], np.broadcast_to(t[:, None, None, None], (3,) + shape))
    s10 = oracle.similarity(imgs[1], W, 3)
    s01 = oracle.similarity(imgs[0], imgs[1], 3)
    assert split[0] == pytest.approx(s10 + s01, rel=1e-12)


def test_quarter_turn_permutes_a_cube():
    n = 9
    rng = np.random.default_rng(4)
    imgs = rng.random((2, n, n, n))
    nf = ((n + 1) // 2,) * 3
    p = oracle.params(K=2, window=3, alpha_ss=0.0, alpha_l2=0.0, alpha_ts=0.0, rigid=1)
    rho = np.zeros((1, 6))
    rho[0, 0] = np.pi / 2  # rotates the (H, W) plane about the centre: grid points to grid points
    R, _ = oracle.rotation(rho[0, :3])
    c = (n - 1) / 2
    z, y, x = np.meshgrid(*[np.arange(n)] * 3, indexing="ij")
    P = np.stack([z, y, x]).reshape(3, -1) - c
    Q = np.rint(R @ P + c).astype(int)
    W = imgs[0][Q[0], Q[1], Q[2]].reshape(n, n, n)
    L, split, _, _ = oracle.loss_grad_rigid(imgs, np.zeros((1, 3) + nf), rho, p)
    expect = oracle.similarity(imgs[1], W, 3) + oracle.similarity(imgs[0], imgs[1], 3)
    assert split[0] == pytest.approx(expect, rel=1e-12)


@pytest.mark.parametrize("tscale", [1.0, 2.0])
def test_rigid_gradient_by_central_differences(tscale):
    imgs, theta, p = setup(N=3, seed=5)
    rho = np.array([[0.05, -0.03, 0.04, 0.3, -0.2, 0.1], [-0.02, 0.06, 0.01, -0.4, 0.25, 0.5]])
    L, _, g, gr = oracle.loss_grad_rigid(imgs, theta, rho, p, tscale)
    h = 1e-6
    for i in range(2):
        for k in range(6):
            rp, rm = rho.copy(), rho.copy()
            rp[i, k] += h
            rm[i, k] -= h
            fd = (oracle.loss_grad_rigid(imgs, theta, rp, p, tscale)[0] - oracle.loss_grad_rigid(imgs, theta, rm, p, tscale)[0]) / (2 * h)
            assert fd == pytest.approx(gr[i, k], rel=2e-4, abs=1e-7), (i, k)
    # the theta gradient with rigid parameters, one entry
    idx = (1, 2, 3, 2, 4)
    tp, tm = theta.copy(), theta.copy()
    tp[idx] += h
    tm[idx] -= h
    fd = (oracle.loss_grad_rigid(imgs, tp, rho, p, tscale)[0] - oracle.loss_grad_rigid(imgs, tm, rho, p, tscale)[0]) / (2 * h)
    assert fd == pytest.approx(g[idx], rel=2e-4, abs=1e-7)


def test_run_with_rigid_moves_parameters_and_decreases_loss():
    imgs, _, p = setup(N=3, seed=6)
    shape = imgs.shape[1:]
    p2 = oracle.params(n_levels=1, steps=(6,), K=3, window=3, alpha_ss=0.1, alpha_l2=0.01, rigid=1, rigid_lr=0.2,
                       lr=0.05)
    loss, theta, hist, rho = oracle.run(imgs, p2, loss_history=True)
    assert rho.shape == (2, 6) and np.abs(rho).max() > 0
    assert hist[-1] < hist[0]
