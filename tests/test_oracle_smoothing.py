"""Pins of the oracle's Gaussian parameterisation (Sec. Regularization; Appendix Gaussian
Smoothing): phi = S(theta) with S the multiplication of the DFT by exp(-1/2 (f/omega)^2)."""
import numpy as np
import pytest

import oracle


def response(n, h, omega):
    f = np.fft.fftfreq(n, d=h)
    return np.exp(-0.5 * (f / omega) ** 2)


@pytest.mark.parametrize("shape,h,omega", [((8, 9, 10), (1.0, 1.0, 1.0), 0.15), ((5, 12, 7), (2.0, 1.5, 1.0), 0.1),
                                           ((1, 6, 4), (1.0, 1.0, 1.0), 0.3)])
def test_smoothing_matches_numpy_fft(shape, h, omega):
    rng = np.random.default_rng(1)
    x = rng.normal(size=shape)
    H = response(shape[0], h[0], omega)[:, None, None] * response(shape[1], h[1], omega)[None, :, None] * \
        response(shape[2], h[2], omega)[None, None, :]
    ref = np.real(np.fft.ifftn(np.fft.fftn(x) * H))
    np.testing.assert_allclose(oracle.smooth(x, omega, h), ref, atol=1e-12)


def test_single_mode_and_constant():
    shape, h, omega = (6, 8, 12), (1.0, 2.0, 0.5), 0.2
    z, y, x = np.meshgrid(*[np.arange(a) for a in shape], indexing="ij")
    k = 3  # along W: frequency k / (n h) cycles per mm
    mode = np.cos(2 * np.pi * k * x / shape[2])
    expect = np.exp(-0.5 * (k / (shape[2] * h[2]) / omega) ** 2) * mode
    np.testing.assert_allclose(oracle.smooth(mode, omega, h), expect, atol=1e-12)
    np.testing.assert_allclose(oracle.smooth(np.full(shape, 2.5), omega, h), 2.5, atol=1e-12)


def test_smoothing_is_symmetric():
    rng = np.random.default_rng(2)
    shape, h, omega = (7, 6, 9), (1.0, 1.0, 2.0), 0.12
    a, b = rng.normal(size=shape), rng.normal(size=shape)
    assert np.sum(oracle.smooth(a, omega, h) * b) == pytest.approx(np.sum(a * oracle.smooth(b, omega, h)), rel=1e-12)


def test_smoothed_loss_gradient_is_the_theta_gradient():
    shape, N = (12, 10, 14), 3
    rng = np.random.default_rng(3)
    imgs = rng.random((N,) + shape)
    nf = tuple((a + 1) // 2 for a in shape)
    theta = rng.normal(scale=0.3, size=(N - 1, 3) + nf)
    p = oracle.params(K=3, window=3, alpha_ss=0.1, alpha_l2=0.01, alpha_ts=0.05, smooth_omega=0.2,
                      spacing=(1.0, 1.2, 0.9))
    L, _, g = oracle.loss_grad(imgs, theta, p)
    # the smoothed loss equals the plain loss at phi = S(theta)
    h = (2.0, 2.4, 1.8)
    phi = np.stack([[oracle.smooth(theta[m, c], 0.2, h) for c in range(3)] for m in range(N - 1)])
    p0 = oracle.params(K=3, window=3, alpha_ss=0.1, alpha_l2=0.01, alpha_ts=0.05)
    L0, _, _ = oracle.loss_grad(imgs, phi, p0)
    assert L == pytest.approx(L0, rel=1e-12)
    eps = 1e-5
    for idx in [(0, 0, 2, 3, 4), (1, 2, 5, 1, 6), (0, 1, 0, 4, 0)]:
        tp, tm = theta.copy(), theta.copy()
        tp[idx] += eps
        tm[idx] -= eps
        fd = (oracle.loss_grad(imgs, tp, p)[0] - oracle.loss_grad(imgs, tm, p)[0]) / (2 * eps)
        assert fd == pytest.approx(g[idx], rel=1e-5, abs=1e-9)
