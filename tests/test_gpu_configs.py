"""GPU parity at the settings of the large-series and session-count workloads, through
the C ABI against the FP64 oracle: K = 8 squarings (Alg. 1) on the 128^3 flow grid of
16 x 256^3 series, the 9^3 window with recomputed squaring intermediates, and the
loss and gradient of 10, 12 and 16 sessions (every ordered pair of the sum of
Sec. MUSTER overview), and the loss and gradient of the full 10 x 160x192x160 series at its
finest level.

Tolerances: displacements max |diff| <= 1e-3 voxel, relative loss <= 1e-5, relative
gradient (global L2) <= 1e-3.
"""
import numpy as np
import pytest
import torch

import oracle
import paper_2412_14671_gb300 as m
from paper_2412_14671_gb300 import phantom

pytestmark = pytest.mark.gpu

DISP_TOL = 1e-3
LOSS_RTOL = 1e-5
GRAD_RTOL = 1e-3


def cuda(x):
    return torch.from_numpy(np.ascontiguousarray(x, dtype=np.float32)).cuda()


def rel_l2(a, b):
    return float(np.linalg.norm(np.asarray(a, np.float64) - b) / max(np.linalg.norm(b), 1e-300))


@pytest.mark.parametrize("shape", [(128, 128, 128), (37, 45, 29)])
def test_exp_eight_squarings(shape):
    phi = phantom.smooth_velocity(shape, 1, seed=21, sigma=4.0, rms=1.5)[0]
    for sign in (1.0, -1.0):
        u = m.op_exp(cuda(phi), 8, sign).cpu().numpy()
        ref = oracle.exp(phi, 8, sign)
        assert np.abs(u - ref).max() < DISP_TOL


def _eval(shape, N, phi, imgs, **kw):
    with m.Muster(shape, N, **kw) as reg:
        reg.set_images(cuda(imgs))
        g = torch.empty((N - 1, 3) + phi.shape[2:], device="cuda")
        loss = reg.eval(cuda(phi), 0, g)
        split = reg.loss_split()
    return loss, g.cpu().numpy(), split


@pytest.mark.parametrize("det", [0, 1])
def test_large_series_settings_K8_w9_recompute(det):
    """K = 8, w = 9, SiLNCC and recomputed squaring intermediates (the settings of the
    16 x 256^3 series) on 3 x 40^3: loss and gradient against the oracle; in the
    deterministic mode the recomputed and stored intermediates give the same bits."""
    shape, N = (40, 40, 40), 3
    imgs = phantom.brain_series(shape, N, seed=22)["images"]
    nf = tuple((a + 1) // 2 for a in shape)
    phi = phantom.smooth_velocity(nf, N - 1, seed=22, sigma=2.0, rms=0.7)
    kw = dict(n_squarings=8, window=9, alpha_ss=0.1, alpha_l2=0.01, alpha_ts=0.05, deterministic=det)
    loss, g, split = _eval(shape, N, phi, imgs, recompute_squaring=1, **kw)
    p = oracle.params(K=8, window=9, alpha_ss=0.1, alpha_l2=0.01, alpha_ts=0.05)
    lo, so, go = oracle.loss_grad(imgs, phi, p)
    assert abs(loss - lo) <= LOSS_RTOL * abs(lo), (loss, lo)
    assert abs(split["sim"] - so[0]) <= LOSS_RTOL * abs(so[0])
    assert rel_l2(g, go) < GRAD_RTOL
    if det:
        loss2, g2, _ = _eval(shape, N, phi, imgs, recompute_squaring=0, **kw)
        assert loss2 == loss and np.array_equal(g2, g)


@pytest.mark.parametrize("shape,N,K,w", [((80, 96, 80), 10, 7, 7), ((20, 18, 22), 12, 7, 5), ((14, 16, 18), 16, 8, 3)])
def test_many_sessions_loss_and_gradient(shape, N, K, w):
    """10 sessions on the 80 x 96 x 80 grid (the second-finest level of the 10 x
    160x192x160 series, 90 ordered pairs), 12 sessions (the end of the session-count
    sweep) and 16 sessions (240 pairs)."""
    gen = phantom.brain_series if shape[0] >= 64 else phantom.blob_series
    imgs = gen(shape, N, seed=23)["images"]
    nf = tuple((a + 1) // 2 for a in shape)
    phi = phantom.smooth_velocity(nf, N - 1, seed=23, sigma=2.0, rms=0.6)
    t = np.cumsum(np.r_[0.0, np.linspace(0.8, 1.6, N - 1)])
    kw = dict(n_squarings=K, window=w, alpha_ss=0.1, alpha_l2=0.01, alpha_ts=0.05)
    with m.Muster(shape, N, **kw) as reg:
        reg.set_images(cuda(imgs), times=t)
        g = torch.empty((N - 1, 3) + nf, device="cuda")
        loss = reg.eval(cuda(phi), 0, g)
    p = oracle.params(K=K, window=w, alpha_ss=0.1, alpha_l2=0.01, alpha_ts=0.05)
    lo, _, go = oracle.loss_grad(imgs, phi, p, t)
    assert abs(loss - lo) <= LOSS_RTOL * abs(lo), (loss, lo)
    assert rel_l2(g.cpu().numpy(), go) < GRAD_RTOL


def test_full_size_series_loss_and_gradient_both_modes():
    """The 10 x 160x192x160 series at its finest level with the registration settings
    of the throughput measurement (K = 7, w = 7, SiLNCC, alpha_ss 0.05, alpha_l2 0.005,
    all 90 ordered pairs in the context's pair batches): loss and gradient against the
    oracle, with the atomic and with the deterministic adjoint."""
    shape, N = (160, 192, 160), 10
    imgs = phantom.cached("brain_series", shape=shape, n_sessions=N, seed=0)["images"]
    nf = (80, 96, 80)
    phi = phantom.smooth_velocity(nf, N - 1, seed=31, sigma=3.0, rms=0.6)
    kw = dict(n_levels=4, n_squarings=7, window=7, similarity=m.SILNCC, alpha_ss=0.05, alpha_l2=0.005,
              alpha_ts=0.0)
    out = {}
    for det in (0, 1):
        with m.Muster(shape, N, deterministic=det, **kw) as reg:
            reg.set_images(cuda(imgs))
            top = 3  # levels run coarse to fine: the finest of the four
            ni, nfl = reg.level_dims(top)
            assert tuple(ni) == shape and tuple(nfl) == nf
            g = torch.empty((N - 1, 3) + nf, device="cuda")
            loss = reg.eval(cuda(phi), top, g)
            out[det] = (loss, g.cpu().numpy())
    p = oracle.params(K=7, window=7, alpha_ss=0.05, alpha_l2=0.005, alpha_ts=0.0)
    lo, _, go = oracle.loss_grad(imgs, phi, p)
    for det, (loss, g) in out.items():
        assert abs(loss - lo) <= LOSS_RTOL * abs(lo), (det, loss, lo)
        assert rel_l2(g, go) < GRAD_RTOL, (det, rel_l2(g, go))
