"""GPU parity, row by row: each step of the registration loop through the C ABI
against the FP64 oracle on the same seeded inputs.

Tolerances: displacements max |diff| <= 1e-3 voxel,
relative loss <= 1e-5, relative gradient (global L2) <= 1e-3.
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


# ---------------------------------------------------------------- a1 pyramid
@pytest.mark.parametrize("shape", [(9, 16, 33), (40, 37, 70), (1, 5, 3)])
def test_downsample(shape):
    rng = np.random.default_rng(1)
    x = rng.uniform(size=(2,) + shape).astype(np.float32)
    out = m.op_downsample(cuda(x)).cpu().numpy()
    for i in range(2):
        ref = oracle.downsample2(x[i])
        assert out[i].shape == ref.shape
        assert np.abs(out[i] - ref).max() < 1e-6


# ---------------------------------------------------------------- a3 scaling and squaring
@pytest.mark.parametrize("shape,K", [((24, 24, 24), 6), ((13, 30, 17), 7), ((33, 9, 40), 0), ((80, 96, 80), 7)])
def test_exp(shape, K):
    phi = phantom.smooth_velocity(shape, 1, seed=2, sigma=3.0, rms=1.2)[0]
    for sign in (1.0, -1.0):
        u = m.op_exp(cuda(phi), K, sign).cpu().numpy()
        ref = oracle.exp(phi, K, sign)
        assert np.abs(u - ref).max() < DISP_TOL


def test_exp_identity_and_translation_exact():
    z = torch.zeros((3, 10, 11, 12), device="cuda")
    assert torch.count_nonzero(m.op_exp(z, 7)) == 0
    c = torch.tensor([0.7, -0.3, 1.1], device="cuda")[:, None, None, None].expand(3, 10, 11, 12).contiguous()
    assert torch.abs(m.op_exp(c, 6) - c).max().item() < 1e-6


# ---------------------------------------------------------------- a6 / a8 similarity and its adjoint
@pytest.mark.parametrize("kind", [m.SILNCC, m.LNCC])
@pytest.mark.parametrize("shape,w", [((20, 21, 40), 3), ((37, 45, 70), 5), ((24, 30, 66), 7), ((30, 26, 35), 9),
                                     ((25, 27, 29), 11), ((6, 40, 9), 5)])
def test_similarity(kind, shape, w):
    series = phantom.blob_series(shape, 2, seed=3)
    F, W = series["images"][0], series["images"][1]
    s, g = m.op_similarity(cuda(F), cuda(W), w, kind, 1e-6)
    so, go = oracle.similarity(F, W, w, kind, 1e-6, grad=True)
    assert abs(s - so) <= LOSS_RTOL * abs(so), (s, so)
    assert rel_l2(g.cpu().numpy(), go) < 1e-4


# widths that are multiples of 4 run the kernels with tensor-memory-accelerator staging;
# ragged heights and depths, windows 3..11, a width of a single copy box and less
@pytest.mark.parametrize("kind", [m.SILNCC, m.LNCC])
@pytest.mark.parametrize("shape,w", [((20, 21, 40), 3), ((37, 45, 72), 5), ((24, 30, 64), 7), ((30, 26, 36), 9),
                                     ((25, 27, 28), 11), ((6, 40, 12), 5), ((13, 9, 4), 3), ((19, 23, 100), 7)])
def test_similarity_staged(kind, shape, w):
    series = phantom.blob_series(shape, 2, seed=5)
    F, W = series["images"][0], series["images"][1]
    s, g = m.op_similarity(cuda(F), cuda(W), w, kind, 1e-6)
    so, go = oracle.similarity(F, W, w, kind, 1e-6, grad=True)
    assert abs(s - so) <= LOSS_RTOL * abs(so), (s, so)
    assert rel_l2(g.cpu().numpy(), go) < 1e-4


def test_similarity_no_window():
    F = torch.rand((4, 20, 20), device="cuda")
    s, g = m.op_similarity(F, F, 5)
    assert s == 0.0 and torch.count_nonzero(g) == 0


# ---------------------------------------------------------------- a3-a5 through the engine
def _ctx(shape, N, **kw):
    base = dict(n_levels=1, steps_per_level=[4], n_squarings=5, window=3, alpha_ss=0.1, alpha_l2=0.01,
                alpha_ts=0.05, lr=0.05)
    base.update(kw)
    return m.Muster(shape, N, **base)


@pytest.mark.parametrize("shape,N,K", [((24, 20, 28), 4, 5), ((17, 33, 12), 3, 0), ((30, 26, 40), 5, 7)])
def test_pair_fields(shape, N, K):
    series = phantom.blob_series(shape, N, seed=4)
    imgs = series["images"]
    with _ctx(shape, N, n_squarings=K) as reg:
        reg.set_images(cuda(imgs))
        reg.set_level(0)
        ni, nf = reg.level_dims(0)
        phi = phantom.smooth_velocity(nf, N - 1, seed=4, sigma=2.0, rms=0.6)
        reg.set_velocity(cuda(phi))
        up = np.stack([oracle.exp(phi[k], K, 1.0) for k in range(N - 1)])
        um = np.stack([oracle.exp(phi[k], K, -1.0) for k in range(N - 1)])
        U = oracle.compose(up, um)
        for i in range(N):
            assert np.abs(reg.get_field(m.IMAGE, i, level=0, device=False) - imgs[i]).max() == 0
            for j in range(N):
                if i == j:
                    continue
                flow = reg.get_field(m.PAIR_FLOW, i, j, level=0, device=False)
                assert np.abs(flow - U[j, i]).max() < DISP_TOL, (i, j)
                disp = reg.get_field(m.PAIR_DISP, i, j, level=0, device=False)
                Ut = oracle.upsample(U[j, i], ni)
                assert np.abs(disp - Ut).max() < 2 * DISP_TOL
                W = reg.get_field(m.WARPED, i, j, level=0, device=False)
                Wo = oracle.warp(imgs[j], Ut)
                assert np.abs(W - Wo).max() < 1e-3


# ---------------------------------------------------------------- a6-a11 loss and gradient
@pytest.mark.parametrize(
    "shape,N,K,w,kind",
    [
        ((20, 22, 24), 2, 0, 3, m.SILNCC),
        ((20, 22, 24), 2, 4, 3, m.SILNCC),
        ((24, 20, 28), 3, 5, 5, m.SILNCC),
        ((18, 26, 21), 4, 6, 3, m.LNCC),
        ((26, 24, 34), 5, 7, 5, m.SILNCC),
    ],
)
def test_loss_and_gradient(shape, N, K, w, kind):
    series = phantom.blob_series(shape, N, seed=5)
    imgs = series["images"]
    times = np.array([0.0, 1.0, 2.5, 3.0, 4.5][:N])
    with _ctx(shape, N, n_squarings=K, window=w, similarity=kind) as reg:
        reg.set_images(cuda(imgs), times=times)
        ni, nf = reg.level_dims(0)
        phi = phantom.smooth_velocity(nf, N - 1, seed=5, sigma=2.0, rms=0.6)
        g = torch.empty((N - 1, 3) + nf, device="cuda")
        loss = reg.eval(cuda(phi), 0, g)
        split = reg.loss_split()
    p = oracle.params(K=K, window=w, sim_kind=kind, alpha_ss=0.1, alpha_l2=0.01, alpha_ts=0.05)
    lo, so, go = oracle.loss_grad(imgs, phi, p, times)
    assert abs(loss - lo) <= LOSS_RTOL * abs(lo), (loss, lo)
    assert abs(split["sim"] - so[0]) <= LOSS_RTOL * abs(so[0])
    for key, ref in zip(("L_ss", "L_L2", "L_ts"), so[1:]):
        assert abs(split[key] - ref) <= 1e-5 * abs(ref) + 1e-12, (key, split[key], ref)
    assert rel_l2(g.cpu().numpy(), go) < GRAD_RTOL


def test_constant_images_isolate_the_regulariser():
    shape, N = (16, 18, 20), 4
    imgs = np.full((N,) + shape, 0.5, np.float32)
    times = np.array([0.0, 1.0, 3.0, 4.0])
    with _ctx(shape, N, alpha_ss=0.7, alpha_l2=0.3, alpha_ts=0.2) as reg:
        reg.set_images(cuda(imgs), times=times)
        ni, nf = reg.level_dims(0)
        phi = phantom.smooth_velocity(nf, N - 1, seed=6, sigma=1.5, rms=0.8)
        g = torch.empty((N - 1, 3) + nf, device="cuda")
        reg.eval(cuda(phi), 0, g)
    L, go = oracle.regulariser(phi, times, (0.7, 0.3, 0.2), grad=True)
    assert rel_l2(g.cpu().numpy(), go) < 1e-5


# ---------------------------------------------------------------- a12 optimiser step
@pytest.mark.parametrize("opt", [m.SGD, m.ADAM])
def test_one_step(opt):
    shape, N = (24, 22, 26), 3
    imgs = phantom.blob_series(shape, N, seed=7)["images"]
    nf = tuple((a + 1) // 2 for a in shape)
    phi = phantom.smooth_velocity(nf, N - 1, seed=7, sigma=2.0, rms=0.5)
    p = oracle.params(K=5, window=3, alpha_ss=0.1, alpha_l2=0.01, alpha_ts=0.05)
    lo, _, go = oracle.loss_grad(imgs, phi, p)
    # SGD: a step large against float32 rounding of phi; Adam: steps of about lr
    T, lr = 5, (0.1 / np.abs(go).max() if opt == m.SGD else 0.2)
    with _ctx(shape, N, optimizer=opt, steps_per_level=[T], lr=lr) as reg:
        reg.set_images(cuda(imgs))
        reg.set_level(0)
        reg.set_velocity(cuda(phi))
        loss = reg.step()
        after = reg.velocities(0, device=False)
    assert abs(loss - lo) <= LOSS_RTOL * abs(lo)
    lr1 = oracle.lr_at(1, T, lr)
    th = phi.astype(np.float64)
    if opt == m.SGD:
        expect = th - lr1 * go
        assert rel_l2(after - th, expect - th) < GRAD_RTOL
    else:
        before = th.copy()
        m1, v1 = np.zeros_like(th), np.zeros_like(th)
        oracle.adam_step(th, m1, v1, go, 1, lr1)
        # Adam's first step moves each entry by lr g/(|g| + eps), about lr sign(g): compare
        # where the gradient is well above its rounding noise
        big = np.abs(go) > 1e-2 * np.abs(go).max()
        assert np.abs(after - th)[big].max() < 1e-3 * lr1
        assert np.abs(after - before).max() <= 1.001 * lr1
