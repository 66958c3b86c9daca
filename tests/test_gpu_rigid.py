"""GPU parity of rigid registration in parallel with the deformable one (Sec. Rigid
Registration) against the oracle: loss and gradients with given rigid parameters at the
finest and a coarser level, the warped images and total displacements of a rotated and
translated session, a multi-level trajectory, and checkpoint / resume."""
import numpy as np
import pytest
import torch

import oracle
import paper_2412_14671_gb300 as m
from paper_2412_14671_gb300 import phantom

pytestmark = pytest.mark.gpu


def cuda(x):
    return torch.from_numpy(np.ascontiguousarray(x, dtype=np.float32)).cuda()


def rel_l2(a, b):
    return float(np.linalg.norm(np.asarray(a, np.float64) - b) / max(np.linalg.norm(b), 1e-300))


KW = dict(n_squarings=4, window=3, alpha_ss=0.1, alpha_l2=0.01, alpha_ts=0.02)
RHO = np.array([[0.04, -0.03, 0.05, 0.6, -0.4, 0.3], [-0.02, 0.05, 0.01, -0.5, 0.8, 0.2]])


@pytest.mark.parametrize("n_levels,level", [(1, 0), (2, 0), (2, 1)])
def test_rigid_loss_and_gradients_match_oracle(n_levels, level):
    shape, N = (26, 22, 30), 3
    imgs = phantom.blob_series(shape, N, seed=9)["images"]
    with m.Muster(shape, N, n_levels=n_levels, steps_per_level=[2] * n_levels, rigid=1, **KW) as reg:
        reg.set_images(cuda(imgs))
        reg.set_level(level)
        reg.set_rigid(RHO)
        ni, nf = reg.level_dims(level)
        theta = phantom.smooth_velocity(nf, N - 1, seed=9, sigma=1.5, rms=0.5)
        g = torch.empty_like(cuda(theta))
        loss = reg.eval(cuda(theta), level, g)
        rho, grho = reg.rigid(grad=True)
        lv = np.stack([reg.get_field(m.IMAGE, i, level=level, device=False) for i in range(N)])
    np.testing.assert_allclose(rho, RHO.astype(np.float32), rtol=0, atol=0)
    p = oracle.params(K=4, window=3, alpha_ss=0.1, alpha_l2=0.01, alpha_ts=0.02, rigid=1)
    lo, _, go, gro = oracle.loss_grad_rigid(lv, theta, RHO.astype(np.float32), p, tscale=2.0 ** (n_levels - 1 - level))
    assert abs(loss - lo) <= 1e-5 * abs(lo)
    assert rel_l2(g.cpu().numpy(), go) < 1e-3
    assert rel_l2(grho, gro) < 1e-3, (grho, gro)


def test_rotated_and_translated_fields():
    shape, N = (24, 24, 28), 2
    imgs = phantom.blob_series(shape, N, seed=10)["images"]
    rho = np.array([[np.pi / 2, 0.0, 0.0, 0.5, -1.25, 2.0]])
    with m.Muster(shape, N, n_levels=1, steps_per_level=[1], rigid=1, **KW) as reg:
        reg.set_images(cuda(imgs))
        reg.set_level(0)
        reg.set_rigid(rho)
        ni, nf = reg.level_dims(0)
        W = reg.get_field(m.WARPED, 1, 0, level=0, device=False)  # image 0 pulled onto grid 1
        disp = reg.get_field(m.PAIR_DISP, 1, 0, level=0, device=False)
    R, _ = oracle.rotation(rho[0, :3].astype(np.float32))
    c = (np.array(ni) - 1) / 2.0
    P = np.stack(np.meshgrid(*[np.arange(a) for a in ni], indexing="ij")).reshape(3, -1).astype(np.float64)
    r = (R @ (P - c[:, None]) + c[:, None] + rho[0, 3:, None] - P).reshape((3,) + tuple(ni))
    assert np.abs(disp - r).max() < 1e-4  # zero velocities: the rigid part only
    Wo = oracle.warp(imgs[0], r)
    assert np.abs(W - Wo).max() < 1e-4


def test_rigid_trajectory_matches_oracle():
    shape, N = (28, 24, 32), 3
    imgs = phantom.blob_series(shape, N, seed=11)["images"]
    steps = (4, 3)
    p = oracle.params(n_levels=2, steps=steps, K=4, window=3, alpha_ss=0.1, alpha_l2=0.01, alpha_ts=0.02,
                      optimizer=oracle.SGD, lr=0.2, rigid=1, rigid_lr=0.3)
    loss_o, theta_o, hist_o, rho_o = oracle.run(imgs, p, loss_history=True)
    with m.Muster(shape, N, n_levels=2, steps_per_level=list(steps), optimizer=m.SGD, lr=0.2, rigid=1, rigid_lr=0.3,
                  **KW) as reg:
        reg.set_images(cuda(imgs))
        loss = reg.run()
        hist = reg.loss_history()
        rho = reg.rigid()
        theta = np.stack([reg.get_field(m.PARAMETERS, k, level=1, device=False) for k in range(N - 1)])
    assert np.abs(rho_o).max() > 1e-3  # the rigid parameters moved
    assert np.abs(hist - hist_o).max() <= 1e-4 * np.abs(hist_o).max()
    assert abs(loss - loss_o) <= 1e-4 * abs(loss_o)
    assert np.abs(theta - theta_o).max() < 1e-3
    assert np.abs(rho - rho_o).max() < 1e-3 * max(1.0, np.abs(rho_o).max())


def test_rigid_checkpoint_resume_is_bitwise():
    shape, N = (20, 22, 24), 3
    imgs = phantom.blob_series(shape, N, seed=12)["images"]
    kw = dict(KW, n_levels=2, steps_per_level=[3, 4], rigid=1, rigid_lr=0.3, deterministic=1)
    with m.Muster(shape, N, **kw) as a:
        a.set_images(cuda(imgs))
        a.run()
        ref_rho = a.rigid()
        ref_v = a.velocities(1, device=False)
    with m.Muster(shape, N, **kw) as b:
        b.set_images(cuda(imgs))
        b.set_level(0)
        for _ in range(3):
            b.step()
        b.set_level(1)
        b.step()
        state = b.get_state()
    with m.Muster(shape, N, **kw) as c:
        c.set_images(cuda(imgs))
        c.set_state(state)
        for _ in range(3):
            c.step()
        assert np.array_equal(c.rigid(), ref_rho)
        assert np.array_equal(c.velocities(1, device=False), ref_v)
