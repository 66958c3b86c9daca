"""GPU parity of the Gaussian parameterisation (Sec. Regularization; Appendix Gaussian
Smoothing): phi = S(theta), the loss at phi and the gradient with respect to theta, the
smoothed velocity field and a multi-level trajectory, against the oracle."""
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


# omega 0.15 / mm keeps a few taps on the 2 mm flow grid; omega 0.02 / mm spreads the kernel
# over the whole (periodic) axis, so the full circle is summed
@pytest.mark.parametrize("omega,spacing", [(0.15, (1.0, 1.0, 1.0)), (0.02, (1.0, 1.2, 0.9)), (0.3, (0.7, 0.7, 0.7))])
def test_smoothed_loss_gradient_and_velocity(omega, spacing):
    shape, N = (24, 20, 28), 3
    imgs = phantom.blob_series(shape, N, seed=6)["images"]
    kw = dict(n_squarings=5, window=3, alpha_ss=0.1, alpha_l2=0.01, alpha_ts=0.05)
    with m.Muster(shape, N, spacing=spacing, smooth_omega=omega, **kw) as reg:
        reg.set_images(cuda(imgs))
        reg.set_level(0)
        ni, nf = reg.level_dims(0)
        theta = phantom.smooth_velocity(nf, N - 1, seed=6, sigma=1.0, rms=0.8)
        g = torch.empty_like(cuda(theta))
        loss = reg.eval(cuda(theta), 0, g)
        p = oracle.params(K=5, window=3, alpha_ss=0.1, alpha_l2=0.01, alpha_ts=0.05, smooth_omega=omega,
                          spacing=spacing)
        lo, _, go = oracle.loss_grad(imgs, theta, p)
        assert abs(loss - lo) <= 1e-5 * abs(lo)
        assert rel_l2(g.cpu().numpy(), go) < 1e-3
        # fields: parameters as set, velocity = S(theta) on the 2x coarser (periodic) flow grid
        reg.set_velocity(cuda(theta))
        h = tuple(2 * a for a in spacing)
        for k in range(N - 1):
            assert np.array_equal(reg.get_field(m.PARAMETERS, k, level=0, device=False), theta[k].astype(np.float32))
            v = reg.get_field(m.VELOCITY, k, level=0, device=False)
            vo = np.stack([oracle.smooth(theta[k, c], omega, h) for c in range(3)])
            assert np.abs(v - vo).max() < 1e-5 * max(1.0, np.abs(vo).max())


def test_smoothed_multilevel_trajectory_matches_oracle():
    shape, N = (28, 24, 32), 3
    imgs = phantom.blob_series(shape, N, seed=8)["images"]
    steps = (4, 3)
    p = oracle.params(n_levels=2, steps=steps, K=4, window=3, alpha_ss=0.1, alpha_l2=0.01, alpha_ts=0.0,
                      optimizer=oracle.SGD, lr=0.2, smooth_omega=0.1, spacing=(1.0, 1.0, 1.0))
    loss_o, theta_o, hist_o = oracle.run(imgs, p, loss_history=True)
    with m.Muster(shape, N, n_levels=2, steps_per_level=list(steps), n_squarings=4, window=3, alpha_ss=0.1,
                  alpha_l2=0.01, alpha_ts=0.0, optimizer=m.SGD, lr=0.2, smooth_omega=0.1) as reg:
        reg.set_images(cuda(imgs))
        loss = reg.run()
        hist = reg.loss_history()
        theta = np.stack([reg.get_field(m.PARAMETERS, k, level=1, device=False) for k in range(N - 1)])
    assert np.abs(hist - hist_o).max() <= 1e-4 * np.abs(hist_o).max()
    assert abs(loss - loss_o) <= 1e-4 * abs(loss_o)
    assert np.abs(theta - theta_o).max() < 1e-3
