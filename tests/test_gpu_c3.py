"""Differentiation check at its full size: 6 sessions of 128^3 brain-like phantoms,
K = 7, w = 7, SiLNCC. The autograd.Function over the hand-written adjoint against the
FP64 oracle gradient (loss 1e-5, gradient 1e-3 relative) and against central
differences (h = 1e-3) of the GPU loss on 64 flow voxels; squaring intermediates
recomputed give the stored ones' gradient bit for bit (deterministic adjoint)."""
import numpy as np
import pytest
import torch

import oracle
import paper_2412_14671_gb300 as m
from paper_2412_14671_gb300 import phantom

pytestmark = pytest.mark.gpu

SHAPE, N = (128, 128, 128), 6
P = dict(n_squarings=7, window=7, alpha_ss=0.05, alpha_l2=0.005, alpha_ts=0.01)


@pytest.fixture(scope="module")
def problem():
    imgs = phantom.cached("brain_series", shape=SHAPE, n_sessions=N, seed=3)["images"]
    nf = tuple((a + 1) // 2 for a in SHAPE)
    phi = phantom.smooth_velocity(nf, N - 1, seed=3, sigma=3.0, rms=0.6)
    return imgs, phi


def test_c3_gradient_matches_oracle_and_central_differences(problem):
    imgs, phi_h = problem
    p = oracle.params(n_levels=1, steps=(1,), K=7, window=7, alpha_ss=0.05, alpha_l2=0.005, alpha_ts=0.01)
    lo, _, go = oracle.loss_grad(imgs, phi_h, p)
    with m.Muster(SHAPE, N, **P) as reg:
        reg.set_images(torch.from_numpy(imgs).cuda())
        phi = torch.from_numpy(phi_h).cuda()
        v = phi.clone().requires_grad_(True)
        L = m.MusterLoss.apply(v, reg, 0)
        L.backward()
        g = v.grad.cpu().numpy().astype(np.float64)
        assert abs(L.item() - lo) <= 1e-5 * abs(lo)
        assert np.linalg.norm(g - go) <= 1e-3 * np.linalg.norm(go)
        # central differences of the float32 GPU loss on 64 entries with |g| >= 0.1 max|g|
        rng = np.random.default_rng(3)
        h, gs, errs = 1e-3, np.abs(g).max(), []
        for _ in range(2000):
            if len(errs) == 64:
                break
            idx = tuple(int(rng.integers(0, s)) for s in phi.shape)
            if abs(g[idx]) < 0.1 * gs:
                continue
            pp, pm = phi.clone(), phi.clone()
            pp[idx] += h
            pm[idx] -= h
            fd = (reg.eval(pp, 0) - reg.eval(pm, 0)) / (2 * h)
            errs.append(abs(fd - g[idx]) / abs(g[idx]))
        assert len(errs) == 64
        assert np.median(errs) < 1e-2 and max(errs) < 0.1, errs


def test_c3_recomputed_squarings_bitwise(problem):
    imgs, phi_h = problem
    phi = torch.from_numpy(phi_h).cuda()
    grads = []
    for rec in (0, 1):
        with m.Muster(SHAPE, N, recompute_squaring=rec, deterministic=1, **P) as reg:
            reg.set_images(torch.from_numpy(imgs).cuda())
            g = torch.empty_like(phi)
            reg.eval(phi, 0, g)
            grads.append(g)
    assert torch.equal(grads[0], grads[1])


def test_c3_central_differences_on_64_uniform_random_entries(problem):
    """64 entries drawn uniformly over the flow grid and the 3 components (no magnitude
    filter): every central difference (h = 1e-3) of the float32 GPU loss agrees with the
    adjoint to 1 % of the largest gradient entry, and the entries above 1e-3 of it to a
    median relative error below 2 %."""
    imgs, phi_h = problem
    with m.Muster(SHAPE, N, deterministic=1, **P) as reg:
        reg.set_images(torch.from_numpy(imgs).cuda())
        phi = torch.from_numpy(phi_h).cuda()
        g_t = torch.empty_like(phi)
        reg.eval(phi, 0, g_t)
        g = g_t.cpu().numpy().astype(np.float64)
        gmax = np.abs(g).max()
        rng = np.random.default_rng(33)
        h, abs_err, rel = 1e-3, [], []
        for _ in range(64):
            idx = tuple(int(rng.integers(0, s)) for s in phi.shape)
            pp, pm = phi.clone(), phi.clone()
            pp[idx] += h
            pm[idx] -= h
            fd = (reg.eval(pp, 0) - reg.eval(pm, 0)) / (2 * h)
            abs_err.append(abs(fd - g[idx]))
            if abs(g[idx]) > 1e-3 * gmax:
                rel.append(abs(fd - g[idx]) / abs(g[idx]))
    assert max(abs_err) <= 1e-2 * gmax, (max(abs_err), gmax)
    assert len(rel) >= 16 and np.median(rel) < 2e-2, rel
