"""Pins of the oracle's multi-level driver (or_run / or_run_rigid).

The driver follows the stage schedule of Sec. Implementation Details: a pyramid of
images, one stage per level from the coarsest, the velocities of a stage initialised
by interpolating those of the previous one, Adam with a linear warm-up over the first
20 % of the stage's iterations and a cosine decay after it. The readings the driver
adds (Adam state and schedule restarted at every level, steps counted from 1 within a
level, the Gaussian taps built with the level's own voxel size, the rigid parameters
kept across levels with their step sizes scaled to `rigid_lr` voxels and `rigid_lr` /
half the largest extent radians) are restated here from their definitions, each step
taken by code that does not call the driver:

  pyramid      numpy 2x2x2 block means of the edge-padded volume
  prolong      2 x scipy.ndimage.map_coordinates(order=1, mode='nearest') at
               (y + 1/2)/2 - 1/2 (clamp-to-edge trilinear, voxel-centre aligned)
  schedule     the closed form lr t/W, then lr (1 + cos(pi (t - W)/(T - W)))/2
  optimiser    torch.optim.Adam in float64, a fresh optimiser per level
  loss, grad   oracle.loss_grad / loss_grad_rigid at one level (pinned by central
               differences and closed forms in the other oracle tests)

The driver's loss history and final parameters must agree to rounding.
"""
import math

import numpy as np
import pytest
import scipy.ndimage
import torch

import oracle


def down2(I):
    pad = [(0, a % 2) for a in I.shape]
    P = np.pad(I, pad, mode="edge")
    d, h, w = (a // 2 for a in P.shape)
    return P.reshape(d, 2, h, 2, w, 2).mean(axis=(1, 3, 5))


def prolong(v, nf):
    coords = np.meshgrid(*[(np.arange(n) + 0.5) / 2.0 - 0.5 for n in nf], indexing="ij")
    return np.stack([2.0 * scipy.ndimage.map_coordinates(v[c], coords, order=1, mode="nearest") for c in range(3)])


def lr_closed_form(t, T, lr, warmup_frac):
    W = max(1, math.ceil(warmup_frac * T))
    if t <= W:
        return lr * t / W
    return lr * 0.5 * (1.0 + math.cos(math.pi * (t - W) / (T - W)))


def level_shapes(n, L):
    shapes = [tuple(n)]
    for _ in range(L - 1):
        shapes.append(tuple((a + 1) // 2 for a in shapes[-1]))
    return shapes[::-1]  # coarsest first


def run_by_hand(imgs, kw, rigid=False, mistake=None):
    """The multi-level schedule restated step by step (see the module docstring).
    mistake (tests only): 'global_step' indexes the schedule by the step count over all
    levels, 'from_zero' starts each level's step counter at 0."""
    N = imgs.shape[0]
    L = kw["n_levels"]
    shapes = level_shapes(imgs.shape[1:], L)
    pyr = [imgs]
    for _ in range(L - 1):
        pyr.append(np.stack([down2(I) for I in pyr[-1]]))
    pyr = pyr[::-1]
    finest = imgs.shape[1:]
    rmax = 0.5 * max(finest)
    theta = None
    rho = np.zeros((N - 1, 6))
    hist = []
    done = 0
    total = sum(kw["steps"][:L])
    for l in range(L):
        ni = shapes[l]
        nf = tuple((a + 1) // 2 for a in ni)
        if theta is None:
            theta = np.zeros((N - 1, 3) + nf)
        else:
            theta = np.stack([prolong(theta[m], nf) for m in range(N - 1)])
        f = 2 ** (L - 1 - l)  # finest voxels per voxel of this level
        spacing = tuple(s * f for s in kw.get("spacing", (1.0, 1.0, 1.0)))
        p = oracle.params(**{**kw, "spacing": spacing})
        T = kw["steps"][l]
        th = torch.tensor(theta, dtype=torch.float64, requires_grad=True)
        ang = torch.tensor(rho[:, :3].copy(), dtype=torch.float64, requires_grad=True)
        tra = torch.tensor(rho[:, 3:].copy(), dtype=torch.float64, requires_grad=True)
        adam = kw.get("optimizer", oracle.ADAM) == oracle.ADAM
        betas = (kw.get("beta1", 0.9), kw.get("beta2", 0.999))
        eps = kw.get("adam_eps", 1e-8)
        if adam:
            opt = torch.optim.Adam([th], lr=kw["lr"], betas=betas, eps=eps)
            ropt = torch.optim.Adam([{"params": [ang]}, {"params": [tra]}], lr=kw["lr"], betas=betas, eps=eps)
        for t in range(1, T + 1):
            if rigid:
                r = np.concatenate([ang.detach().numpy(), tra.detach().numpy()], axis=1)
                loss, _, g, gr = oracle.loss_grad_rigid(pyr[l], th.detach().numpy(), r, p, tscale=float(f))
            else:
                loss, _, g = oracle.loss_grad(pyr[l], th.detach().numpy(), p)
            hist.append(loss)
            if mistake == "global_step":
                lr_t = lr_closed_form(done + t, total, kw["lr"], kw.get("warmup_frac", 0.2))
            elif mistake == "from_zero":
                lr_t = lr_closed_form(t - 1, T, kw["lr"], kw.get("warmup_frac", 0.2))
            else:
                lr_t = lr_closed_form(t, T, kw["lr"], kw.get("warmup_frac", 0.2))
            r_lr = (lr_t / kw["lr"]) * kw.get("rigid_lr", 0.5)
            if adam:
                opt.param_groups[0]["lr"] = lr_t
                th.grad = torch.tensor(g)
                opt.step()
                if rigid:
                    ropt.param_groups[0]["lr"] = r_lr / rmax
                    ropt.param_groups[1]["lr"] = r_lr
                    ang.grad = torch.tensor(gr[:, :3].copy())
                    tra.grad = torch.tensor(gr[:, 3:].copy())
                    ropt.step()
            else:
                with torch.no_grad():
                    th -= lr_t * torch.tensor(g)
                    if rigid:
                        ang -= (r_lr / rmax) * torch.tensor(gr[:, :3].copy())
                        tra -= r_lr * torch.tensor(gr[:, 3:].copy())
        done += T
        theta = th.detach().numpy().copy()
        rho = np.concatenate([ang.detach().numpy(), tra.detach().numpy()], axis=1)
    return np.array(hist), theta, rho


def series(N, shape, seed):
    rng = np.random.default_rng(seed)
    z, y, x = np.meshgrid(*[np.arange(a, dtype=float) for a in shape], indexing="ij")
    out = []
    for s in range(N):
        c = np.array(shape) / 2.0 + 0.6 * s * np.array([0.5, -0.3, 0.4])
        r2 = ((z - c[0]) / 4.5) ** 2 + ((y - c[1]) / 4.0) ** 2 + ((x - c[2]) / 3.5) ** 2
        out.append(np.exp(-r2) + 0.3 * np.sin(0.5 * z + 0.2 * x) + 0.02 * rng.normal(size=shape))
    return np.stack(out)


def compare(imgs, kw, rigid=False, tol=1e-12):
    p = oracle.params(**kw)
    res = oracle.run(imgs, p, loss_history=True)
    loss, theta, hist = res[0], res[1], res[2]
    h2, th2, rho2 = run_by_hand(imgs, kw, rigid=rigid)
    assert hist.shape == h2.shape
    np.testing.assert_allclose(hist, h2, rtol=tol, atol=0)
    assert loss == hist[-1]
    scale = np.abs(th2).max()
    assert scale > 0
    assert np.abs(theta - th2).max() <= tol * scale
    if rigid:
        rho = res[3]
        assert np.abs(rho2).max() > 0
        assert np.abs(rho - rho2).max() <= tol * np.abs(rho2).max()
    return hist


BASE = dict(n_levels=3, steps=(4, 3, 3), K=3, window=3, alpha_ss=0.2, alpha_l2=0.01, alpha_ts=0.05, lr=0.3)


def test_pyramid_by_hand_equals_oracle_downsampling():
    imgs = series(1, (13, 10, 9), 7)[0]
    np.testing.assert_allclose(down2(imgs), oracle.downsample2(imgs), atol=1e-15)
    rng = np.random.default_rng(1)
    v = rng.normal(size=(3, 4, 5, 3))
    np.testing.assert_allclose(prolong(v, (7, 9, 6)), oracle.prolong(v, (7, 9, 6)), atol=1e-14)


@pytest.mark.parametrize("optimizer", [oracle.ADAM, oracle.SGD])
def test_three_level_run_matches_the_schedule_by_hand(optimizer):
    imgs = series(3, (16, 14, 12), 11)
    kw = dict(BASE, optimizer=optimizer, lr=0.3 if optimizer == oracle.ADAM else 40.0)
    compare(imgs, kw)


def test_lncc_two_levels_uneven_steps_and_warmup():
    imgs = series(4, (12, 11, 10), 12)
    kw = dict(BASE, n_levels=2, steps=(5, 2), sim_kind=oracle.LNCC, warmup_frac=0.4, lr=0.2)
    compare(imgs, kw)


def test_gaussian_parameterisation_uses_each_level_voxel_size():
    imgs = series(3, (16, 12, 14), 13)
    kw = dict(BASE, smooth_omega=0.12, spacing=(1.0, 1.2, 0.9), lr=0.4)
    compare(imgs, kw)


def test_rigid_parameters_carry_across_levels():
    imgs = series(3, (16, 14, 12), 14)
    kw = dict(BASE, rigid=1, rigid_lr=0.3)
    # the rotation enters every sample point, so the two Adam implementations' last-bit
    # differences in the angles reach theta amplified: 1e-10 instead of 1e-12
    compare(imgs, kw, rigid=True, tol=1e-10)


@pytest.mark.parametrize("mistake", ["global_step", "from_zero"])
def test_planted_schedule_mistakes_are_visible(mistake):
    """The restatement is sensitive to the readings it pins: a schedule indexed by the
    step count over all levels, or a step counter starting at 0, moves the loss history
    far outside the tolerance of the comparison above."""
    imgs = series(3, (12, 10, 10), 15)
    kw = dict(BASE, n_levels=2, steps=(4, 4), optimizer=oracle.SGD, lr=40.0)
    hist = oracle.run(imgs, oracle.params(**kw), loss_history=True)[2]
    h_ok, _, _ = run_by_hand(imgs, kw)
    np.testing.assert_allclose(hist, h_ok, rtol=1e-9)
    h_bad, _, _ = run_by_hand(imgs, kw, mistake=mistake)
    assert np.abs(h_bad - hist).max() > 1e-5 * np.abs(hist).max()
