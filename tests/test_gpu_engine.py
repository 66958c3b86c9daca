"""GPU tests of the whole engine through the C ABI: trajectories and the
multi-resolution schedule against the oracle, recompute vs store, checkpoint /
resume, the autograd.Function against central differences, argument and state
errors, and full-size (160x192x160) checks on sampled pairs."""
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


C1 = dict(n_levels=1, steps_per_level=[20], n_squarings=6, window=5, alpha_ss=0.1, alpha_l2=0.01, alpha_ts=0.0)


def test_c1_trajectory_sgd_matches_oracle():
    """Config 1 (3 x 48^3 blob phantom, flow 24^3, K=6, w=5, 20 steps) with plain
    gradient steps: the loss curve and the final velocities follow the oracle."""
    imgs = phantom.cached("blob_series", shape=(48, 48, 48), n_sessions=3, seed=0)["images"]
    p = oracle.params(n_levels=1, steps=(20,), K=6, window=5, alpha_ss=0.1, alpha_l2=0.01, alpha_ts=0.0,
                      optimizer=oracle.SGD, lr=1.0)
    lo, _, go = oracle.loss_grad(imgs, np.zeros((2, 3, 24, 24, 24)), p)
    lr = 0.3 / np.abs(go).max()
    p.lr = lr
    loss_o, theta_o, hist_o = oracle.run(imgs, p, loss_history=True)
    with m.Muster((48, 48, 48), 3, optimizer=m.SGD, lr=lr, **C1) as reg:
        reg.set_images(cuda(imgs))
        loss = reg.run()
        hist = reg.loss_history()
        theta = reg.velocities(0, device=False)
    assert len(hist) == 20
    assert np.abs(hist - hist_o).max() <= 1e-4 * np.abs(hist_o).max()
    assert hist[-1] < hist[0]
    assert rel_l2(theta, theta_o) < 1e-2
    assert abs(loss - loss_o) <= 1e-4 * abs(loss_o)


def test_c1_adam_run_decreases_loss_and_tracks_oracle_loss():
    imgs = phantom.cached("blob_series", shape=(48, 48, 48), n_sessions=3, seed=0)["images"]
    p = oracle.params(n_levels=1, steps=(20,), K=6, window=5, alpha_ss=0.1, alpha_l2=0.01, alpha_ts=0.0, lr=0.05)
    loss_o, theta_o, hist_o = oracle.run(imgs, p, loss_history=True)
    with m.Muster((48, 48, 48), 3, lr=0.05, **C1) as reg:
        reg.set_images(cuda(imgs))
        reg.run()
        hist = reg.loss_history()
        theta = reg.velocities(0, device=False)
    assert hist[-1] < 0.9 * hist[0]
    # Adam amplifies rounding where g ~ 0; the trajectory stays close, not bitwise
    assert np.abs(hist - hist_o).max() <= 1e-3 * np.abs(hist_o).max()
    assert rel_l2(theta, theta_o) < 5e-2


def test_multilevel_schedule_matches_oracle():
    shape, N = (40, 36, 44), 3
    imgs = phantom.blob_series(shape, N, seed=8)["images"]
    kw = dict(n_levels=3, steps_per_level=[4, 3, 2], n_squarings=4, window=3, alpha_ss=0.1, alpha_l2=0.01,
              alpha_ts=0.0)
    p = oracle.params(n_levels=3, steps=(4, 3, 2), K=4, window=3, alpha_ss=0.1, alpha_l2=0.01, optimizer=oracle.SGD)
    lo, _, go = oracle.loss_grad(
        np.stack([oracle.downsample2(oracle.downsample2(im)) for im in imgs]), np.zeros((2, 3, 5, 5, 6)), p)
    p.lr = 0.2 / np.abs(go).max()
    loss_o, theta_o, hist_o = oracle.run(imgs, p, loss_history=True)
    with m.Muster(shape, N, optimizer=m.SGD, lr=p.lr, **kw) as reg:
        reg.set_images(cuda(imgs))
        reg.run()
        hist = reg.loss_history()
        theta = reg.velocities(2, device=False)
        ni, nf = reg.level_dims(0)
        assert nf == (5, 5, 6)
    assert len(hist) == 9
    assert np.abs(hist - hist_o).max() <= 1e-4 * np.abs(hist_o).max()
    assert rel_l2(theta, theta_o) < 1e-2


@pytest.mark.parametrize("K", [1, 5])
def test_recompute_squaring_is_bitwise_identical(K):
    shape, N = (32, 30, 34), 4
    imgs = phantom.blob_series(shape, N, seed=9)["images"]
    nf = tuple((a + 1) // 2 for a in shape)
    phi = cuda(phantom.smooth_velocity(nf, N - 1, seed=9, sigma=2.0, rms=0.6))
    grads = []
    for rec in (0, 1):
        with m.Muster(shape, N, n_squarings=K, recompute_squaring=rec, deterministic=1) as reg:
            reg.set_images(cuda(imgs))
            g = torch.empty_like(phi)
            reg.eval(phi, 0, g)
            grads.append(g)
    # recomputed intermediates are bitwise the stored ones and the deterministic adjoint
    # sums in a fixed order: identical gradients
    assert torch.equal(grads[0], grads[1])


def test_deterministic_mode_is_bit_reproducible_and_matches_oracle():
    shape, N = (30, 28, 34), 4
    imgs = phantom.blob_series(shape, N, seed=13)["images"]
    kw = dict(n_levels=2, steps_per_level=[3, 4], n_squarings=5, window=3, alpha_ss=0.1, alpha_l2=0.01,
              alpha_ts=0.05, lr=0.05, deterministic=1)
    runs = []
    for _ in range(3):
        with m.Muster(shape, N, **kw) as reg:
            reg.set_images(cuda(imgs))
            reg.run()
            runs.append((reg.loss_history(), reg.velocities(1, device=False)))
    for h, th in runs[1:]:
        assert np.array_equal(h, runs[0][0]) and np.array_equal(th, runs[0][1])
    # the deterministic gradient is the same gradient
    nf = tuple((a + 1) // 2 for a in shape)
    phi = phantom.smooth_velocity(nf, N - 1, seed=13, sigma=2.0, rms=0.6)
    with m.Muster(shape, N, n_squarings=5, window=3, alpha_ss=0.1, alpha_l2=0.01, alpha_ts=0.05,
                  deterministic=1) as reg:
        reg.set_images(cuda(imgs))
        g = torch.empty((N - 1, 3) + nf, device="cuda")
        loss = reg.eval(cuda(phi), 0, g)
    p = oracle.params(K=5, window=3, alpha_ss=0.1, alpha_l2=0.01, alpha_ts=0.05)
    lo, _, go = oracle.loss_grad(imgs, phi, p)
    assert abs(loss - lo) <= 1e-5 * abs(lo)
    assert rel_l2(g.cpu().numpy(), go) < 1e-3



@pytest.mark.parametrize("deterministic", [0, 1])
def test_no_squarings_matches_oracle(deterministic):
    """K = 0 (u = v, no scaling and squaring): the step's first launch is the
    plain u_0 kernel, the pair gradients go through the separate add kernel,
    and in deterministic mode that first launch also zeroes the fixed-point
    scale word. Gradient against the oracle; deterministic runs reproduce."""
    shape, N = (30, 28, 34), 4
    imgs = phantom.blob_series(shape, N, seed=17)["images"]
    nf = tuple((a + 1) // 2 for a in shape)
    phi = phantom.smooth_velocity(nf, N - 1, seed=17, sigma=2.0, rms=0.6)
    kw = dict(n_squarings=0, window=3, alpha_ss=0.1, alpha_l2=0.01, alpha_ts=0.05,
              deterministic=deterministic)
    with m.Muster(shape, N, **kw) as reg:
        reg.set_images(cuda(imgs))
        g = torch.empty((N - 1, 3) + nf, device="cuda")
        loss = reg.eval(cuda(phi), 0, g)
        g2 = torch.empty_like(g)
        loss2 = reg.eval(cuda(phi), 0, g2)
    p = oracle.params(K=0, window=3, alpha_ss=0.1, alpha_l2=0.01, alpha_ts=0.05)
    lo, _, go = oracle.loss_grad(imgs, phi, p)
    assert abs(loss - lo) <= 1e-5 * abs(lo)
    assert rel_l2(g.cpu().numpy(), go) < 1e-3
    if deterministic:
        assert loss2 == loss and torch.equal(g2, g)
    runs = []
    for _ in range(2):
        with m.Muster(shape, N, n_levels=2, steps_per_level=[3, 4], lr=0.05, **kw) as reg:
            reg.set_images(cuda(imgs))
            reg.run()
            runs.append((reg.loss_history(), reg.velocities(1, device=False)))
    assert np.all(np.isfinite(runs[0][0]))
    if deterministic:
        assert np.array_equal(runs[1][0], runs[0][0]) and np.array_equal(runs[1][1], runs[0][1])

def test_checkpoint_resume():
    shape, N = (24, 26, 22), 3
    imgs = phantom.blob_series(shape, N, seed=10)["images"]
    kw = dict(n_levels=1, steps_per_level=[6], n_squarings=4, window=3, lr=0.05, deterministic=1)
    with m.Muster(shape, N, **kw) as a:
        a.set_images(cuda(imgs))
        a.set_level(0)
        for _ in range(3):
            a.step()
        state = a.get_state()
        for _ in range(3):
            a.step()
        ref = a.velocities(0, device=False)
    with m.Muster(shape, N, **kw) as b:
        b.set_images(cuda(imgs))
        b.set_state(state)
        for _ in range(3):
            b.step()
        with pytest.raises(m.MusterError):
            b.step()  # schedule finished
        got = b.velocities(0, device=False)
    # deterministic mode: the resumed run is the uninterrupted run, bit for bit
    assert np.array_equal(got, ref)


def test_autograd_function_and_central_differences():
    """Config 3 pattern on a reduced volume: MusterLoss backward is the eval
    gradient, and matches central differences (h = 1e-3) of the GPU loss."""
    shape, N = (48, 44, 40), 4
    imgs = phantom.brain_series(shape, N, seed=11)["images"]
    with m.Muster(shape, N, n_squarings=7, window=5, alpha_ss=0.01, alpha_l2=0.001) as reg:
        reg.set_images(cuda(imgs))
        ni, nf = reg.level_dims(0)
        phi = cuda(phantom.smooth_velocity(nf, N - 1, seed=11, sigma=2.0, rms=0.5))
        v = phi.clone().requires_grad_(True)
        L = m.MusterLoss.apply(v, reg, 0)
        (2.0 * L).backward()
        g = torch.empty_like(phi)
        reg.eval(phi, 0, g)
        assert torch.allclose(v.grad, 2.0 * g)
        rng = np.random.default_rng(11)
        h = 1e-3
        gs = g.abs().max().item()
        errs = []
        for _ in range(400):
            if len(errs) == 64:
                break
            idx = tuple(int(rng.integers(0, s)) for s in phi.shape)
            # central differences of a float32 loss: keep entries well above its rounding noise
            if abs(g[idx].item()) < 0.1 * gs:
                continue
            pp, pm = phi.clone(), phi.clone()
            pp[idx] += h
            pm[idx] -= h
            fd = (reg.eval(pp, 0) - reg.eval(pm, 0)) / (2 * h)
            errs.append(abs(fd - g[idx].item()) / abs(g[idx].item()))
        assert len(errs) >= 32
        assert np.median(errs) < 1e-2 and max(errs) < 0.1, errs


def test_errors_are_reported():
    with pytest.raises(m.MusterError) as e:
        m.Muster((8, 8, 8), 1)
    assert e.value.code == -1
    with pytest.raises(m.MusterError):
        m.Muster((8, 8, 8), 3, window=4)
    with m.Muster((10, 10, 10), 3, steps_per_level=[2]) as reg:
        with pytest.raises(m.MusterError) as e:
            reg.step()
        assert e.value.code == -2
        bad = np.zeros((3, 10, 10, 10), np.float32)
        bad[1, 2, 3, 4] = np.nan
        with pytest.raises(m.MusterError) as e:
            reg.set_images(bad)
        assert e.value.code == -1
        with pytest.raises(m.MusterError):
            reg.set_images(np.zeros((3, 10, 10, 10), np.float32), times=[0.0, 2.0, 1.0])
        reg.set_images(np.random.default_rng(0).uniform(size=(3, 10, 10, 10)).astype(np.float32))
        reg.set_level(0)
        reg.step()
        reg.step()
        with pytest.raises(m.MusterError):
            reg.step()


def test_full_size_sampled_pair():
    """Config 2 finest grid (160x192x160, flow 80x96x80, K=7, w=7) with 4 sessions:
    the farthest pair's flow displacement, warp and SiLNCC against the oracle."""
    shape, N = (160, 192, 160), 4
    imgs = phantom.cached("brain_series", shape=shape, n_sessions=N, seed=0)["images"]
    with m.Muster(shape, N, n_squarings=7, window=7) as reg:
        reg.set_images(cuda(imgs))
        reg.set_level(0)
        ni, nf = reg.level_dims(0)
        phi = phantom.smooth_velocity(nf, N - 1, seed=12, sigma=3.0, rms=0.6)
        reg.set_velocity(cuda(phi))
        flow = reg.get_field(m.PAIR_FLOW, 0, N - 1, level=0, device=False)
        W = reg.get_field(m.WARPED, 0, N - 1, level=0)
        s_gpu = m.op_similarity(cuda(imgs[0]), W, 7, m.SILNCC, 1e-6, grad=False)
        loss = reg.eval(None, 0)
    up = np.stack([oracle.exp(phi[k], 7, 1.0) for k in range(N - 1)])
    um = np.stack([oracle.exp(phi[k], 7, -1.0) for k in range(N - 1)])
    U = oracle.compose(up, um)
    assert np.abs(flow - U[N - 1, 0]).max() < 1e-3
    Wo = oracle.warp(imgs[N - 1], oracle.upsample(U[N - 1, 0], shape))
    assert np.abs(W.cpu().numpy() - Wo).max() < 1e-3
    so = oracle.similarity(imgs[0], Wo, 7, oracle.SILNCC, 1e-6)
    assert abs(s_gpu - so) <= 1e-5 * abs(so)
    assert np.isfinite(loss) and loss > 0


def _stats(reg):
    return {s["name"]: s for s in reg.profile_end()}


PROF = dict(n_squarings=4, window=3, alpha_ss=0.1, alpha_l2=0.01, alpha_ts=0.02, deterministic=1)


def test_profiled_run_times_sampled_steps_and_changes_nothing():
    """A profiled run replays graph copies with event nodes on steps 0 and 8 of each level
    and the plain graph on the others: the result is bitwise the unprofiled one, every
    launch is counted, and the timed launches carry their algorithmic bytes."""
    shape, N = (24, 20, 28), 3
    imgs = phantom.blob_series(shape, N, seed=13)["images"]
    with m.Muster(shape, N, n_levels=2, steps_per_level=[10, 12], **PROF) as reg:
        reg.set_images(cuda(imgs))
        reg.run()
        v_ref, l_ref = reg.velocities(1, device=False), reg.loss_split()["total"]
        reg.profile_begin()
        reg.run()
        st = _stats(reg)
        assert np.array_equal(reg.velocities(1, device=False), v_ref)
        assert reg.loss_split()["total"] == l_ref
        Vf1 = int(np.prod(reg.level_dims(1)[1]))
        Vf0 = int(np.prod(reg.level_dims(0)[1]))
    adam = st["adam"]
    assert adam["all_launches"] == 22 and adam["launches"] == 4
    assert adam["bytes"] == pytest.approx(2 * (N - 1) * (Vf0 + Vf1) * 112.0)
    for name in ("warp", "sim_fwd", "sim_bwd", "warp_bwd", "squaring", "squaring_bwd", "loss_reduce"):
        s = st[name]
        assert s["all_launches"] >= 22 and 0 < s["launches"] < s["all_launches"] and s["ms"] > 0, name
    for s in st.values():
        assert s["all_launches"] >= s["launches"] >= 0


def test_profiled_long_level_wraps_the_copy_ring_and_survives_new_times():
    """40 steps a level, two runs in one window: steps 0, 8, ..., 32 of each run are timed
    (10 replays, more than the ring of 8 copies holds unread); new times between the runs
    drop the graphs with copies still unread, whose events are read at the end."""
    shape, N = (20, 22, 18), 3
    imgs = phantom.blob_series(shape, N, seed=14)["images"]
    kw = dict(PROF, n_levels=1, steps_per_level=[40])
    with m.Muster(shape, N, **kw) as ref:
        ref.set_images(cuda(imgs), times=[0.0, 1.5, 4.0])
        ref.run()
        v_ref = ref.velocities(0, device=False)
    with m.Muster(shape, N, **kw) as reg:
        reg.set_images(cuda(imgs))
        reg.profile_begin()
        reg.run()
        reg.set_images(cuda(imgs), times=[0.0, 1.5, 4.0])
        reg.run()
        st = _stats(reg)
        assert np.array_equal(reg.velocities(0, device=False), v_ref)
    timed = 2 * (1 + 39 // 8)
    assert st["adam"]["all_launches"] == 80 and st["adam"]["launches"] == timed
    assert st["sim_fwd"]["launches"] == timed * st["sim_fwd"]["all_launches"] // 80
    assert all(s["ms"] > 0 for s in st.values() if s["launches"])


def test_clearing_level_survives_an_evaluation_at_a_larger_level():
    """Atomic adjoint: on a flow grid whose two exp-gradient buffers take at most 16 MiB
    (level 0 here, 34 x 32 x 32 nodes) the kernels that read those buffers clear them, and
    no clearing pass runs; an evaluation at level 1 (68 x 64 x 64 nodes, 17.8 MB, cleared
    by passes) leaves them written, and the engine zeroes them again. The steps after the
    evaluation match the same steps without it."""
    shape, N = (136, 128, 128), 3
    imgs = phantom.cached("blob_series", shape=shape, n_sessions=N, seed=21)["images"]
    kw = dict(n_levels=2, steps_per_level=[4, 1], n_squarings=4, window=3, alpha_ss=0.1, alpha_l2=0.01,
              alpha_ts=0.0, optimizer=m.SGD, lr=0.05, deterministic=0)
    v1 = 0.3 * torch.randn((N - 1, 3, 68, 64, 64), generator=torch.Generator().manual_seed(5)).cuda()
    out = []
    for with_eval in (False, True):
        with m.Muster(shape, N, **kw) as reg:
            reg.set_images(cuda(imgs))
            assert reg.level_dims(1)[1] == (68, 64, 64)
            reg.set_level(0)
            reg.step()
            reg.step()
            if with_eval:
                assert np.isfinite(reg.eval(v1, 1))
            losses = [reg.step(), reg.step()]
            out.append((losses, reg.velocities(0, device=False)))
    (la, va), (lb, vb) = out
    assert np.allclose(la, lb, rtol=1e-5, atol=0.0), (la, lb)
    assert rel_l2(vb, va) < 1e-4
