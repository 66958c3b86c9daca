"""Oracle pins: windowed moments, LNCC / SiLNCC (Eq. LNCC, Eq. sum_lncc, the SiLNCC
equation, Eq. E_lncc) and the regularisers (Eq. reg_ss, the L2 term, Eq. reg_ts)."""
import itertools
import json
import os

import numpy as np
import pytest

import oracle

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


@pytest.mark.parametrize("shape,w", [((8, 8, 8), 3), ((7, 9, 11), 3), ((7, 9, 11), 5), ((7, 9, 11), 7), ((8, 8, 8), 5)])
def test_window_stats_brute_force(shape, w):
    rng = np.random.default_rng(7)
    F = rng.uniform(size=shape)
    W = rng.uniform(size=shape)
    st = oracle.window_stats(F, W, w)
    m = tuple(a - w + 1 for a in shape)
    for c in itertools.product(*[range(a) for a in m]):
        f = F[c[0] : c[0] + w, c[1] : c[1] + w, c[2] : c[2] + w].ravel()
        g = W[c[0] : c[0] + w, c[1] : c[1] + w, c[2] : c[2] + w].ravel()
        assert abs(st["muF"][c] - f.mean()) < 1e-12
        assert abs(st["muW"][c] - g.mean()) < 1e-12
        # textbook sums of squares through np.var / np.cov (ML normalisation * n)
        assert abs(st["Sff"][c] - f.var() * f.size) < 1e-11
        assert abs(st["Sww"][c] - g.var() * g.size) < 1e-11
        assert abs(st["Sfw"][c] - np.cov(f, g, bias=True)[0, 1] * f.size) < 1e-11


def test_similarity_of_identical_and_affine_images():
    rng = np.random.default_rng(8)
    F = rng.uniform(size=(10, 11, 12))
    eps = 1e-9
    assert abs(oracle.similarity(F, F, 3, oracle.SILNCC, eps)) < 1e-9
    assert abs(oracle.similarity(F, F, 3, oracle.LNCC, eps)) < 1e-9
    W = 1.7 * F + 0.3
    assert abs(oracle.similarity(F, W, 5, oracle.SILNCC, eps)) < 1e-8
    assert abs(oracle.similarity(F, W, 5, oracle.LNCC, eps)) < 1e-9
    assert abs(oracle.similarity(F, -0.8 * F + 2.0, 5, oracle.LNCC, eps) - 2.0) < 1e-9
    # F = W with eps: SiLNCC_R = S_FF eps / (S_FF + eps) / |R| exactly
    st = oracle.window_stats(F, F, 3)
    expect = (st["Sff"] * 1e-2 / (st["Sff"] + 1e-2) / 27).mean()
    assert abs(oracle.similarity(F, F, 3, oracle.SILNCC, 1e-2) - expect) < 1e-13


def test_no_valid_window_gives_zero():
    F = np.ones((4, 9, 9))
    s, d = oracle.similarity(F, F, 5, oracle.SILNCC, 1e-6, grad=True)
    assert s == 0.0 and np.all(d == 0)


def _golden(name):
    with open(os.path.join(GOLDEN, name)) as fh:
        return json.load(fh)


def test_expected_lncc_matches_closed_form():
    """Eq. E_lncc: E[LNCC_R] ~ 1 - 1/sqrt(1 + sigma^2/(a^2 S_i^2)); the paper reports
    a Monte Carlo bias of at most ~0.02 already at |R| = 9 (appendix on E[LNCC])."""
    g = _golden("paper_lncc_bias.json")
    rng = np.random.default_rng(9)
    n = (40, 40, 40)
    F = rng.normal(size=n)
    for a, sigma in [(1.0, 0.5), (1.0, 1.0), (2.0, 1.5), (0.5, 1.0)]:
        W = a * F + 0.2 + sigma * rng.normal(size=n)
        st = oracle.window_stats(F, W, 3)
        S2 = (st["Sff"] / 27).mean()  # average ML variance of I_i over the regions
        expect = 1 - 1 / np.sqrt(1 + sigma**2 / (a**2 * S2))
        got = oracle.similarity(F, W, 3, oracle.LNCC, 0.0)
        assert abs(got - expect) < g["max_bias"], (a, sigma, got, expect)


def test_expected_silncc_is_ols_residual_variance():
    """SiLNCC_R = RSS/|R| of the least-squares fit W = aF + b; E[RSS] = sigma^2 (|R| - 2)."""
    rng = np.random.default_rng(10)
    n = (40, 40, 40)
    F = rng.normal(size=n)
    for sigma in (0.1, 0.5):
        W = 1.3 * F - 0.4 + sigma * rng.normal(size=n)
        got = oracle.similarity(F, W, 3, oracle.SILNCC, 0.0)
        expect = sigma**2 * (27 - 2) / 27
        assert abs(got / expect - 1) < 0.03, (sigma, got, expect)


@pytest.mark.parametrize("kind", [oracle.SILNCC, oracle.LNCC])
def test_similarity_gradient_central_differences(kind):
    rng = np.random.default_rng(11)
    n = (7, 8, 9)
    F = rng.uniform(size=n)
    W = 0.5 * F + 0.5 * rng.uniform(size=n)
    s, d = oracle.similarity(F, W, 3, kind, 1e-6, grad=True)
    h = 1e-6
    for _ in range(40):
        idx = tuple(rng.integers(0, a) for a in n)
        Wp, Wm = W.copy(), W.copy()
        Wp[idx] += h
        Wm[idx] -= h
        fd = (oracle.similarity(F, Wp, 3, kind, 1e-6) - oracle.similarity(F, Wm, 3, kind, 1e-6)) / (2 * h)
        assert abs(fd - d[idx]) < 1e-7 * max(1.0, abs(fd)) + 1e-9, (idx, fd, d[idx])


def _grid(n):
    return np.stack(np.meshgrid(*[np.arange(a, dtype=np.float64) for a in n], indexing="ij"))


def test_regulariser_closed_forms():
    n = (5, 6, 7)
    A = np.array([[0.2, -0.1, 0.3], [0.05, 0.4, 0.0], [-0.3, 0.1, 0.25]])
    phi_lin = np.einsum("ca,azyx->czyx", A, _grid(n)) + 0.7
    phi = np.stack([phi_lin, phi_lin, phi_lin])
    L = oracle.regulariser(phi)
    assert abs(L[0] - (A**2).sum()) < 1e-12
    c = np.array([0.3, -0.2, 0.5])
    const = np.broadcast_to(c[:, None, None, None], (3,) + n)
    L = oracle.regulariser(np.stack([const, 2 * const]))
    assert L[0] == 0.0
    assert abs(L[1] - 0.5 * ((c**2).sum() + 4 * (c**2).sum())) < 1e-12
    # flows proportional to the time gaps: zero temporal penalty
    t = np.array([0.0, 1.0, 3.5, 4.0, 6.0])
    phis = np.stack([(t[i + 1] - t[i]) * phi_lin for i in range(4)])
    assert oracle.regulariser(phis, t)[2] < 1e-24
    # constant flows: L_ts = mean_i |c_{i-1}/dt_{i-1} - c_i/dt_i|^2
    cs = np.array([[0.1, 0.0, 0.2], [0.3, -0.1, 0.0], [0.0, 0.2, 0.1], [-0.2, 0.1, 0.3]])
    phis = np.stack([np.broadcast_to(cs[i][:, None, None, None], (3,) + n) for i in range(4)])
    dt = np.diff(t)
    expect = np.mean([((cs[i - 1] / dt[i - 1] - cs[i] / dt[i]) ** 2).sum() for i in (1, 2, 3)])
    assert abs(oracle.regulariser(phis, t)[2] - expect) < 1e-12


def test_regulariser_gradient_central_differences():
    rng = np.random.default_rng(12)
    n = (4, 5, 6)
    phi = rng.normal(size=(3, 3) + n)
    t = np.array([0.0, 0.7, 2.0, 2.5])
    al = (0.7, 0.3, 0.2)
    L, g = oracle.regulariser(phi, t, al, grad=True)
    f = lambda p: np.dot(al, oracle.regulariser(p, t))  # noqa: E731
    h = 1e-6
    for _ in range(40):
        idx = tuple(rng.integers(0, a) for a in phi.shape)
        pp, pm = phi.copy(), phi.copy()
        pp[idx] += h
        pm[idx] -= h
        fd = (f(pp) - f(pm)) / (2 * h)
        assert abs(fd - g[idx]) < 1e-7, (idx, fd, g[idx])
