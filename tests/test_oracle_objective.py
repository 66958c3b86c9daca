"""Oracle pin of the objective's pair structure (Sec. MUSTER overview, Eq. cum_deformation,
Sec. Background). With constant velocities whose image-grid length is a whole number of
voxels, every pair map is an exact translation: Phi_ki, which pulls session k onto the grid
of session i, moves by the sum of the velocities between them (plus going forward in time,
minus going back), times the flow factor 2. Each warped image is then a shifted copy of a
session (edges replicated), and the similarity part of the oracle's loss must equal the sum,
over all N(N-1) ordered pairs with the fixed session as the regressor, of the windowed
similarity of those copies -- computed here by brute force over the valid windows with
numpy. Planted mistakes (half of the pairs, fixed and moving swapped, the chain's sign
reversed) move the total far outside the tolerance."""
import numpy as np
import pytest

import oracle


def _shift(I, s):
    """I sampled at p + s for an integer vector s, coordinates clamped to the grid."""
    idx = [np.clip(np.arange(n) + int(d), 0, n - 1) for n, d in zip(I.shape, s)]
    return I[np.ix_(*idx)]


def _brute_similarity(F, W, w, kind, eps):
    """Mean over the valid w^3 windows of SiLNCC_R = (S_WW - S_FW^2/(S_FF + eps))/|R| or
    LNCC_R = 1 - S_FW/sqrt(S_FF S_WW + eps), with centred sums from numpy."""
    sw = np.lib.stride_tricks.sliding_window_view
    f = sw(F, (w, w, w)).reshape(-1, w**3)
    g = sw(W, (w, w, w)).reshape(-1, w**3)
    fc = f - f.mean(1, keepdims=True)
    gc = g - g.mean(1, keepdims=True)
    sff, sww, sfw = (fc * fc).sum(1), (gc * gc).sum(1), (fc * gc).sum(1)
    if kind == oracle.SILNCC:
        r = (sww - sfw**2 / (sff + eps)) / w**3
    else:
        r = 1.0 - sfw / np.sqrt(sff * sww + eps)
    return r.mean()


def _pair_shift(c, k, i, f=2):
    """Image-grid displacement of Phi_ki for constant flow-grid velocities c[m] (m -> m+1)."""
    if k > i:
        return f * sum(c[m] for m in range(i, k))
    return -f * sum(c[m] for m in range(k, i))


def _expected(imgs, c, w, kind, eps, pairs=None, swap=False, sign=1):
    N = imgs.shape[0]
    tot = 0.0
    for i in range(N):
        for k in range(N):
            if k == i or (pairs is not None and (k, i) not in pairs):
                continue
            W = _shift(imgs[k], sign * _pair_shift(c, k, i))
            F = imgs[i]
            tot += _brute_similarity(W, F, w, kind, eps) if swap else _brute_similarity(F, W, w, kind, eps)
    return tot


@pytest.mark.parametrize("kind,w", [(oracle.SILNCC, 3), (oracle.LNCC, 5)])
def test_similarity_total_is_the_sum_over_ordered_pairs_of_exact_translations(kind, w):
    rng = np.random.default_rng(11)
    N, shape = 4, (18, 16, 20)
    nf = tuple((a + 1) // 2 for a in shape)
    imgs = np.stack([
        np.cumsum(np.cumsum(rng.normal(size=shape), 0), 2) * 0.05 + rng.uniform(size=shape) for _ in range(N)
    ])
    # flow-grid velocities of whole voxels: image-grid shifts of 2 voxels per unit
    c = [np.array([1.0, 0.0, -1.0]), np.array([0.0, 1.0, 1.0]), np.array([-1.0, 0.0, 1.0])]
    phi = np.zeros((N - 1, 3) + nf)
    for m in range(N - 1):
        phi[m] = c[m].reshape(3, 1, 1, 1)
    eps = 1e-6
    p = oracle.params(n_levels=1, steps=(1,), K=5, window=w, sim_kind=kind, alpha_ss=0.0, alpha_l2=0.0,
                      alpha_ts=0.0, sim_eps=eps)
    tot, split, _ = oracle.loss_grad(imgs, phi, p, grad=False)
    expect = _expected(imgs, c, w, kind, eps)
    assert split[0] == pytest.approx(expect, rel=1e-10, abs=1e-13)
    assert tot == pytest.approx(expect, rel=1e-10, abs=1e-13)
    # each planted mistake moves the total by far more than the tolerance
    half = {(k, i) for i in range(N) for k in range(N) if k > i}
    wrong = [_expected(imgs, c, w, kind, eps, pairs=half), _expected(imgs, c, w, kind, eps, sign=-1)]
    if kind == oracle.SILNCC:  # LNCC is symmetric in F and W; SiLNCC regresses on the fixed image
        wrong.append(_expected(imgs, c, w, kind, eps, swap=True))
    for x in wrong:
        assert abs(x - expect) > 1e-3 * abs(expect)


def test_regulariser_weights_add_to_the_similarity_total():
    """The total is the similarity sum plus alpha_ss L_ss + alpha_L2 L_L2 + alpha_ts L_ts (Eq. reg_sum),
    each term as the regulariser alone returns it."""
    rng = np.random.default_rng(12)
    N, shape = 3, (12, 14, 10)
    nf = tuple((a + 1) // 2 for a in shape)
    imgs = rng.uniform(size=(N,) + shape)
    phi = rng.normal(size=(N - 1, 3) + nf) * 0.3
    t = np.array([0.0, 1.0, 3.0])
    a = (0.3, 0.02, 0.7)
    p0 = oracle.params(n_levels=1, steps=(1,), K=4, window=3, alpha_ss=0.0, alpha_l2=0.0, alpha_ts=0.0)
    p1 = oracle.params(n_levels=1, steps=(1,), K=4, window=3, alpha_ss=a[0], alpha_l2=a[1], alpha_ts=a[2])
    sim, _, _ = oracle.loss_grad(imgs, phi, p0, t, grad=False)
    tot, split, _ = oracle.loss_grad(imgs, phi, p1, t, grad=False)
    L = oracle.regulariser(phi, t)
    assert split[0] == pytest.approx(sim, rel=1e-12)
    assert tot == pytest.approx(sim + a[0] * L[0] + a[1] * L[1] + a[2] * L[2], rel=1e-12)
