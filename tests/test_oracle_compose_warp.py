"""Oracle pins: composition chains (Eq. cum_deformation), displacement upsampling,
image warp, pyramid down-sampling and velocity prolongation (Sec. Implementation Details)."""
import numpy as np
import scipy.ndimage

import oracle


def _grid(n):
    return np.stack(np.meshgrid(*[np.arange(a, dtype=np.float64) for a in n], indexing="ij"))


def _const(c, n):
    return np.broadcast_to(np.asarray(c, float)[:, None, None, None], (3,) + tuple(n)).copy()


def test_compose_constant_fields_add_along_the_chain():
    # distinct translations per consecutive pair pin which field each chain step uses
    N, n = 5, (6, 5, 7)
    c = np.array([[0.3, -0.1, 0.2], [0.05, 0.4, -0.3], [-0.25, 0.15, 0.1], [0.2, 0.2, -0.45]])
    up = np.stack([_const(c[m], n) for m in range(N - 1)])
    um = np.stack([_const(-c[m], n) for m in range(N - 1)])
    U = oracle.compose(up, um)
    for i in range(N):
        assert np.all(U[i, i] == 0)
        for k in range(N):
            if k > i:
                expect = c[i:k].sum(0)
            elif k < i:
                expect = -c[k:i].sum(0)
            else:
                continue
            assert np.abs(U[k, i] - _const(expect, n)).max() < 1e-12, (k, i)


def test_compose_affine_is_matrix_product_in_order():
    n = (20, 20, 20)
    x0 = np.array([9.5, 9.5, 9.5])
    X = _grid(n) - x0[:, None, None, None]
    A1 = np.array([[0.04, 0.03, 0.0], [-0.02, 0.01, 0.05], [0.03, 0.0, -0.02]])
    A2 = np.array([[-0.03, 0.0, 0.06], [0.04, 0.02, 0.0], [0.0, -0.05, 0.01]])
    lin = lambda A: np.einsum("ca,azyx->czyx", A, X)  # noqa: E731
    up = np.stack([lin(A1), lin(A2)])
    um = np.stack([lin(-A1), lin(-A2)])
    U = oracle.compose(up, um)
    I3 = np.eye(3)
    sl = (slice(None),) + tuple(slice(5, 15) for _ in range(3))
    # U[2,0] = u+_0 + u+_1 o (x + u+_0): first step 0 -> 1, then 1 -> 2
    expect = lin((I3 + A2) @ (I3 + A1) - I3)
    assert np.abs(U[2, 0][sl] - expect[sl]).max() < 1e-12
    wrong = lin((I3 + A1) @ (I3 + A2) - I3)
    assert np.abs(U[2, 0][sl] - wrong[sl]).max() > 1e-4
    # U[0,2] = u-_1 + u-_0 o (x + u-_1)
    expect = lin((I3 - A1) @ (I3 - A2) - I3)
    assert np.abs(U[0, 2][sl] - expect[sl]).max() < 1e-12


def test_upsample_zero_constant_affine():
    nf, ni = (6, 7, 5), (12, 13, 10)
    assert np.all(oracle.upsample(np.zeros((3,) + nf), ni) == 0)
    c = np.array([0.3, -1.25, 0.5])
    assert np.abs(oracle.upsample(_const(c, nf), ni) - 2 * _const(c, ni)).max() < 1e-12
    A = np.array([[0.1, 0.2, -0.1], [0.0, 0.3, 0.1], [-0.2, 0.1, 0.05]])
    b = np.array([0.5, -0.2, 0.1])
    Uf = np.einsum("ca,azyx->czyx", A, _grid(nf)) + b[:, None, None, None]
    Ut = oracle.upsample(Uf, ni)
    q = (_grid(ni) + 0.5) / 2 - 0.5
    expect = 2 * (np.einsum("ca,azyx->czyx", A, q) + b[:, None, None, None])
    inner = (slice(None), slice(1, 11), slice(1, 12), slice(1, 9))  # q not clamped
    assert np.abs(Ut[inner] - expect[inner]).max() < 1e-12


def test_upsample_adjoint_dot_product():
    rng = np.random.default_rng(4)
    nf, ni = (5, 6, 4), (9, 12, 8)
    d = rng.normal(size=(3,) + nf)
    g = rng.normal(size=(3,) + ni)
    lhs = (oracle.upsample(d, ni) * g).sum()
    rhs = (d * oracle.upsample_adjoint(g, nf)).sum()
    assert abs(lhs - rhs) < 1e-11 * abs(lhs)


def test_warp_identity_shift_affine():
    rng = np.random.default_rng(5)
    n = (9, 10, 11)
    I = rng.normal(size=n)
    assert np.array_equal(oracle.warp(I, np.zeros((3,) + n)), I)
    W = oracle.warp(I, _const([1.0, -2.0, 3.0], n))
    assert np.array_equal(W[:-1, 2:, :-3], I[1:, :-2, 3:])
    a = np.array([0.3, -0.7, 0.2])
    Ia = np.tensordot(a, _grid(n), 1) + 1.0
    Ut = 0.8 * np.sin(_grid(n) / 3.0)  # |Ut| < 1, keep sample points inside with a margin
    Wa = oracle.warp(Ia, Ut)
    expect = np.tensordot(a, _grid(n) + Ut, 1) + 1.0
    inner = (slice(1, -1),) * 3
    assert np.abs(Wa[inner] - expect[inner]).max() < 1e-12


def test_warp_adjoint_matches_central_differences():
    rng = np.random.default_rng(6)
    n = (7, 8, 9)
    I = scipy.ndimage.gaussian_filter(rng.normal(size=n), 1.0)
    Ut = rng.uniform(-1.3, 1.3, size=(3,) + n)
    gW = rng.normal(size=n)
    g = oracle.warp_adjoint(I, Ut, gW)
    d = rng.normal(size=Ut.shape)
    h = 1e-6
    fd = ((oracle.warp(I, Ut + h * d) - oracle.warp(I, Ut - h * d)) * gW).sum() / (2 * h)
    assert abs(fd - (g * d).sum()) < 1e-6 * max(1.0, abs(fd))


def test_downsample_constant_affine_and_odd_sizes():
    n = (9, 8, 7)
    assert np.allclose(oracle.downsample2(np.full(n, 0.37)), 0.37, atol=1e-15)
    a = np.array([0.2, -0.1, 0.3])
    I = np.tensordot(a, _grid(n), 1)
    out = oracle.downsample2(I)
    assert out.shape == (5, 4, 4)
    centre = 2 * _grid(out.shape) + 0.5
    expect = np.tensordot(a, centre, 1)
    assert np.abs(out[:4, :4, :3] - expect[:4, :4, :3]).max() < 1e-12
    # last (odd) plane: mean of plane 8 replicated -> centre at 8 along axis 0
    ex = np.tensordot(a, np.stack([np.full(out.shape[1:], 8.0), centre[1, 0], centre[2, 0]]), 1)
    assert np.abs(out[4, :, :3] - ex[:, :3]).max() < 1e-12


def test_prolong_constant_and_affine():
    nc, nf = (5, 6, 4), (10, 12, 8)
    c = np.array([0.1, -0.4, 0.25])
    assert np.abs(oracle.prolong(_const(c, nc), nf) - 2 * _const(c, nf)).max() < 1e-12
    A = np.array([[0.1, 0.0, 0.2], [0.05, -0.1, 0.0], [0.0, 0.3, 0.1]])
    v = np.einsum("ca,azyx->czyx", A, _grid(nc))
    out = oracle.prolong(v, nf)
    q = (_grid(nf) + 0.5) / 2 - 0.5
    expect = 2 * np.einsum("ca,azyx->czyx", A, q)
    inner = (slice(None), slice(1, 9), slice(1, 11), slice(1, 7))
    assert np.abs(out[inner] - expect[inner]).max() < 1e-12
