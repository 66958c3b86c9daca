"""Pins of the oracle's Jacobian determinant maps and deformation metrics (Sec. Evaluation
Metrics; the determinant maps of Sec. Sensitivity to clinical outcomes)."""
import numpy as np
import pytest

import oracle


def grid(shape):
    return np.stack(np.meshgrid(*[np.arange(a, dtype=np.float64) for a in shape], indexing="ij"))


@pytest.mark.parametrize("shape", [(7, 9, 11), (1, 6, 5), (4, 1, 3)])
def test_affine_field_gives_det_of_I_plus_A(shape):
    rng = np.random.default_rng(1)
    A = rng.normal(scale=0.2, size=(3, 3))
    for a in range(3):
        if shape[a] == 1:
            A[:, a] = 0.0  # no derivative along an axis of one plane
    X = grid(shape)
    u = np.einsum("ca,a...->c...", A, X) + rng.normal(size=(3, 1, 1, 1))
    J = oracle.jacobian_det(u)
    np.testing.assert_allclose(J, np.linalg.det(np.eye(3) + A), rtol=0, atol=1e-12)


def test_zero_translation_and_scaling():
    shape = (6, 5, 8)
    assert np.all(oracle.jacobian_det(np.zeros((3,) + shape)) == 1.0)
    assert np.allclose(oracle.jacobian_det(np.full((3,) + shape, 2.5)), 1.0)
    s = 0.1
    np.testing.assert_allclose(oracle.jacobian_det(s * grid(shape)), (1 + s) ** 3, atol=1e-12)


def test_random_field_matches_numpy_gradient():
    rng = np.random.default_rng(2)
    shape = (9, 8, 10)
    u = rng.normal(scale=0.3, size=(3,) + shape)
    D = np.stack([np.stack(np.gradient(u[c], edge_order=1), 0) for c in range(3)], 0)  # D[c, a]
    M = np.eye(3)[:, :, None, None, None] + D
    ref = np.linalg.det(np.moveaxis(M, (0, 1), (-2, -1)))
    np.testing.assert_allclose(oracle.jacobian_det(u), ref, atol=1e-12)


def test_metrics_identical_fields():
    rng = np.random.default_rng(3)
    u = rng.normal(size=(3, 5, 6, 7))
    m = oracle.deformation_metrics(u, u)
    assert m["Eu"] == 0.0 and m["count"] == 5 * 6 * 7
    assert m["PCC"] == pytest.approx(1.0, abs=1e-14)
    np.testing.assert_allclose(m["A"], np.eye(3), atol=1e-12)
    np.testing.assert_allclose(m["b"], 0.0, atol=1e-12)
    assert m["B"] == pytest.approx(1.0, abs=1e-12)


def test_metrics_exact_affine_relation():
    rng = np.random.default_rng(4)
    ut = rng.normal(size=(3, 6, 7, 8))
    A = rng.normal(size=(3, 3))
    b = rng.normal(size=3)
    ue = np.einsum("rc,c...->r...", A, ut) + b[:, None, None, None]
    m = oracle.deformation_metrics(ut, ue)
    np.testing.assert_allclose(m["A"], A, atol=1e-10)
    np.testing.assert_allclose(m["b"], b, atol=1e-10)
    assert m["B"] == pytest.approx(np.trace(A) / 3, abs=1e-10)
    # scaled copy: slope 2, perfect correlation; the negated copy: correlation -1
    m2 = oracle.deformation_metrics(ut, 2 * ut)
    assert m2["B"] == pytest.approx(2.0, abs=1e-12) and m2["PCC"] == pytest.approx(1.0, abs=1e-12)
    assert oracle.deformation_metrics(ut, -ut)["PCC"] == pytest.approx(-1.0, abs=1e-12)


def test_metrics_euclidean_distance_and_roi():
    rng = np.random.default_rng(5)
    shape = (5, 6, 7)
    ut = rng.normal(size=(3,) + shape)
    c = np.array([3.0, 4.0, 12.0])  # |c| = 13
    assert oracle.deformation_metrics(ut, ut + c[:, None, None, None])["Eu"] == pytest.approx(13.0, abs=1e-12)
    ue = ut + rng.normal(scale=0.5, size=ut.shape)
    roi = rng.random(shape) < 0.4
    m = oracle.deformation_metrics(ut, ue, roi)
    sel_t, sel_e = ut[:, roi], ue[:, roi]  # (3, n)
    assert m["count"] == roi.sum()
    assert m["Eu"] == pytest.approx(np.linalg.norm(sel_t - sel_e, axis=0).mean(), rel=1e-12)
    a = sel_t - sel_t.mean(1, keepdims=True)
    e = sel_e - sel_e.mean(1, keepdims=True)
    assert m["PCC"] == pytest.approx((a * e).sum() / np.sqrt((a * a).sum() * (e * e).sum()), rel=1e-12)
