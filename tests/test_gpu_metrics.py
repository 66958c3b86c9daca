"""GPU parity of the Jacobian determinant maps and the deformation metrics (Sec. Evaluation
Metrics) against the oracle, through the C ABI."""
import numpy as np
import pytest
import torch

import oracle
import paper_2412_14671_gb300 as m
from paper_2412_14671_gb300 import phantom

pytestmark = pytest.mark.gpu


def cuda(x):
    return torch.from_numpy(np.ascontiguousarray(x, dtype=np.float32)).cuda()


@pytest.mark.parametrize("shape", [(9, 16, 33), (40, 37, 70), (1, 5, 3), (6, 1, 9), (2, 2, 2), (160, 192, 160)])
def test_jacobian_det_matches_oracle(shape):
    rng = np.random.default_rng(sum(shape))
    u = (rng.normal(scale=0.4, size=(3,) + shape)).astype(np.float32)
    J = m.op_jacobian_det(cuda(u)).cpu().numpy()
    Jo = oracle.jacobian_det(u)
    assert np.abs(J - Jo).max() <= 2e-5 * max(1.0, np.abs(Jo).max())


def test_jacobian_det_affine_and_identity():
    shape = (12, 10, 14)
    X = np.stack(np.meshgrid(*[np.arange(a, dtype=np.float64) for a in shape], indexing="ij"))
    A = np.array([[0.1, -0.05, 0.02], [0.03, -0.08, 0.0], [0.0, 0.04, 0.12]])
    u = np.einsum("ca,a...->c...", A, X)
    J = m.op_jacobian_det(cuda(u)).cpu().numpy()
    assert np.abs(J - np.linalg.det(np.eye(3) + A)).max() < 1e-5
    assert torch.all(m.op_jacobian_det(torch.zeros((3,) + shape, device="cuda")) == 1.0)


@pytest.mark.parametrize("shape,with_roi", [((20, 24, 28), False), ((33, 17, 41), True), ((160, 192, 160), True)])
def test_metrics_match_oracle(shape, with_roi):
    rng = np.random.default_rng(7)
    ut = rng.normal(size=(3,) + shape).astype(np.float32)
    A = np.array([[0.8, 0.1, 0.0], [-0.05, 0.9, 0.02], [0.0, 0.03, 1.1]])
    ue = (np.einsum("rc,c...->r...", A, ut) + 0.3 * rng.normal(size=ut.shape) + 0.2).astype(np.float32)
    roi = (rng.random(shape) < 0.6) if with_roi else None
    got = m.op_deformation_metrics(cuda(ut), cuda(ue), torch.from_numpy(roi).cuda() if with_roi else None)
    ref = oracle.deformation_metrics(ut, ue, roi)
    assert got["count"] == ref["count"]
    for k in ("Eu", "PCC", "B"):
        assert got[k] == pytest.approx(ref[k], rel=1e-9, abs=1e-12), k
    np.testing.assert_allclose(got["A"], ref["A"], rtol=1e-9, atol=1e-11)
    np.testing.assert_allclose(got["b"], ref["b"], rtol=1e-9, atol=1e-11)


def test_metrics_are_reproducible_and_empty_roi():
    rng = np.random.default_rng(8)
    shape = (30, 31, 32)
    ut, ue = cuda(rng.normal(size=(3,) + shape)), cuda(rng.normal(size=(3,) + shape))
    a, b = m.op_deformation_metrics(ut, ue), m.op_deformation_metrics(ut, ue)
    assert a["Eu"] == b["Eu"] and a["PCC"] == b["PCC"] and np.array_equal(a["A"], b["A"])
    empty = m.op_deformation_metrics(ut, ue, torch.zeros(shape, dtype=torch.uint8, device="cuda"))
    assert empty["count"] == 0 and empty["Eu"] == 0.0


def test_engine_jacobian_field():
    shape, N = (24, 20, 28), 3
    imgs = phantom.blob_series(shape, N, seed=4)["images"]
    with m.Muster(shape, N, n_levels=1, steps_per_level=[3], n_squarings=5, window=3) as reg:
        reg.set_images(cuda(imgs))
        reg.set_level(0)
        ni, nf = reg.level_dims(0)
        reg.set_velocity(cuda(phantom.smooth_velocity(nf, N - 1, seed=4, sigma=2.0, rms=0.8)))
        for i, j in ((0, 2), (2, 0), (1, 0)):
            disp = reg.get_field(m.PAIR_DISP, i, j, level=0)
            Jf = reg.get_field(m.JACOBIAN, i, j, level=0)
            assert torch.equal(Jf, m.op_jacobian_det(disp))
            Jh = reg.get_field(m.JACOBIAN, i, j, level=0, device=False)
            assert np.array_equal(Jh, Jf.cpu().numpy())
            Jo = oracle.jacobian_det(disp.cpu().numpy())
            assert np.abs(Jh - Jo).max() < 2e-5 * max(1.0, np.abs(Jo).max())
