"""GPU tests of the launch-configuration knobs and the autotuner: fields per thread of the
flow-grid kernels do not change a single bit of a deterministic registration; each D-chunk
rule is reproducible and within the oracle tolerances of the default; a tuned
configuration taken from the cache gives the registration of the same explicit knobs."""
import numpy as np
import pytest
import torch

import paper_2412_14671_gb300 as m
from paper_2412_14671_gb300 import autotune, phantom

pytestmark = pytest.mark.gpu

SHAPE, N = (40, 36, 44), 4
KW = dict(n_levels=2, steps_per_level=[5, 6], n_squarings=5, window=5, alpha_ss=0.1, alpha_l2=0.01,
          alpha_ts=0.02, lr=0.05, deterministic=1)


def cuda(x):
    return torch.from_numpy(np.ascontiguousarray(x, dtype=np.float32)).cuda()


def run(imgs, **kw):
    with m.Muster(SHAPE, N, **dict(KW, **kw)) as reg:
        reg.set_images(cuda(imgs))
        reg.run()
        return reg.loss_history(), reg.velocities(1, device=False)


def test_flow_fields_per_thread_do_not_change_results():
    imgs = phantom.blob_series(SHAPE, N, seed=61)["images"]
    h2, v2 = run(imgs, flow_nf=2)
    h1, v1 = run(imgs, flow_nf=1)
    assert np.array_equal(h1, h2) and np.array_equal(v1, v2)


@pytest.mark.parametrize("pct", [50, 400])
def test_chunk_rule_is_reproducible_and_close_to_the_default(pct):
    imgs = phantom.blob_series(SHAPE, N, seed=62)["images"]
    h0, v0 = run(imgs)
    ha, va = run(imgs, chunk_pct=pct)
    hb, vb = run(imgs, chunk_pct=pct)
    assert np.array_equal(ha, hb) and np.array_equal(va, vb)
    assert np.abs(ha - h0).max() <= 1e-4 * np.abs(h0).max()
    assert np.abs(va - v0).max() <= 1e-3


def test_tuned_configuration_from_the_cache(tmp_path):
    path = str(tmp_path / "tune.json")
    imgs = phantom.blob_series(SHAPE, N, seed=63)["images"]
    res = autotune.tune(SHAPE, N, KW, images=cuda(imgs), path=path)
    assert not res["cached"] and len(res["trials"]) >= 6
    assert all(ms > 0 for _, _, ms in res["trials"])
    p = autotune.tuned_params(SHAPE, N, KW, path)
    explicit = dict(KW, **autotune.knob_params(res["choice"], N))
    with m.Muster(SHAPE, N, **p) as a, m.Muster(SHAPE, N, **explicit) as b:
        for reg in (a, b):
            reg.set_images(cuda(imgs))
            reg.run()
        assert np.array_equal(a.loss_history(), b.loss_history())
        assert np.array_equal(a.velocities(1, device=False), b.velocities(1, device=False))
    assert autotune.tune(SHAPE, N, KW, images=cuda(imgs), path=path)["cached"]
