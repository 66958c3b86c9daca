"""The allocation-free similarity entry point (muster_op_similarity_noalloc), for
callers that cannot allocate device memory at call time. Called through the C
ABI and compared with the allocating entry point on two calls in a row (the
second call must not see the first call's leftovers in the shared scratch).
Collected last on purpose: if it fails, a run stopping at the first failure has
already run every other test."""
import ctypes

import numpy as np
import pytest
import torch

from paper_2412_14671_gb300 import _native, phantom

pytestmark = pytest.mark.gpu

LOSS_RTOL = 1e-5


def _call(fn, F, W, w, kind, grad):
    D, H, Wd = F.shape
    out = ctypes.c_double()
    g = torch.empty_like(W)
    s = ctypes.c_void_p(torch.cuda.current_stream().cuda_stream or None)
    rc = fn(F.data_ptr(), W.data_ptr(), D, H, Wd, w, kind, ctypes.c_float(1e-6), ctypes.byref(out),
            g.data_ptr() if grad else None, s)
    return rc, out.value, g


def test_noalloc_matches_allocating_entry_point_on_two_calls():
    lib = _native.lib()
    cases = [((40, 37, 70), 5, _native.SILNCC), ((33, 29, 45), 7, _native.LNCC)]
    for seed, (shape, w, kind) in enumerate(cases):
        imgs = phantom.blob_series(shape, 2, seed=30 + seed)["images"]
        F = torch.from_numpy(imgs[0]).cuda()
        W = torch.from_numpy(imgs[1]).cuda()
        rc0, s0, g0 = _call(lib.muster_op_similarity, F, W, w, kind, True)
        rc1, s1, g1 = _call(lib.muster_op_similarity_noalloc, F, W, w, kind, True)
        assert rc0 == 0 and rc1 == 0, lib.muster_ops_last_error()
        assert abs(s1 - s0) <= LOSS_RTOL * abs(s0)
        rel = (torch.linalg.vector_norm(g1 - g0) / torch.linalg.vector_norm(g0)).item()
        assert rel < 1e-6


def test_noalloc_rejects_volumes_over_the_limit():
    lib = _native.lib()
    n = int(round((_native_max() + 1) ** (1 / 3))) + 1
    F = torch.zeros((n, n, n), device="cuda")
    rc, _, _ = _call(lib.muster_op_similarity_noalloc, F, F, 3, _native.SILNCC, False)
    assert rc == _native.EINVAL
    assert b"MUSTER_NOALLOC_MAX_VOXELS" in lib.muster_ops_last_error()


def _native_max():
    import os
    import re

    here = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
    text = open(os.path.join(here, "include", "muster_ops.h")).read()
    return int(re.search(r"#define MUSTER_NOALLOC_MAX_VOXELS (\d+)", text).group(1))
