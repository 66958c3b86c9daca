"""The allocation-free similarity entry point (muster_op_similarity_noalloc), for
callers that cannot allocate device memory at call time. Called through the C ABI
and compared with the allocating entry point and with the FP64 oracle, on two calls
in a row (the second call must not see the first call's leftovers in the shared
scratch), and checked to take no device memory. Collected last on purpose: if it
fails, a run stopping at the first failure has already run every other test."""
import ctypes

import numpy as np
import pytest
import torch

import oracle
from paper_2412_14671_gb300 import _native, phantom

pytestmark = pytest.mark.gpu

LOSS_RTOL = 1e-5
GRAD_RTOL = 1e-3


def _call(fn, F, W, w, kind, g):
    D, H, Wd = F.shape
    out = ctypes.c_double()
    s = ctypes.c_void_p(torch.cuda.current_stream().cuda_stream or None)
    rc = fn(F.data_ptr(), W.data_ptr(), D, H, Wd, w, kind, ctypes.c_float(1e-6), ctypes.byref(out),
            g.data_ptr() if g is not None else None, s)
    return rc, out.value


def test_noalloc_matches_allocating_entry_point_on_two_calls():
    lib = _native.lib()
    cases = [((40, 37, 70), 5, _native.SILNCC), ((33, 29, 45), 7, _native.LNCC), ((64, 48, 64), 7, _native.SILNCC)]
    for seed, (shape, w, kind) in enumerate(cases):
        imgs = phantom.blob_series(shape, 2, seed=30 + seed)["images"]
        F = torch.from_numpy(imgs[0]).cuda()
        W = torch.from_numpy(imgs[1]).cuda()
        g0, g1, g2 = (torch.empty_like(W) for _ in range(3))
        rc0, s0 = _call(lib.muster_op_similarity, F, W, w, kind, g0)
        rc1, s1 = _call(lib.muster_op_similarity_noalloc, F, W, w, kind, g1)
        rc2, s2 = _call(lib.muster_op_similarity_noalloc, F, W, w, kind, g2)
        assert rc0 == 0 and rc1 == 0 and rc2 == 0, lib.muster_ops_last_error()
        assert abs(s1 - s0) <= LOSS_RTOL * abs(s0)
        rel = (torch.linalg.vector_norm(g1 - g0) / torch.linalg.vector_norm(g0)).item()
        assert rel < 1e-6
        # the second call in a row gives the first call's result
        assert s2 == s1 and torch.equal(g2, g1)


def test_noalloc_matches_the_oracle():
    lib = _native.lib()
    for seed, (shape, w, kind) in enumerate([((20, 18, 24), 5, _native.SILNCC), ((17, 21, 19), 3, _native.LNCC)]):
        imgs = phantom.blob_series(shape, 2, seed=40 + seed)["images"]
        F = torch.from_numpy(imgs[0]).cuda()
        W = torch.from_numpy(imgs[1]).cuda()
        g = torch.empty_like(W)
        for _ in range(2):
            rc, s = _call(lib.muster_op_similarity_noalloc, F, W, w, kind, g)
            assert rc == 0, lib.muster_ops_last_error()
            so, go = oracle.similarity(imgs[0], imgs[1], w, kind, 1e-6, grad=True)
            assert abs(s - so) <= LOSS_RTOL * abs(so), (s, so)
            gn = g.cpu().numpy().astype(np.float64)
            assert np.linalg.norm(gn - go) <= GRAD_RTOL * np.linalg.norm(go)


def test_noalloc_takes_no_device_memory():
    lib = _native.lib()
    shape, w = (48, 52, 40), 7
    imgs = phantom.blob_series(shape, 2, seed=50)["images"]
    F = torch.from_numpy(imgs[0]).cuda()
    W = torch.from_numpy(imgs[1]).cuda()
    g = torch.empty_like(W)
    rc, s_first = _call(lib.muster_op_similarity_noalloc, F, W, w, _native.SILNCC, g)  # warm-up: loads the kernels
    assert rc == 0, lib.muster_ops_last_error()
    torch.cuda.synchronize()
    free0 = torch.cuda.mem_get_info()[0]
    allocs0 = torch.cuda.memory_stats().get("allocation.all.allocated", 0)
    for _ in range(3):
        rc, s = _call(lib.muster_op_similarity_noalloc, F, W, w, _native.SILNCC, g)
        assert rc == 0 and s == s_first
    torch.cuda.synchronize()
    assert torch.cuda.mem_get_info()[0] == free0
    assert torch.cuda.memory_stats().get("allocation.all.allocated", 0) == allocs0


def test_noalloc_rejects_volumes_over_the_limit():
    lib = _native.lib()
    n = int(round((_native_max() + 1) ** (1 / 3))) + 1
    F = torch.zeros((n, n, n), device="cuda")
    rc, _ = _call(lib.muster_op_similarity_noalloc, F, F, 3, _native.SILNCC, None)
    assert rc == _native.EINVAL
    assert b"MUSTER_NOALLOC_MAX_VOXELS" in lib.muster_ops_last_error()


def _native_max():
    import os
    import re

    here = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
    text = open(os.path.join(here, "include", "muster_ops.h")).read()
    return int(re.search(r"#define MUSTER_NOALLOC_MAX_VOXELS (\d+)", text).group(1))
