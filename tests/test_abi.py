"""Host-side checks of the C ABI (no GPU needed): every function declared in
include/*.h is exported by libmuster.so, the binding's ctypes table covers them,
and calls that need a device fail with an error code instead of crashing."""
import ctypes
import os
import re
import subprocess

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
INCLUDE = os.path.join(ROOT, "include")


def declared_functions():
    names = set()
    for h in sorted(os.listdir(INCLUDE)):
        if not h.endswith(".h"):
            continue
        text = open(os.path.join(INCLUDE, h)).read()
        text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
        text = re.sub(r"//[^\n]*", "", text)
        for mt in re.finditer(r"\b(muster_\w+)\s*\(", text):
            names.add(mt.group(1))
    return names


@pytest.fixture(scope="module")
def lib():
    from paper_2412_14671_gb300 import build

    build.build()
    from paper_2412_14671_gb300 import _native

    return _native.lib()


def test_headers_declare_the_boundary():
    names = declared_functions()
    for required in ("muster_create", "muster_set_images", "muster_step", "muster_run", "muster_get_fields",
                     "muster_destroy", "muster_eval", "muster_op_similarity", "muster_op_exp"):
        assert required in names


def test_every_declared_symbol_is_exported(lib):
    out = subprocess.run(["nm", "-D", "--defined-only", os.path.join(ROOT, "paper_2412_14671_gb300", "libmuster.so")],
                         capture_output=True, text=True, check=True).stdout
    exported = {ln.split()[-1] for ln in out.splitlines() if ln.strip()}
    missing = declared_functions() - exported
    assert not missing, missing


def test_binding_covers_every_symbol(lib):
    from paper_2412_14671_gb300 import _native

    assert declared_functions() == set(_native.SIGNATURES)


def test_create_without_device_fails_cleanly(lib):
    import torch

    if torch.cuda.is_available():
        pytest.skip("a GPU is present")
    from paper_2412_14671_gb300 import _native

    p = _native.MusterParams()
    lib.muster_default_params(ctypes.byref(p))
    ctx = ctypes.c_void_p()
    shape = (ctypes.c_int64 * 3)(8, 8, 8)
    rc = lib.muster_create(shape, 3, None, ctypes.byref(p), ctypes.byref(ctx))
    assert rc == _native.ECUDA and not ctx.value
    assert b"CUDA" in lib.muster_last_error(None)


def test_argument_validation_precedes_device_use(lib):
    from paper_2412_14671_gb300 import _native

    p = _native.MusterParams()
    lib.muster_default_params(ctypes.byref(p))
    ctx = ctypes.c_void_p()
    shape = (ctypes.c_int64 * 3)(8, 8, 8)
    assert lib.muster_create(shape, 1, None, ctypes.byref(p), ctypes.byref(ctx)) == _native.EINVAL
    p.window = 4
    assert lib.muster_create(shape, 3, None, ctypes.byref(p), ctypes.byref(ctx)) == _native.EINVAL
    assert b"window" in lib.muster_last_error(None)
    lib.muster_destroy(None)  # NULL-safe
    assert lib.muster_op_exp(None, 4, 4, 4, 3, ctypes.c_float(1.0), None, None) == _native.EINVAL


def test_pair_batch_is_capped_by_the_grid_limit():
    """The image-grid launches put depth x pairs on grid z (at most 65535): a deep, narrow
    volume of 32 sessions (flow depth 2048) runs at most 31 of its 992 pairs per launch,
    whatever batch is asked for; the footprint's pair scratch shows it (no device needed)."""
    from paper_2412_14671_gb300 import footprint

    kw = dict(n_squarings=2, window=3)
    capped = footprint((4096, 8, 16), 32, pair_batch=31, **kw)
    assert footprint((4096, 8, 16), 32, **kw) == capped
    assert footprint((4096, 8, 16), 32, pair_batch=992, **kw) == capped
    assert footprint((4096, 8, 16), 32, pair_batch=30, **kw) < capped
    # a cube of the same volume keeps all 992 pairs in one launch
    assert footprint((128, 64, 64), 32, **kw) == footprint((128, 64, 64), 32, pair_batch=992, **kw)


def test_binding_fails_loudly_without_the_library(monkeypatch, tmp_path):
    """No CPU fallback: with the CUDA library missing, the first call raises."""
    from paper_2412_14671_gb300 import _native

    monkeypatch.setattr(_native, "LIB_PATH", str(tmp_path / "libmuster.so"))
    monkeypatch.setattr(_native, "_lib", None)
    with pytest.raises(RuntimeError, match="no CPU fallback"):
        _native.lib()


def test_binding_rejects_wrongly_sized_tensors_before_any_device_call():
    """The library reads or writes a fixed number of floats behind each device pointer, so the
    binding checks sizes first. A stand-in context (no device) reports a level's dims; a tensor
    of the right size gets past the size check to the device check, one of another size does not."""
    import torch

    from paper_2412_14671_gb300 import api

    class Ctx:
        n_sessions, shape = 3, (10, 12, 14)

        def level_dims(self, level):
            return (10, 12, 14), (5, 6, 7)

    reg = Ctx()
    good = torch.zeros((2, 3, 5, 6, 7))
    with pytest.raises(ValueError, match="CUDA tensor"):
        api.Muster.eval(reg, good, 0, torch.zeros(2 * 3 * 5 * 6 * 7))
    for v, g in ((torch.zeros((2, 3, 5, 6, 6)), None), (good, torch.zeros((1, 3, 5, 6, 7))),
                 (None, torch.zeros(10))):
        with pytest.raises(ValueError, match="elements"):
            api.Muster.eval(reg, v, 0, g)
    with pytest.raises(ValueError, match="vector field"):
        api.op_exp(torch.zeros((2, 4, 4, 4)), 3)
    with pytest.raises(ValueError, match="vector field"):
        api.op_jacobian_det(torch.zeros((4, 4, 4)))
    with pytest.raises(ValueError, match="vector field"):
        api.op_deformation_metrics(torch.zeros((1, 4, 4, 4)), torch.zeros((1, 4, 4, 4)))
    with pytest.raises(ValueError, match="one shape"):
        api.op_similarity(torch.zeros((4, 5, 6)), torch.zeros((4, 5, 7)), 3)
    with pytest.raises(ValueError, match="CUDA tensor"):
        api.op_similarity(torch.zeros((4, 5, 6)), torch.zeros((4, 5, 6)), 3)


def test_set_velocity_checks_the_size_of_the_current_level():
    """set_velocity reads (N-1) x 3 x the current level's flow voxels: a host array or a tensor of
    another size is rejected before the copy; before a level is selected the library decides
    (MUSTER_ESTATE). Stand-in context and library, no device."""
    import numpy as np
    import torch

    from paper_2412_14671_gb300 import _native, api

    calls = []

    class Lib:
        def muster_set_velocity(self, ctx, ptr, on_device):
            calls.append(on_device)
            return 0

    class Ctx:
        n_sessions, _ctx, _lib = 3, None, Lib()
        current = 0

        def level(self):
            return self.current, 0

        def level_dims(self, level):
            return (10, 12, 14), (5, 6, 7)

        def _check(self, rc):
            assert rc == 0

    reg = Ctx()
    api.Muster.set_velocity(reg, np.zeros((2, 3, 5, 6, 7), np.float32))
    assert calls == [0]
    for bad in (np.zeros((2, 3, 5, 6, 6), np.float32), np.zeros(10, np.float32)):
        with pytest.raises(ValueError, match="elements"):
            api.Muster.set_velocity(reg, bad)
    with pytest.raises(ValueError, match="elements"):  # a host tensor takes the host path
        api.Muster.set_velocity(reg, torch.zeros((2, 3, 5, 6, 6)))
    reg.current = -1  # no level yet: nothing to compare with, the library answers
    api.Muster.set_velocity(reg, np.zeros(10, np.float32))
    assert calls == [0, 0]
    lib = _native.lib()
    assert lib.muster_get_level(None, None, None) == _native.EINVAL
