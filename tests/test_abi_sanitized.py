"""The host side of the C ABI under AddressSanitizer and UndefinedBehaviorSanitizer (no GPU).

libmuster.so is compiled a second time with the host compiler's sanitizers into a temporary
directory and loaded into a child Python process with the ASan runtime preloaded. Without a
device, the child drives every path that runs before device work: argument validation of
muster_create and the stateless ops, the allocation plan of muster_footprint over small,
ragged, deep-and-narrow, many-session and large shapes with every option that changes the
plan, and the clean failure of muster_create when no device is present. Any out-of-bounds
access or undefined behaviour in that host code ends the child with a sanitizer report."""
import concurrent.futures as cf
import glob
import os
import shutil
import subprocess
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))

CHILD = r"""
import ctypes
from paper_2412_14671_gb300 import _native

_native.LIB_PATH = LIB
_native._lib = None
from paper_2412_14671_gb300 import footprint

L = _native.lib()
shapes = [((8, 8, 8), 3), ((1, 5, 7), 2), ((9, 1, 13), 4), ((160, 192, 160), 10), ((256, 256, 256), 16),
          ((4096, 8, 16), 32), ((3, 3, 3), 12)]
options = [{}, dict(recompute_squaring=1), dict(deterministic=1), dict(rigid=1), dict(smooth_omega=0.2),
           dict(n_levels=4, steps_per_level=[5] * 4), dict(n_squarings=0), dict(window=11, similarity=_native.LNCC),
           dict(pair_batch=7, flow_nf=1, chunk_pct=50)]
sizes = {}
for shape, n in shapes:
    for i, kw in enumerate(options):
        sizes[(shape, n, i)] = footprint(shape, n, **kw)
assert all(b > 0 for b in sizes.values())
# storing the squaring intermediates takes more than recomputing them; exact sums take more too
for shape, n in shapes:
    assert sizes[(shape, n, 1)] < sizes[(shape, n, 0)] < sizes[(shape, n, 2)]

p = _native.MusterParams()
L.muster_default_params(ctypes.byref(p))
ctx = ctypes.c_void_p()
shp = (ctypes.c_int64 * 3)(8, 8, 8)
assert L.muster_create(shp, 1, None, ctypes.byref(p), ctypes.byref(ctx)) == _native.EINVAL
for field, bad in [("window", 4), ("window", 13), ("n_levels", 0), ("n_levels", 9), ("flow_factor", 3),
                   ("n_squarings", -1), ("similarity", 7), ("lr", float("nan"))]:
    L.muster_default_params(ctypes.byref(p))
    setattr(p, field, bad)
    assert L.muster_create(shp, 3, None, ctypes.byref(p), ctypes.byref(ctx)) == _native.EINVAL, field
    assert L.muster_last_error(None)
L.muster_default_params(ctypes.byref(p))
big = (ctypes.c_int64 * 3)(2048, 2048, 1024)
assert L.muster_create(big, 3, None, ctypes.byref(p), ctypes.byref(ctx)) == _native.EINVAL
assert L.muster_create(shp, 3, None, ctypes.byref(p), ctypes.byref(ctx)) == _native.ECUDA and not ctx.value
L.muster_destroy(None)
assert L.muster_op_exp(None, 4, 4, 4, 3, ctypes.c_float(1.0), None, None) == _native.EINVAL
assert L.muster_ops_last_error()
print("SANITIZED-OK")
"""


def _runtime(name):
    path = subprocess.run(["gcc", "-print-file-name=" + name], capture_output=True, text=True).stdout.strip()
    return path if os.path.isabs(path) and os.path.exists(path) else None


def test_host_side_of_the_abi_is_clean_under_sanitizers(tmp_path):
    import torch

    if torch.cuda.is_available():
        pytest.skip("checks the no-device paths")
    from paper_2412_14671_gb300 import build

    nvcc = build._nvcc()
    if not shutil.which(nvcc) or not shutil.which("gcc"):
        pytest.skip("nvcc or gcc missing")
    asan = _runtime("libasan.so")
    if asan is None or _runtime("libubsan.so") is None:
        pytest.skip("gcc sanitizer runtimes are not installed")
    san = ["-Xcompiler", "-fsanitize=address", "-Xcompiler", "-fsanitize=undefined"]
    flags = [*build.ARCH, "-O1", "-std=c++17", "-Xcompiler", "-fPIC", "-Xcompiler", "-fno-omit-frame-pointer", *san,
             "-I", build.INCLUDE, "-I", build.CSRC]
    srcs = sorted(glob.glob(os.path.join(build.CSRC, "*.cu")))
    objs = [str(tmp_path / (os.path.basename(s)[:-3] + ".o")) for s in srcs]
    with cf.ThreadPoolExecutor(8) as ex:
        runs = list(ex.map(lambda so: subprocess.run([nvcc, *flags, "-c", so[0], "-o", so[1]], capture_output=True,
                                                     text=True), zip(srcs, objs)))
    for r in runs:
        assert r.returncode == 0, r.stderr[-3000:]
    lib = str(tmp_path / "libmuster_asan.so")
    r = subprocess.run([nvcc, *build.ARCH, "-shared", *san, "-o", lib, *objs, "-lcudart"], capture_output=True,
                       text=True)
    assert r.returncode == 0, r.stderr[-3000:]
    env = dict(os.environ)
    env.update(LD_PRELOAD=asan, ASAN_OPTIONS="detect_leaks=0:halt_on_error=1:protect_shadow_gap=0",
               UBSAN_OPTIONS="halt_on_error=1:print_stacktrace=1",
               PYTHONPATH=ROOT + os.pathsep + env.get("PYTHONPATH", ""))
    r = subprocess.run([sys.executable, "-c", "LIB = %r\n" % lib + CHILD], capture_output=True, text=True, env=env,
                       cwd=ROOT, timeout=600)
    report = r.stdout[-4000:] + r.stderr[-4000:]
    assert r.returncode == 0 and "SANITIZED-OK" in r.stdout, report
    assert "AddressSanitizer" not in r.stderr and "runtime error" not in r.stderr, report
