"""The FP64 oracle under AddressSanitizer and UndefinedBehaviorSanitizer (no GPU).

The oracle is compiled a second time with -fsanitize=address,undefined into a temporary
directory and loaded into a child Python process that has the ASan runtime preloaded;
the child drives every oracle entry point on small volumes that include ragged shapes,
odd sizes, single-plane axes, windows that do not fit, fields that sample outside the
grid, an ROI and the multi-level driver with rigid parameters and the Gaussian
parameterisation. Any out-of-bounds access, use after free or undefined behaviour ends
the child with a sanitizer report, and the test fails with it."""
import os
import shutil
import subprocess
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))

CHILD = r"""
import numpy as np
import oracle

oracle._LIB = LIB
oracle._lib = None
rng = np.random.default_rng(0)

for shape in [(7, 9, 11), (1, 6, 5), (4, 1, 3), (6, 5, 1)]:
    nf = tuple((a + 1) // 2 for a in shape)
    phi = rng.normal(size=(3,) + nf) * 1.5          # samples reach outside the grid
    up = oracle.exp(phi, 3, +1.0)
    um, inter = oracle.exp(phi, 3, -1.0, intermediates=True)
    oracle.exp_adjoint(phi, 3, -1.0, rng.normal(size=up.shape))
    N = 4
    ups = np.stack([up] * (N - 1)); ums = np.stack([um] * (N - 1))
    U = oracle.compose(ups, ums)
    oracle.compose_adjoint(ups, ums, rng.normal(size=U.shape))
    Ut = oracle.upsample(U[1, 0], shape)
    oracle.upsample_adjoint(rng.normal(size=Ut.shape), nf)
    I = rng.uniform(size=shape)
    W = oracle.warp(I, Ut)
    oracle.warp_adjoint(I, Ut, rng.normal(size=W.shape))
    for w in (3, 5, 13):                              # 13: no window fits
        for kind in (oracle.SILNCC, oracle.LNCC):
            oracle.similarity(I, W, w, kind, 1e-6, grad=True)
    oracle.regulariser(rng.normal(size=(N - 1, 3) + nf), np.array([0.0, 1.0, 2.5, 4.0]), grad=True)
    oracle.downsample2(I)
    oracle.jacobian_det(rng.normal(size=(3,) + shape))
    roi = rng.uniform(size=shape) > 0.5
    oracle.deformation_metrics(rng.normal(size=(3,) + shape), rng.normal(size=(3,) + shape), roi)
    oracle.deformation_metrics(rng.normal(size=(3,) + shape), rng.normal(size=(3,) + shape), np.zeros(shape, bool))
    oracle.smooth(rng.normal(size=shape), 0.2, (1.0, 1.5, 2.0))
    oracle.sample(I, np.array([-3.0, 100.0, 0.5]))

for nc, nfine in [((3, 4, 5), (5, 8, 9)), ((1, 2, 2), (2, 3, 4))]:
    oracle.prolong(rng.normal(size=(3,) + nc), nfine)

imgs = rng.uniform(size=(3, 13, 10, 9))
for kind in (oracle.SILNCC, oracle.LNCC):
    p = oracle.params(n_levels=2, steps=(3, 2), K=3, window=3, sim_kind=kind, alpha_ts=0.1)
    oracle.run(imgs, p, t=np.array([0.0, 1.0, 3.0]), loss_history=True)
p = oracle.params(n_levels=2, steps=(2, 2), K=2, window=3, rigid=1, smooth_omega=0.3, spacing=(1.0, 1.2, 0.9))
oracle.run(imgs, p, loss_history=True)
nf = tuple((a + 1) // 2 for a in imgs.shape[1:])
oracle.loss_grad_rigid(imgs, rng.normal(size=(2, 3) + nf) * 0.3, rng.normal(size=(2, 6)) * 0.1,
                       oracle.params(n_levels=1, steps=(1,), K=3, window=3), tscale=2.0)
th = rng.normal(size=(2, 3) + nf)
m, v = np.zeros_like(th), np.zeros_like(th)
oracle.adam_step(th, m, v, rng.normal(size=th.shape), 1, oracle.lr_at(1, 10, 0.1))
oracle.rotation(np.array([0.1, -0.2, 0.3]))
print("SANITIZED-OK")
"""


def _runtime(name):
    gcc = shutil.which("gcc")
    if not gcc:
        return None
    path = subprocess.run([gcc, "-print-file-name=" + name], capture_output=True, text=True).stdout.strip()
    return path if os.path.isabs(path) and os.path.exists(path) else None


def test_oracle_is_clean_under_address_and_undefined_behaviour_sanitizers(tmp_path):
    asan = _runtime("libasan.so")
    if asan is None or _runtime("libubsan.so") is None:
        pytest.skip("gcc sanitizer runtimes are not installed")
    lib = str(tmp_path / "libmuster_oracle_asan.so")
    src = os.path.join(ROOT, "oracle", "muster_oracle.c")
    subprocess.run(["gcc", "-O1", "-g", "-std=c11", "-fopenmp", "-fPIC", "-shared", "-fno-omit-frame-pointer",
                    "-fsanitize=address,undefined", "-fno-sanitize-recover=undefined", "-o", lib, src, "-lm"],
                   check=True)
    env = dict(os.environ)
    env.update(LD_PRELOAD=asan, ASAN_OPTIONS="detect_leaks=0:halt_on_error=1",
               UBSAN_OPTIONS="halt_on_error=1:print_stacktrace=1", OMP_NUM_THREADS="2",
               PYTHONPATH=ROOT + os.pathsep + env.get("PYTHONPATH", ""))
    r = subprocess.run([sys.executable, "-c", "LIB = %r\n" % lib + CHILD], capture_output=True, text=True,
                       env=env, cwd=ROOT, timeout=600)
    report = r.stdout[-4000:] + r.stderr[-4000:]
    assert r.returncode == 0 and "SANITIZED-OK" in r.stdout, report
    assert "AddressSanitizer" not in r.stderr and "runtime error" not in r.stderr, report
