"""Launch geometry of the image-grid kernels, checked on the host (no GPU): the C++ program
launch_geometry.cu, linked against the built library, walks shapes from 1 to 4096 voxels per
axis, every window and pair batches up to 992, and checks that the D chunks cover each depth
exactly once and that no batch needs more chunks or CTAs per pair than a batch of one pair,
which is what the engine sizes its partial-sum buffers and its grid-row cap by."""
import os
import shutil
import subprocess

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def test_chunks_cover_the_depth_and_batch_one_bounds_every_batch(tmp_path):
    from paper_2412_14671_gb300 import build

    nvcc = build._nvcc()
    if not shutil.which(nvcc):
        pytest.skip("nvcc missing")
    lib = build.build()
    exe = str(tmp_path / "launch_geometry")
    subprocess.run([nvcc, *build.ARCH, "-std=c++17", "-I", build.INCLUDE, "-I", build.CSRC,
                    os.path.join(ROOT, "tests", "launch_geometry.cu"), "-L", os.path.dirname(lib), "-lmuster",
                    "-Xlinker", "-rpath=" + os.path.dirname(lib), "-o", exe], check=True)
    r = subprocess.run([exe], capture_output=True, text=True, timeout=300)
    assert r.returncode == 0 and "GEOMETRY-OK" in r.stdout, r.stdout + r.stderr
    assert int(r.stdout.split()[-1]) > 400_000
