"""The tile geometry of the step kernels, checked on the host: the staging
box, slope and flux index maps of every compiled tile shape are
collision-free and in range in both layouts, and the quad kernel's layout
has the odd rows that keep its y-running halo work items on distinct
shared-memory bank groups (tests/_tile_geometry.cu, built with nvcc for the
host only; no GPU is used)."""
import os
import shutil
import subprocess
import tempfile

import pytest

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(HERE)


def test_tile_geometry_maps():
    nvcc = shutil.which(os.environ.get("NVCC", "nvcc"))
    if nvcc is None:
        pytest.skip("nvcc not found")
    with tempfile.TemporaryDirectory() as tmp:
        exe = os.path.join(tmp, "tile_geometry")
        cmd = [nvcc, "-std=c++17", "-O1", "-gencode", "arch=compute_103a,code=sm_103a",
               "-I", os.path.join(ROOT, "include"), "-I", os.path.join(ROOT, "paper_1403_6126_gb300", "csrc"),
               os.path.join(HERE, "_tile_geometry.cu"), "-o", exe]
        b = subprocess.run(cmd, capture_output=True, text=True, timeout=600)
        assert b.returncode == 0, b.stderr[-3000:]
        r = subprocess.run([exe], capture_output=True, text=True, timeout=120)
        assert r.returncode == 0 and r.stdout.strip().endswith("OK"), (r.stdout[-3000:], r.stderr[-2000:])
