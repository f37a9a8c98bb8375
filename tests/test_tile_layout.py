"""The structured trend's shared-memory layout and per-patch geometry blocks
(csrc/sww_tile.cuh), checked on the host for every working precision and patch
side (tests/tile_layout_check.cu): the alignments and sizes the bulk copies, the
element copies and the mbarriers need, and the shared memory of a block.  Runs
without a GPU (nvcc compiles the check; no device call)."""
import os
import shutil
import subprocess
import tempfile

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def test_tile_layout():
    nvcc = shutil.which("nvcc") or "/usr/local/cuda/bin/nvcc"
    if not os.path.exists(nvcc):
        pytest.skip("nvcc not found")
    with tempfile.TemporaryDirectory() as d:
        exe = os.path.join(d, "tile_layout_check")
        subprocess.run([nvcc, "-gencode", "arch=compute_103a,code=sm_103a", "-std=c++17", "--extended-lambda",
                        "-I", os.path.join(ROOT, "include"), "-I", os.path.join(ROOT, "paper_1404_0405_gb300", "csrc"),
                        os.path.join(ROOT, "tests", "tile_layout_check.cu"), "-o", exe], check=True)
        r = subprocess.run([exe], capture_output=True, text=True, timeout=60)
    print(r.stdout)
    assert r.returncode == 0, r.stdout + r.stderr
    assert "tile layout ok" in r.stdout
