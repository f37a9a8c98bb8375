"""The integer-pipe FP64 -> FP32 rounding that the FP32 form applies to the FP64
geometry (csrc/f64conv.cuh) equals the hardware conversion __double2float_rn bit
for bit (tests/convert_check.cu: 2^27 values including exact ties, near-ties,
exponent carries, zeros and out-of-range inputs)."""
import os
import shutil
import subprocess
import tempfile

import pytest

pytestmark = pytest.mark.gpu

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def test_integer_rounding_matches_hardware_conversion():
    nvcc = shutil.which("nvcc") or "/usr/local/cuda/bin/nvcc"
    with tempfile.TemporaryDirectory() as d:
        exe = os.path.join(d, "convert_check")
        subprocess.run([nvcc, "-gencode", "arch=compute_103a,code=sm_103a", "-O3", "-I",
                        os.path.join(ROOT, "paper_1404_0405_gb300", "csrc"),
                        os.path.join(ROOT, "tests", "convert_check.cu"), "-o", exe], check=True)
        r = subprocess.run([exe], capture_output=True, text=True, timeout=300)
    print(r.stdout)
    assert r.returncode == 0, r.stdout + r.stderr
    assert "mismatches 0" in r.stdout
