"""The device helpers' integer-arithmetic conversions (binary64 -> binary32
round-to-nearest-even, int -> binary64; used by the set-up kernel to keep
its FP64 pipe free) equal the hardware conversions bit for bit over 2^28
random and edge-case inputs (conv_check.cu, built here with nvcc)."""
import os
import shutil
import subprocess

import pytest

HERE = os.path.dirname(os.path.abspath(__file__))
CSRC = os.path.join(HERE, "..", "paper_2202_11001_gb300", "csrc")


@pytest.mark.gpu
def test_integer_conversions_equal_hardware(tmp_path):
    nvcc = shutil.which("nvcc") or "/usr/local/cuda/bin/nvcc"
    exe = str(tmp_path / "conv_check")
    subprocess.run([nvcc, "-gencode", "arch=compute_103a,code=sm_103a", "-O3", "-std=c++17", "-I", CSRC, "-o", exe,
                    os.path.join(HERE, "conv_check.cu")], check=True, capture_output=True)
    out = subprocess.run([exe], capture_output=True, text=True, timeout=120)
    assert out.returncode == 0 and "mismatches 0" in out.stdout, out.stdout + out.stderr
