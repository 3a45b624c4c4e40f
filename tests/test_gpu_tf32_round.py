"""The TF32 rounding of the tensor-core kernels is done with integer operations
(half a TF32 unit added to the bit pattern, the 13 low bits cleared).  This test
compiles a small CUDA program against the library's own header and checks that
rounding against the hardware conversion cvt.rna.tf32.f32 on every non-NaN
32-bit pattern, and the big + small split on a sample of them."""
import os
import shutil
import subprocess

import pytest

pytestmark = pytest.mark.gpu

HERE = os.path.dirname(os.path.abspath(__file__))
CSRC = os.path.join(HERE, "..", "paper_2211_12709_gb300", "csrc")


def test_integer_tf32_rounding_matches_the_hardware_conversion(tmp_path):
    nvcc = shutil.which("nvcc") or "/usr/local/cuda/bin/nvcc"
    exe = str(tmp_path / "tf32_round_check")
    subprocess.run([nvcc, "-gencode", "arch=compute_103a,code=sm_103a", "-O3", "-I", CSRC,
                    os.path.join(HERE, "cuda", "tf32_round_check.cu"), "-o", exe], check=True)
    out = subprocess.run([exe], capture_output=True, text=True, timeout=300)
    print(out.stdout)
    assert out.returncode == 0, out.stdout + out.stderr
    assert "round mismatches 0 split mismatches 0" in out.stdout
