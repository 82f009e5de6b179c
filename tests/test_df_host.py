"""Host-side pins of the double-float arithmetic used by the complex128 pass
kernel: the FP64 <-> FP32-pair conversions (with the exponent shift of the
range normalisation) and the error-free sum / product building blocks, run on
the CPU from the kernel's own __host__ __device__ functions against long
double arithmetic (tests/native/df_host_check.cu)."""
import os
import shutil
import subprocess

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _nvcc():
    for c in (shutil.which("nvcc"), "/usr/local/cuda/bin/nvcc"):
        if c and os.path.exists(c):
            return c
    return None


def test_df_conversions_and_arithmetic(tmp_path):
    nvcc = _nvcc()
    if nvcc is None:
        pytest.skip("nvcc not available")
    exe = str(tmp_path / "df_host_check")
    src = os.path.join(ROOT, "tests", "native", "df_host_check.cu")
    inc = os.path.join(ROOT, "paper_2606_18981_gb300", "csrc")
    r = subprocess.run([nvcc, "-std=c++17", "-O2", f"-I{inc}", "-o", exe, src], capture_output=True, text=True)
    assert r.returncode == 0, r.stdout + r.stderr
    r = subprocess.run([exe], capture_output=True, text=True, timeout=300)
    print(r.stdout)
    assert r.returncode == 0 and "ALL OK" in r.stdout, r.stdout + r.stderr
