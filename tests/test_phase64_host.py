"""Host pins of the phase-estimation sweep's complex64 phase evaluation:
the exact quarter-turn reduction of a 64-bit fixed-point phase and the FP32
Taylor sine/cosine of the rest, run on the CPU from the kernel's own
__host__ __device__ functions against long double (tests/native/phase64_check.cu)."""
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


def test_phase64_f32_against_long_double(tmp_path):
    nvcc = _nvcc()
    if nvcc is None:
        pytest.skip("nvcc not available")
    exe = str(tmp_path / "phase64_check")
    src = os.path.join(ROOT, "tests", "native", "phase64_check.cu")
    inc = os.path.join(ROOT, "paper_2606_18981_gb300", "csrc")
    r = subprocess.run([nvcc, "-std=c++17", "-O2", f"-I{inc}", "-o", exe, src], capture_output=True, text=True)
    assert r.returncode == 0, r.stdout + r.stderr
    r = subprocess.run([exe], capture_output=True, text=True, timeout=300)
    print(r.stdout)
    assert r.returncode == 0 and "ALL OK" in r.stdout, r.stdout + r.stderr
