"""Host check of the batched launch's queue order (csrc/batch_order.hpp),
compiled and run on the CPU (tests/native/batch_order_check.cpp): every group
queued once, dependencies only on earlier items, later passes at least a
block behind their predecessors, runs of one pass shape per block; and a
simulation of the kernel's claim protocol (claim the next item while
computing, wait for its producers after) on such orders, which must always
finish (a queue with later passes first does not: the simulation reports it)."""
import os
import shutil
import subprocess

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def test_wavefront_queue_order(tmp_path):
    cxx = shutil.which("g++") or shutil.which("c++")
    if cxx is None:
        pytest.skip("no C++ compiler")
    exe = str(tmp_path / "batch_order_check")
    src = os.path.join(ROOT, "tests", "native", "batch_order_check.cpp")
    inc = os.path.join(ROOT, "paper_2606_18981_gb300", "csrc")
    r = subprocess.run([cxx, "-std=c++17", "-O2", f"-I{inc}", "-o", exe, src], capture_output=True, text=True)
    assert r.returncode == 0, r.stdout + r.stderr
    r = subprocess.run([exe], capture_output=True, text=True, timeout=300)
    assert r.returncode == 0 and "ALL OK" in r.stdout, r.stdout + r.stderr
