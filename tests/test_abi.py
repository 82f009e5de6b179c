"""The C ABI library loads and exports every function include/*.h declares (no GPU needed)."""
import ctypes
import glob
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
LIB = os.path.join(ROOT, "paper_2606_18981_gb300", "libqftfft.so")


def declared_functions():
    names = set()
    for h in glob.glob(os.path.join(ROOT, "include", "*.h")):
        text = open(h).read()
        text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
        for m in re.finditer(r"^[A-Za-z_][\w\s\*]*?\b(qft_\w+)\s*\(", text, flags=re.M):
            names.add(m.group(1))
    return sorted(names)


def test_header_declares_functions():
    names = declared_functions()
    assert "qft_plan_create" in names and "qft_execute" in names and len(names) >= 10


def test_library_exports_every_declared_symbol():
    if not os.path.exists(LIB):
        pytest.fail("libqftfft.so is not built (run __graft_entry__.build())")
    lib = ctypes.CDLL(LIB)
    missing = [n for n in declared_functions() if not hasattr(lib, n)]
    assert not missing, f"declared but not exported: {missing}"


def test_strerror_and_version():
    lib = ctypes.CDLL(LIB)
    lib.qft_strerror.restype = ctypes.c_char_p
    assert lib.qft_strerror(0) == b"ok"
    assert lib.qft_strerror(-2).startswith(b"length")
    assert lib.qft_version() > 0


def test_load_rejects_bad_sizes():
    import paper_2606_18981_gb300 as q

    p = q.Plan(4)
    dummy = ctypes.c_void_p(256)
    # len != 2^n -> QFT_ERR_SIZE before any CUDA call
    assert q.lib.qft_load(p._h, dummy, dummy, 15, 1, None) == q.ERR_SIZE
    assert q.lib.qft_load(p._h, dummy, dummy, 0, 1, None) == q.ERR_SIZE
    assert q.lib.qft_load(None, dummy, dummy, 16, 1, None) == q.ERR_BAD_ARG
    # misaligned device pointers are refused before any launch
    assert q.lib.qft_execute(p._h, ctypes.c_void_p(8), dummy, None, 0, None) == q.ERR_BAD_ARG
    assert q.lib.qft_execute(p._h, dummy, dummy, None, 9, None) == q.ERR_BAD_ARG
