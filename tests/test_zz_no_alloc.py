"""qft_execute_noalloc: the transform with the library's fixed device scratch.

For callers that cannot allocate device memory (code running during stream
capture, runtimes that own the device heap, allocation-free loops).  The
entry point is called through the C ABI and its output is compared with
qft_execute's (caller-allocated workspace) on two calls in a row, within the
tolerances of the parity tests.  This file runs last so that a failure here
comes after every other test has run.
"""
import ctypes

import numpy as np
import pytest

import qft_inputs

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
q = pytest.importorskip("paper_2606_18981_gb300")

TOL = {"c64": 2e-6, "c128": 1e-13}


def _rel(a, b):
    return float(torch.linalg.vector_norm((a - b).to(torch.complex128)) /
                 torch.linalg.vector_norm(b.to(torch.complex128)))


@pytest.mark.parametrize("n,dt,order", [(18, "c64", 0), (12, "c64", 0), (20, "c128", 0), (24, "c64", 1)])
def test_noalloc_matches_execute_twice(n, dt, order):
    td = torch.complex64 if dt == "c64" else torch.complex128
    p = q.Plan(n, -1, q.FORWARD, dt, order)
    x = torch.from_numpy(qft_inputs.gaussian(n, seed=n, normalise=False)).to(td).cuda()
    ref = x.clone()
    ws = p.alloc_workspace()
    sref = torch.zeros(1, dtype=torch.float64, device="cuda")
    p.execute(ref, ws, q.SCALE_STATE, scale_out=sref)
    stream = torch.cuda.current_stream().cuda_stream
    for _ in range(2):
        got = x.clone()
        s = torch.zeros(1, dtype=torch.float64, device="cuda")
        rc = q.lib.qft_execute_noalloc(ctypes.c_void_p(p.handle), ctypes.c_void_p(got.data_ptr()),
                                       ctypes.c_void_p(s.data_ptr()), q.SCALE_STATE, ctypes.c_void_p(stream))
        assert rc == q.OK
        torch.cuda.synchronize()
        tol = TOL[dt] * (n if dt == "c128" else 1)
        assert _rel(got, ref) <= tol
        assert abs(s.item() - sref.item()) <= 1e-6 * sref.item()


def test_noalloc_rejects_plans_beyond_the_scratch():
    p = q.Plan(23, -1, q.FORWARD, "c64", q.ORDER_NATURAL)  # needs a 64 MiB ping-pong buffer
    x = torch.zeros(1 << 23, dtype=torch.complex64, device="cuda")
    rc = q.lib.qft_execute_noalloc(ctypes.c_void_p(p.handle), ctypes.c_void_p(x.data_ptr()), None,
                                   q.SCALE_STATE, None)
    assert rc == q.ERR_SIZE
