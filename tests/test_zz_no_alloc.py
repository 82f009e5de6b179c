"""qft_execute_noalloc: the transform with the library's fixed device scratch.

For callers that cannot allocate device memory (code running during stream
capture, runtimes that own the device heap, allocation-free loops).  The
entry point is called through the C ABI and its output is compared with
qft_execute's (caller-allocated workspace) on two calls in a row, within the
tolerances of the parity tests.  Also covered: the exact size limit of the
scratch (accepted at 32 MiB + 4 KiB, rejected one size up), the status
reader qft_noalloc_status (a wait made to expire on purpose), the refusal of
tensor-core tier plans before their first execute (which would allocate),
and the call captured into a CUDA graph and replayed.  This file runs last
so that a failure here comes after every other test has run.
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


def _call(p, state, scale_ptr=None, stream=None, mode=None):
    return q.lib.qft_execute_noalloc(ctypes.c_void_p(p.handle), ctypes.c_void_p(state.data_ptr()),
                                     ctypes.c_void_p(scale_ptr) if scale_ptr else None,
                                     q.SCALE_STATE if mode is None else mode,
                                     ctypes.c_void_p(stream) if stream else None)


@pytest.mark.parametrize("n,dt", [(22, "c64"), (21, "c128")])
def test_noalloc_at_the_exact_scratch_limit(n, dt):
    """Natural-order multi-pass plans at n = 22 (complex64) and n = 21
    (complex128) need exactly 32 MiB + 4 KiB, the whole scratch: accepted and
    equal to qft_execute; one size up is rejected."""
    td = torch.complex64 if dt == "c64" else torch.complex128
    p = q.Plan(n, -1, q.FORWARD, dt, q.ORDER_NATURAL)
    assert p.info().workspace_bytes == (32 << 20) + 4096
    x = torch.from_numpy(qft_inputs.gaussian(n, seed=3, normalise=False)).to(td).cuda()
    ref = x.clone()
    p.execute(ref, p.alloc_workspace(), q.SCALE_STATE)
    got = x.clone()
    assert _call(p, got) == q.OK
    torch.cuda.synchronize()
    assert _rel(got, ref) <= TOL[dt] * (n if dt == "c128" else 1)
    big = q.Plan(n + 1, -1, q.FORWARD, dt, q.ORDER_NATURAL)
    y = torch.zeros(1 << (n + 1), dtype=td, device="cuda")
    assert _call(big, y) == q.ERR_SIZE


def test_noalloc_status_reports_an_expired_wait():
    """A plan whose first tile load is never issued (test hook) with a 20 ms
    wait limit: the call returns QFT_OK (the kernels are asynchronous), and
    qft_noalloc_status reports QFT_ERR_TIMEOUT; the next good call clears it."""
    n = 18
    bad = q.Plan(n, -1, q.FORWARD, "c64", q.ORDER_NATURAL, wait_limit_ms=20, test_skip_first_load=1)
    x = torch.zeros(1 << n, dtype=torch.complex64, device="cuda")
    assert _call(bad, x) == q.OK
    assert q.lib.qft_noalloc_status(None) == q.ERR_TIMEOUT
    good = q.Plan(n, -1, q.FORWARD, "c64", q.ORDER_NATURAL)
    y = torch.from_numpy(qft_inputs.gaussian(n, seed=1)).to(torch.complex64).cuda()
    assert _call(good, y) == q.OK
    assert q.lib.qft_noalloc_status(None) == q.OK


def test_noalloc_refuses_tensor_tier_plans_before_their_first_execute():
    """A tensor-core tier plan uploads its block matrices on its first
    qft_execute; before that the allocation-free call refuses it, after it the
    call runs and matches qft_execute."""
    n = 14
    p = q.Plan(n, -1, q.FORWARD, "c64", q.ORDER_NATURAL, precision=q.PREC_FP16X3)
    x = torch.from_numpy(qft_inputs.gaussian(n, seed=2)).to(torch.complex64).cuda()
    got = x.clone()
    assert _call(p, got) == q.ERR_UNSUPPORTED
    ref = x.clone()
    p.execute(ref, p.alloc_workspace(), q.SCALE_STATE)
    assert _call(p, got) == q.OK
    torch.cuda.synchronize()
    assert torch.equal(got, ref)


def test_noalloc_captured_in_a_graph():
    """The use named in the header: one warm-up call on the device (it caches
    the scratch address), then the call captured into a CUDA graph on a side
    stream and the graph replayed twice; each replay equals qft_execute."""
    n = 18
    p = q.Plan(n, -1, q.FORWARD, "c64", q.ORDER_NATURAL)
    x = torch.from_numpy(qft_inputs.gaussian(n, seed=9, normalise=False)).to(torch.complex64).cuda()
    ref = x.clone()
    p.execute(ref, p.alloc_workspace(), q.SCALE_STATE)
    state = x.clone()
    side = torch.cuda.Stream()
    with torch.cuda.stream(side):
        assert _call(p, state, stream=side.cuda_stream) == q.OK  # warm-up, outside the capture
    torch.cuda.synchronize()
    g = torch.cuda.CUDAGraph()
    with torch.cuda.graph(g, stream=side):
        rc = _call(p, state, stream=side.cuda_stream)
    assert rc == q.OK
    for _ in range(2):
        state.copy_(x)
        torch.cuda.synchronize()
        g.replay()
        torch.cuda.synchronize()
        assert _rel(state, ref) <= TOL["c64"]
    assert q.lib.qft_noalloc_status(None) == q.OK
