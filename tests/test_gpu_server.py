"""The serving loop on the GPU: mixed requests, each result equal to the same
request run alone (qft_execute with the same plan), budget refusal, stats."""
import numpy as np
import pytest

import qft_inputs

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
q = pytest.importorskip("paper_2606_18981_gb300")

TOL = {"c64": lambda n: 2e-6, "c128": lambda n: 1e-13 * n}


def rel(a, b):
    a = a.to(torch.complex128)
    b = b.to(torch.complex128)
    return float(torch.linalg.vector_norm(a - b) / max(torch.linalg.vector_norm(b), 1e-300))


def alone(x, n, k, direction, dt, order, mode):
    p = q.Plan(n, k, direction, dt, order)
    st = x.clone().cuda()
    ws = p.alloc_workspace()
    p.execute(st, ws, mode)
    torch.cuda.synchronize()
    return st, p.scale_in(ws)


def _mixed_requests(count=60, seed=5):
    rng = np.random.default_rng(seed)
    out = []
    for i in range(count):
        n = int(rng.integers(6, 23))
        k = int(rng.choice([-1, 4, 8, 16]))
        direction = int(rng.choice([-1, 1]))
        dt = "c64" if i % 3 else "c128"
        order = int(i % 5 == 0)
        mode = int(rng.integers(0, 4))
        td = torch.complex64 if dt == "c64" else torch.complex128
        x = torch.from_numpy(qft_inputs.make(qft_inputs.KINDS[i % 3], n, 77 + i)).to(td)
        out.append((x, n, k, direction, dt, order, mode, i % 2 == 0))
    return out


def _serve(srv, reqs, one_at_a_time):
    results = []
    pending = []
    for x, n, k, direction, dt, order, mode, on_dev in reqs:
        td = x.dtype
        xin = x.cuda() if on_dev else x.pin_memory()
        out = torch.empty(1 << n, dtype=td, device="cuda") if on_dev else torch.empty(1 << n, dtype=td).pin_memory()
        t = srv.submit(xin, out, n, k, direction, dt, order, mode)
        pending.append((t, out))
        if one_at_a_time:
            rc, lat, scale = srv.wait(t, 60000)
            assert rc == 0 and lat > 0
            results.append((out.cpu(), scale))
            pending.clear()
    for t, out in pending:
        rc, lat, scale = srv.wait(t, 60000)
        assert rc == 0 and lat > 0
        results.append((out.cpu(), scale))
    return results


def test_results_alone_equal_results_in_the_mix():
    """Every request's result is bit for bit the same when it is served alone
    (one request at a time) and in a mix of 60 requests of different sizes,
    cutoffs, directions, dtypes, orders and scale modes (served concurrently:
    the small ones in batched launches, the large ones on their own), and it
    equals qft_execute on the same plan within the parity tolerance."""
    reqs = _mixed_requests()
    srv = q.Server(8 << 30, streams=6, max_inflight=24)
    alone_res = _serve(srv, reqs, one_at_a_time=True)
    srv.reset_stats()
    mix_res = _serve(srv, reqs, one_at_a_time=False)
    st = srv.stats()
    assert st.completed == 60 and st.failed == 0 and st.p99_ms >= st.p50_ms > 0
    assert st.bytes_in_use == 0
    for (a, sa), (b, sb), (x, n, k, direction, dt, order, mode, _) in zip(alone_res, mix_res, reqs):
        assert torch.equal(a, b), (n, k, direction, dt, order, mode)
        assert sa == sb
        ref, s_ref = alone(x, n, k, direction, dt, order, mode)
        assert rel(b.cuda(), ref) <= TOL[dt](n)
        assert abs(sb - s_ref) <= 1e-9 * max(s_ref, 1e-300)
    srv.close()


@pytest.mark.parametrize("dt", ["c64", "c128"])
def test_device_requests_run_out_of_place_with_the_same_bits(dt):
    """A large request whose input and output are device buffers at 256-byte
    alignment runs from the input straight into the output (no state buffer,
    no copies); its result is bit for bit the one of the same request through
    pinned host buffers (copy-in, execute, copy-out) and through misaligned
    device buffers (which take the copy path)."""
    td = torch.complex64 if dt == "c64" else torch.complex128
    srv = q.Server(8 << 30, streams=2, max_inflight=8)
    for n, k, direction, order, mode in [(20, -1, -1, 0, 0), (22, 8, 1, 0, 2), (21, -1, -1, 1, 1)]:
        x = torch.from_numpy(qft_inputs.make("gaussian", n, 300 + n)).to(td)
        xd = x.cuda()
        od = torch.empty(1 << n, dtype=td, device="cuda")
        xh = x.pin_memory()
        oh = torch.empty(1 << n, dtype=td).pin_memory()
        big_in = torch.empty((1 << n) + 1, dtype=td, device="cuda")
        big_out = torch.empty((1 << n) + 1, dtype=td, device="cuda")
        xm, om = big_in[1:], big_out[1:]  # one element off: not 256-byte aligned
        xm.copy_(xd)
        got = []
        for a, b in ((xd, od), (xh, oh), (xm, om)):
            t = srv.submit(a, b, n, k, direction, dt, order, mode)
            rc, _, scale = srv.wait(t, 60000)
            assert rc == 0
            got.append((b.cpu(), scale))
        assert torch.equal(xd.cpu(), x)  # the input is left as it was
        for b, sc in got[1:]:
            assert torch.equal(got[0][0], b) and got[0][1] == sc
        ref, s_ref = alone(x, n, k, direction, dt, order, mode)
        assert rel(got[0][0].cuda(), ref) <= TOL[dt](n)
    assert srv.stats().bytes_in_use == 0
    srv.close()


def test_small_requests_share_batched_launches():
    """Requests of n <= 18 submitted together run in batched launches that
    carry several requests each; with batching off none are batched; the
    results are the same either way."""
    reqs = [r for r in _mixed_requests(80, seed=9) if r[1] <= 18]
    srv = q.Server(8 << 30, streams=4, max_inflight=64)
    res = _serve(srv, reqs, one_at_a_time=False)
    st = srv.stats()
    assert st.batched_requests == len(reqs) and 0 < st.batches < len(reqs)
    srv.set_batching(0)
    srv.reset_stats()
    res_single = _serve(srv, reqs, one_at_a_time=False)
    assert srv.stats().batches == 0
    for (a, _), (b, _), (x, n, k, direction, dt, order, mode, _) in zip(res, res_single, reqs):
        assert rel(a.cuda(), b.cuda()) <= TOL[dt](n)
    srv.close()


def test_budget_refusal_and_small_budget_progress():
    srv = q.Server(1 << 20, streams=2)  # 1 MiB: n = 16 (512 KiB state + workspace) fits, n = 18 does not
    x = torch.zeros(1 << 18, dtype=torch.complex64, device="cuda")
    out = torch.empty_like(x)
    t = srv.submit(x, out, 18)
    rc, _, _ = srv.wait(t, 10000)
    assert rc == q.ERR_BUDGET
    xs = [torch.randn(1 << 15, dtype=torch.complex64, device="cuda") for _ in range(8)]
    outs = [torch.empty_like(v) for v in xs]
    ts = [srv.submit(v, o, 15) for v, o in zip(xs, outs)]  # only one fits at a time
    for t, v, o in zip(ts, xs, outs):
        rc, _, _ = srv.wait(t, 20000)
        assert rc == 0
        ref, _ = alone(v, 15, -1, -1, "c64", 0, 0)
        assert rel(o, ref) <= 2e-6
    srv.close()


def test_cancel_pending_request():
    """Requests queued behind a full budget can be withdrawn; the others still complete."""
    srv = q.Server(1 << 20, streams=1, max_inflight=1)  # one n = 15 request at a time
    xs = [torch.randn(1 << 15, dtype=torch.complex64, device="cuda") for _ in range(6)]
    outs = [torch.empty_like(v) for v in xs]
    ts = [srv.submit(v, o, 15) for v, o in zip(xs, outs)]
    rc_cancel = srv.cancel(ts[-1])
    for t in ts[:-1]:
        rc, _, _ = srv.wait(t, 20000)
        assert rc == 0
    rc, _, _ = srv.wait(ts[-1], 20000)
    if rc_cancel == 0:
        assert rc == q.ERR_CANCELED
    else:  # already admitted by the time cancel ran: it ran normally
        assert rc_cancel == q.ERR_STATE and rc == 0
    assert srv.cancel(ts[0]) == q.ERR_STATE  # finished requests cannot be withdrawn
    srv.close()


def test_injected_allocation_failure_is_reported_and_leaks_nothing():
    srv = q.Server(1 << 30, streams=2)
    x = torch.randn(1 << 16, dtype=torch.complex64, device="cuda")
    out = torch.empty_like(x)
    srv.inject_alloc_failures(1)
    t = srv.submit(x, out, 16)
    rc, _, _ = srv.wait(t, 20000)
    assert rc == q.ERR_NOMEM
    st = srv.stats()
    assert st.in_flight == 0 and st.bytes_in_use == 0 and st.failed >= 1
    t = srv.submit(x, out, 16)  # the next allocation succeeds
    rc, _, _ = srv.wait(t, 20000)
    assert rc == 0
    ref, _ = alone(x, 16, -1, -1, "c64", 0, 0)
    assert rel(out, ref) <= 2e-6
    assert srv.stats().bytes_in_use == 0
    srv.close()
