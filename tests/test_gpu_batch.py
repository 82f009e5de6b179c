"""Batched execution on the GPU: one persistent launch over many uneven transforms.

Every transform of a mixed batch must give the result it gives alone
(qft_execute with the same plan), within the parity tolerances; a sample is
also checked against the CPU oracle.  Graph capture and replay of the batch
launch must reproduce the same results.
"""
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


def make_batch(count, nmin, nmax, dt, order, seed, direction=q.FORWARD, opts=None):
    rng = np.random.default_rng(seed)
    td = torch.complex64 if dt == "c64" else torch.complex128
    plans, xs, ks = {}, [], []
    specs = []
    for i in range(count):
        n = int(rng.integers(nmin, nmax + 1))
        k = int(rng.choice([4, 8, n]))
        kind = qft_inputs.KINDS[i % 3]
        specs.append((n, k, kind))
    for i, (n, k, kind) in enumerate(specs):
        key = (n, k)
        if key not in plans:
            plans[key] = q.Plan(n, k, direction, dt, order, **(opts or {}))
        xs.append(torch.from_numpy(qft_inputs.make(kind, n, seed * 1000 + i)).to(td).cuda())
    return specs, plans, xs


# plan shapes: defaults; 2^12-amplitude tiles (the batch runs two CTAs per SM);
# 512-thread plans (the batch runs 512-thread CTAs)
@pytest.mark.parametrize("dt,order,opts", [("c64", 0, None), ("c64", 1, None), ("c128", 0, None),
                                           ("c128", 1, None), ("c128", 0, {"threads": 512}),
                                           ("c128", 0, {"precision": q.PREC_FP64}),
                                           ("c64", 0, {"tile_bits": 12}), ("c64", 1, {"tile_bits": 12}),
                                           ("c64", 0, {"threads": 512}), ("c64", 1, {"threads": 512})])
def test_batch_matches_single_transforms(oracle_mod, dt, order, opts):
    specs, plans, xs = make_batch(96, 3, 17, dt, order, seed=7, opts=opts)
    states = [x.clone() for x in xs]
    scales = torch.zeros(len(xs), dtype=torch.float64, device="cuda")
    b = q.Batch([plans[(n, k)] for n, k, _ in specs], states, q.SCALE_STATE, scale_out=scales)
    b.execute()
    assert b.status() == 0
    for i, (n, k, _) in enumerate(specs):
        p = plans[(n, k)]
        ref = xs[i].clone()
        ws = p.alloc_workspace()
        p.execute(ref, ws, q.SCALE_STATE)
        torch.cuda.synchronize()
        assert rel(states[i], ref) <= TOL[dt](n), (i, n, k)
        assert abs(scales[i].item() - p.scale_in(ws)) <= 1e-6 * max(p.scale_in(ws), 1e-300)
    for i in (0, 1, 2, 50, 95):
        n, k, _ = specs[i]
        want, _ = oracle_mod.qft(xs[i].cpu().numpy().astype(np.complex128), k, -1, 0, order == 0)
        got = states[i].cpu().numpy().astype(np.complex128)
        err = np.linalg.norm(got - want) / np.linalg.norm(want)
        assert err <= TOL[dt](n)


def test_batch_graph_capture_replay():
    specs, plans, xs = make_batch(64, 8, 18, "c64", 0, seed=11)
    states = [x.clone() for x in xs]
    b = q.Batch([plans[(n, k)] for n, k, _ in specs], states, q.SCALE_STATE)
    s = torch.cuda.Stream()
    with torch.cuda.stream(s):
        b.execute(stream=s)
    torch.cuda.synchronize()
    first = [st.clone() for st in states]
    g = torch.cuda.CUDAGraph()
    with torch.cuda.graph(g, stream=s):
        b.execute(stream=s)
    for _ in range(2):
        for st, x in zip(states, xs):
            st.copy_(x)
        g.replay()
        torch.cuda.synchronize()
        for st, f in zip(states, first):
            assert torch.equal(st, f)


def test_batch_inverse_round_trip():
    specs, plans, xs = make_batch(40, 5, 16, "c64", 0, seed=3)
    inv = {key: q.Plan(key[0], key[1], q.INVERSE, "c64", 0) for key in plans}
    states = [x.clone() for x in xs]
    q.Batch([plans[(n, k)] for n, k, _ in specs], states, q.SCALE_UNITARY).execute()
    q.Batch([inv[(n, k)] for n, k, _ in specs], states, q.SCALE_UNITARY).execute()
    torch.cuda.synchronize()
    for st, x, (n, _, _) in zip(states, xs, specs):
        assert rel(st, x) <= 4e-6


def test_batch_rejects_tensor_tier_plans():
    p = q.Plan(14, -1, q.FORWARD, "c64", 0, precision=q.PREC_FP16X3)
    x = torch.zeros(1 << 14, dtype=torch.complex64, device="cuda")
    with pytest.raises(q.QftError):
        q.Batch([p], [x], q.SCALE_STATE)


def test_batch_double_float_per_transform_range():
    """A complex128 (double-float) batch whose transforms differ by up to 2^1000
    in magnitude: each transform gets its own exponent shift, so every result
    equals the transform run alone."""
    specs, plans, xs = make_batch(40, 3, 16, "c128", 0, seed=19)
    rng = np.random.default_rng(19)
    xs = [x * (2.0 ** int(rng.integers(-500, 501))) for x in xs]
    states = [x.clone() for x in xs]
    b = q.Batch([plans[(n, k)] for n, k, _ in specs], states, q.SCALE_STATE)
    b.execute()
    assert b.status() == 0
    for i, (n, k, _) in enumerate(specs):
        p = plans[(n, k)]
        ref = xs[i].clone()
        p.execute(ref, p.alloc_workspace(), q.SCALE_STATE)
        torch.cuda.synchronize()
        assert rel(states[i], ref) <= 1e-13 * n, (i, n, k)


def test_batch_rejects_mixed_complex128_arithmetic():
    a = q.Plan(10, -1, q.FORWARD, "c128")
    f = q.Plan(10, -1, q.FORWARD, "c128", precision=q.PREC_FP64)
    xs = [torch.zeros(1 << 10, dtype=torch.complex128, device="cuda") for _ in range(2)]
    with pytest.raises(q.QftError):
        q.Batch([a, f], xs, q.SCALE_STATE)


def test_batch_bounded_wait_reports_timeout():
    """Tile loads that never arrive (a planner test hook leaves each CTA's first
    load unissued) make the batch kernel's bounded waits expire: it reports
    QFT_ERR_TIMEOUT in its status word, and the context stays usable."""
    plans = [q.Plan(n, -1, q.FORWARD, "c64", 0, test_skip_first_load=1, wait_limit_ms=20) for n in (14, 16, 17)]
    states = [torch.zeros(1 << p.info().n, dtype=torch.complex64, device="cuda") for p in plans]
    b = q.Batch(plans, states, q.SCALE_STATE)
    b.execute()
    torch.cuda.synchronize()
    assert b.status() == q.ERR_TIMEOUT
    specs, good, xs = make_batch(8, 8, 14, "c64", 0, seed=5)
    st = [x.clone() for x in xs]
    q.Batch([good[(n, k)] for n, k, _ in specs], st, q.SCALE_STATE).execute()
    torch.cuda.synchronize()
    for s_, x in zip(st, xs):
        assert torch.isfinite(torch.view_as_real(s_)).all()
        assert abs(float(torch.linalg.vector_norm(s_)) - 1.0) < 1e-5


# ---------------------------------------------------------------- wide groups
# Complex64 natural-order transforms of 14..20 qubits run on the 2^14-tile pass
# kernel in group mode (one launch per pass per (n, direction), the cutoff k
# per transform).

@pytest.mark.parametrize("direction,mode", [(q.FORWARD, q.SCALE_STATE), (q.INVERSE, q.SCALE_UNITARY),
                                            (q.FORWARD, q.SCALE_UNNORM)])
def test_wide_groups_match_single_transforms_and_oracle(oracle_mod, direction, mode):
    specs, plans, xs = make_batch(72, 10, 20, "c64", 0, seed=23, direction=direction)
    states = [x.clone() for x in xs]
    scales = torch.zeros(len(xs), dtype=torch.float64, device="cuda")
    b = q.Batch([plans[(n, k)] for n, k, _ in specs], states, mode, scale_out=scales)
    info = b.info()
    grouped = sum(1 for n, _, _ in specs if 14 <= n <= 20)
    assert info.wide_transforms == grouped > 0
    assert info.wide_groups == len({n for n, _, _ in specs if 14 <= n <= 20})  # one group per n: k is per transform
    assert info.kernel_launches == 2 * info.wide_groups + (1 if grouped < len(specs) else 0)
    b.execute()
    assert b.status() == 0
    for i, (n, k, _) in enumerate(specs):
        p = plans[(n, k)]
        ref = xs[i].clone()
        ws = p.alloc_workspace()
        p.execute(ref, ws, mode)
        torch.cuda.synchronize()
        assert rel(states[i], ref) <= TOL["c64"](n), (i, n, k)
        assert abs(scales[i].item() - p.scale_in(ws)) <= 1e-6 * max(p.scale_in(ws), 1e-300), (i, n)
    for i in [j for j, (n, _, _) in enumerate(specs) if n >= 14][:6]:
        n, k, _ = specs[i]
        want, _ = oracle_mod.qft(xs[i].cpu().numpy().astype(np.complex128), k, direction, mode, True)
        got = states[i].cpu().numpy().astype(np.complex128)
        assert np.linalg.norm(got - want) / np.linalg.norm(want) <= TOL["c64"](n), (i, n, k)


def test_wide_groups_elementwise_parity(oracle_mod):
    """Every amplitude of grouped transforms against the oracle within the
    element-wise bound of the wide plan's shape (2 passes, natural order)."""
    from parity import elementwise_bound, plan_shape

    ns = [14, 15, 17, 20, 14, 20]
    plans = {n: q.Plan(n, -1, q.FORWARD, "c64", 0) for n in set(ns)}
    xs = [torch.from_numpy(qft_inputs.gaussian(n, seed=40 + i)).to(torch.complex64).cuda() for i, n in enumerate(ns)]
    states = [x.clone() for x in xs]
    b = q.Batch([plans[n] for n in ns], states, q.SCALE_STATE)
    assert b.info().wide_transforms == len(ns)
    b.execute()
    assert b.status() == 0
    wide = {n: q.Plan(n, -1, q.FORWARD, "c64", 0, tile_bits=14) for n in set(ns)}
    for i, n in enumerate(ns):
        ref, _ = oracle_mod.qft(xs[i].cpu().numpy().astype(np.complex128), -1, -1, 0, True)
        a_last, natural = plan_shape(wide[n])
        bound = elementwise_bound(ref, "c64", n, a_last, natural)
        got = states[i].cpu().numpy().astype(np.complex128)
        assert np.max(np.abs(got - ref) / bound) <= 1.0, (i, n)


def test_wide_groups_are_deterministic():
    specs, plans, xs = make_batch(48, 12, 19, "c64", 0, seed=29)
    states = [x.clone() for x in xs]
    b = q.Batch([plans[(n, k)] for n, k, _ in specs], states, q.SCALE_STATE)
    assert b.info().wide_transforms > 0
    b.execute()
    torch.cuda.synchronize()
    first = [st.clone() for st in states]
    for st, x in zip(states, xs):
        st.copy_(x)
    b.execute()
    torch.cuda.synchronize()
    for st, f in zip(states, first):
        assert torch.equal(st, f)


def test_wide_groups_take_tile14_plans_in_range_only():
    xs = {n: torch.from_numpy(qft_inputs.gaussian(n, seed=n)).to(torch.complex64).cuda() for n in (16, 24)}
    p16 = q.Plan(16, 8, q.FORWARD, "c64", 0, tile_bits=14)
    st = xs[16].clone()
    b = q.Batch([p16], [st], q.SCALE_STATE)
    assert b.info().wide_transforms == 1 and b.info().persistent_items == 0
    b.execute()
    ref = xs[16].clone()
    p16.execute(ref, p16.alloc_workspace(), q.SCALE_STATE)
    torch.cuda.synchronize()
    assert rel(st, ref) <= 1e-6
    p24 = q.Plan(24, -1, q.FORWARD, "c64", 0)  # 2^14-amplitude tiles by default from n = 23
    assert p24.info().tile_bits[0] == 14
    with pytest.raises(q.QftError):
        q.Batch([p24], [xs[24].clone()], q.SCALE_STATE)


def test_wide_groups_bounded_wait_reports_timeout():
    """Group-mode passes whose first tile loads are never issued (the planner
    test hook on 2^14-tile plans) let their bounded waits expire: the batch
    status reads QFT_ERR_TIMEOUT and the next batch runs normally."""
    plans = [q.Plan(n, -1, q.FORWARD, "c64", 0, tile_bits=14, test_skip_first_load=1, wait_limit_ms=20)
             for n in (14, 16)]
    states = [torch.zeros(1 << p.info().n, dtype=torch.complex64, device="cuda") for p in plans]
    b = q.Batch(plans, states, q.SCALE_STATE)
    assert b.info().wide_transforms == 2
    b.execute()
    torch.cuda.synchronize()
    assert b.status() == q.ERR_TIMEOUT
    specs, good, xs = make_batch(8, 14, 17, "c64", 0, seed=6)
    st = [x.clone() for x in xs]
    b2 = q.Batch([good[(n, k)] for n, k, _ in specs], st, q.SCALE_STATE)
    b2.execute()
    assert b2.status() == 0
    for s_ in st:
        assert abs(float(torch.linalg.vector_norm(s_)) - 1.0) < 1e-5
