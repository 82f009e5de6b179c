"""GPU parity: the CUDA path (through the C ABI) against the CPU FP64 oracle.

Bounds (tests/parity.py, where they are derived): relative L2 error <= 2e-6
for complex64 and <= 1e-13 * n for complex128, and element by element
|got_i - ref_i| <= 8 eps log2 N (|ref_i| + RMS + max(||ref_col(i)||,
||ref||_inf) / 2^(a/2)), a = the wires of the plan's last pass -- a bound
that rounding meets and a single wrong bin does not
(test_planted_single_bin_error_is_caught).  Index maps (the qubit-reversal
permutation, the bit-reversed order, argmax bins) are compared bit-exactly.
"""
import numpy as np
import pytest

import qft_inputs
from parity import TOL, check_close, elementwise_bound, plan_shape, rel_l2  # noqa: F401

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
q = pytest.importorskip("paper_2606_18981_gb300")


def assert_close(got, ref, dt, n, shape=None):
    """Both bounds of tests/parity.py; shape = (last-pass wires, natural order)."""
    a_last, natural = shape if shape is not None else (None, True)
    msg = check_close(got, ref, dt, n, a_last, natural)
    assert msg is None, msg


def tdt(dt):
    return torch.complex64 if dt == "c64" else torch.complex128


def run(x, n, k=-1, direction=-1, dt="c64", order=0, mode=0, tile_bits=0, plan=None):
    """Load x, execute, read back: (output, scale_in, plan shape for assert_close)."""
    p = plan or q.Plan(n, k, direction, dt, order, tile_bits=tile_bits)
    state = torch.empty(1 << n, dtype=tdt(dt), device="cuda")
    pinned = torch.from_numpy(np.ascontiguousarray(x)).to(tdt(dt)).pin_memory()
    p.load(state, pinned)
    ws = p.alloc_workspace()
    p.execute(state, ws, mode)
    out = state.cpu().numpy().astype(np.complex128)
    assert p.status(ws) == 0
    return out, p.scale_in(ws), plan_shape(p)


def as_dt(x, dt):
    return x.astype(np.complex64 if dt == "c64" else np.complex128).astype(np.complex128)


@pytest.mark.parametrize("dt", ["c64", "c128"])
@pytest.mark.parametrize("order", [0, 1])
@pytest.mark.parametrize("n", [1, 2, 3, 4, 5, 7, 8, 10, 12, 13])
def test_single_pass(oracle_mod, dt, order, n):
    x = as_dt(qft_inputs.gaussian(n, seed=n, normalise=False), dt)
    for direction in (-1, +1):
        got, s, sh = run(x, n, -1, direction, dt, order)
        ref, s_ref = oracle_mod.qft(x, -1, direction, 0, order == 0)
        assert abs(s - s_ref) <= 1e-6 * s_ref
        assert_close(got, ref, dt, n, sh)


@pytest.mark.parametrize("dt", ["c64", "c128"])
@pytest.mark.parametrize("order", [0, 1])
@pytest.mark.parametrize("n", [14, 16, 19, 20, 22])
def test_multi_pass(oracle_mod, dt, order, n):
    x = as_dt(qft_inputs.tones(n, seed=n), dt)
    for direction in (-1, +1):
        got, _, sh = run(x, n, -1, direction, dt, order)
        ref, _ = oracle_mod.qft(x, -1, direction, 0, order == 0)
        assert_close(got, ref, dt, n, sh)


@pytest.mark.parametrize("dt", ["c64", "c128"])
@pytest.mark.parametrize("n,tbits", [(12, 5), (13, 6), (15, 7), (16, 6), (11, 8), (14, 9), (9, 4)])
def test_small_tiles_many_passes(oracle_mod, dt, n, tbits):
    """Small tiles force 3..7 passes with ragged wire groups."""
    x = as_dt(qft_inputs.gaussian(n, seed=3 * n, normalise=False), dt)
    for order in (0, 1):
        for k in (-1, 1, 3):
            got, _, sh = run(x, n, k, -1, dt, order, tile_bits=tbits)
            ref, _ = oracle_mod.qft(x, k, -1, 0, order == 0)
            assert_close(got, ref, dt, n, sh)


@pytest.mark.parametrize("dt", ["c64", "c128"])
@pytest.mark.parametrize("n", [6, 13, 18, 21])
def test_aqft_cutoffs(oracle_mod, dt, n):
    x = as_dt(qft_inputs.gaussian(n, seed=7 + n, normalise=False), dt)
    for k in (0, 1, 2, 3, 4, 8, 16):
        if k >= n:
            continue
        for direction in (-1, +1):
            got, _, sh = run(x, n, k, direction, dt, 0)
            ref, _ = oracle_mod.qft(x, k, direction, 0, True)
            assert_close(got, ref, dt, n, sh)


@pytest.mark.parametrize("dt", ["c64", "c128"])
def test_scale_modes_against_numpy_fft(dt):
    for n in (9, 17):
        x = as_dt(qft_inputs.gaussian(n, seed=11, normalise=False), dt)
        N = 1 << n
        F = np.fft.fft(x)
        G = np.fft.ifft(x)
        cases = [(-1, q.SCALE_UNNORM, F), (-1, q.SCALE_UNITARY, F / np.sqrt(N)), (+1, q.SCALE_INV_N, G),
                 (+1, q.SCALE_UNNORM, G * N), (-1, q.SCALE_STATE, F / (np.linalg.norm(x) * np.sqrt(N)))]
        for direction, mode, ref in cases:
            got, s, sh = run(x, n, -1, direction, dt, 0, mode)
            assert abs(s - np.linalg.norm(x)) <= 1e-6 * np.linalg.norm(x)
            assert_close(got, ref, dt, n, sh)


@pytest.mark.parametrize("dt", ["c64", "c128"])
def test_zero_input(dt):
    for n in (5, 16):
        got, s, sh = run(np.zeros(1 << n, dtype=np.complex128), n, -1, -1, dt, 0)
        assert s == 0.0 and np.all(got == 0)


@pytest.mark.parametrize("dt", ["c64", "c128"])
@pytest.mark.parametrize("order", [0, 1])
@pytest.mark.parametrize("n,tbits", [(6, 0), (12, 0), (15, 0), (20, 0), (13, 7)])
def test_index_maps_bit_exact(dt, order, n, tbits):
    """k = 0 on small-integer input, unnormalised: every operation is exact, so the
    output must equal the integer Walsh-Hadamard transform permuted by the
    qubit reversal (NATURAL) or not (BITREV), bit for bit."""
    rng = np.random.default_rng(n)
    xi = rng.integers(-4, 5, size=1 << n) + 1j * rng.integers(-4, 5, size=1 << n)
    x = xi.astype(np.complex128)
    # fast integer WHT (Sylvester order), exact in int64
    w = xi.astype(np.complex128).copy()
    h = 1
    while h < w.size:
        w = w.reshape(-1, 2, h)
        w = np.stack([w[:, 0] + w[:, 1], w[:, 0] - w[:, 1]], axis=1).reshape(-1)
        h *= 2
    if order == 0:
        rev = np.array([int(format(i, f"0{n}b")[::-1], 2) for i in range(1 << n)])
        w = w[rev]
    got, _, sh = run(x, n, 0, -1, dt, order, q.SCALE_UNNORM, tile_bits=tbits)
    assert np.array_equal(got, w)


@pytest.mark.parametrize("dt", ["c64", "c128"])
def test_single_tone_peak_and_basis(dt):
    for n in (8, 14, 20):
        for direction in (-1, +1):
            x = qft_inputs.single_tone(n, 2, direction)
            got, s, sh = run(x, n, -1, direction, dt, 0)
            assert int(np.argmax(np.abs(got))) == 2
            assert abs(abs(got[2]) - 1) < 1e-5
            j = 5 + n
            got, _, sh = run(qft_inputs.basis(n, j), n, -1, direction, dt, 0)
            y = np.arange(1 << n, dtype=np.int64)
            ref = np.exp(direction * 2j * np.pi * ((j * y) % (1 << n)) / (1 << n)) / np.sqrt(1 << n)
            assert_close(got, ref, dt, n, sh)


def test_deterministic():
    for n in (11, 21):
        x = qft_inputs.gaussian(n, seed=5)
        a, _, _ = run(x, n, -1, -1, "c64", 0)
        b, _, _ = run(x, n, -1, -1, "c64", 0)
        assert np.array_equal(a, b)


@pytest.mark.parametrize("dt,k", [("c64", -1), ("c64", 4), ("c128", -1), ("c128", 8)])
def test_n24_full_oracle(oracle_mod, dt, k):
    n = 24
    x = as_dt(qft_inputs.gaussian(n, seed=24, normalise=True), dt)
    got, _, sh = run(x, n, k, -1, dt, 0)
    ref, _ = oracle_mod.qft(x, k, -1, 0, True)
    assert_close(got, ref, dt, n, sh)


def test_graph_capture_replay():
    n = 18
    p = q.Plan(n)
    x = torch.from_numpy(qft_inputs.gaussian(n, seed=1)).to(torch.complex64).cuda()
    state = x.clone()
    ws = p.alloc_workspace()
    s = torch.cuda.Stream()
    with torch.cuda.stream(s):
        p.execute(state, ws, q.SCALE_STATE, stream=s)  # warm-up encodes the tensor maps
    torch.cuda.synchronize()
    ref = state.clone()
    g = torch.cuda.CUDAGraph()
    with torch.cuda.graph(g, stream=s):
        p.execute(state, ws, q.SCALE_STATE, stream=s)
    for _ in range(2):
        state.copy_(x)
        g.replay()
        torch.cuda.synchronize()
        assert torch.equal(state, ref)


def test_bounded_wait_reports_timeout():
    """A tile load that never arrives makes the bounded mbarrier wait expire;
    the kernel reports QFT_ERR_TIMEOUT in the status word and the context stays usable."""
    p = q.Plan(18, test_skip_first_load=1, wait_limit_ms=20)
    state = torch.zeros(1 << 18, dtype=torch.complex64, device="cuda")
    ws = p.alloc_workspace()
    p.execute(state, ws, q.SCALE_STATE)
    assert p.status(ws) == q.ERR_TIMEOUT
    got, _, sh = run(qft_inputs.gaussian(10, seed=1), 10)  # context still usable
    assert np.isfinite(got).all()


def _bench_like(n, dt, seed):
    x = qft_inputs.device_gaussian(n, seed, dt)
    return x


def _column_stats(state, n, a_last, natural, chunk=1 << 27):
    """Peak magnitude and per-column norms (last-pass columns) of a device
    output, accumulated in chunks of rows so no full-size temporary is made."""
    rows, cols = (1 << a_last, 1 << (n - a_last)) if natural else (1 << (n - a_last), 1 << a_last)
    view = state.view(rows, cols)
    step = max(1, chunk // cols)
    peak = 0.0
    col = torch.zeros(cols if natural else rows, dtype=torch.float64, device=state.device)
    for r in range(0, rows, step):
        m2 = view[r:r + step].abs().to(torch.float64) ** 2
        peak = max(peak, float(m2.max().sqrt().item()))
        if natural:
            col += m2.sum(dim=0)
        else:
            col[r:r + step] = m2.sum(dim=1)
    return peak, col.sqrt()


def _bound_at(ys, ref, state, n, dt, shape, rms):
    """Element-wise bound (tests/parity.py) at sampled bins, with the output's
    peak and last-pass column norms taken from the device result."""
    a_last, natural = shape
    peak, col = _column_stats(state, n, a_last, natural)
    cidx = torch.from_numpy((ys % (1 << (n - a_last))) if natural else (ys >> a_last)).cuda()
    colv = col[cidx].cpu().numpy()
    eps = 2.0 ** -24 if dt == "c64" else 2.0 ** -46
    return 8 * eps * n * (np.abs(ref) + rms + np.maximum(colv, peak) / np.sqrt(2.0 ** a_last))


@pytest.mark.parametrize("n,dt", [(30, "c64"), (33, "c64"), (28, "c128")])
def test_large_sampled_bins(oracle_mod, n, dt):
    """The benchmark's exact plan (the same constructor call as bench.py) at
    full size.  Input: 2^16 Gaussian amplitudes at random positions, zero
    elsewhere, so the oracle's DFT definition summed over the nonzeros gives
    any output bin exactly and quickly; 64 bins, each within the element-wise
    bound at 1x, and the output norm."""
    free, _ = torch.cuda.mem_get_info()
    eb = 8 if dt == "c64" else 16
    if free < 2.2 * (1 << n) * eb + (4 << 30):
        pytest.skip("not enough device memory")
    N = 1 << n
    p = q.Plan(n, -1, q.FORWARD, dt, q.ORDER_NATURAL, tuned=True)
    rng = np.random.default_rng(n)
    idx = np.unique(rng.integers(0, N, size=1 << 16))
    vals = rng.standard_normal(idx.size) + 1j * rng.standard_normal(idx.size)
    state = torch.zeros(N, dtype=tdt(dt), device="cuda")
    state[torch.from_numpy(idx).cuda()] = torch.from_numpy(vals).to(tdt(dt)).cuda()
    vals = vals.astype(np.complex64 if dt == "c64" else np.complex128).astype(np.complex128)
    ws = p.alloc_workspace()
    p.execute(state, ws, q.SCALE_UNITARY)
    assert p.status(ws) == 0
    ys = np.unique(np.concatenate([[0, 1, 2, N - 1, N >> 1, int(idx[0])], rng.integers(0, N, size=80)]))[:64]
    got = state[torch.from_numpy(ys).cuda()].cpu().numpy().astype(np.complex128)
    ref = oracle_mod.dft_bins_sparse(idx, vals, n, ys, q.FORWARD) / np.sqrt(N)
    norm = float(np.linalg.norm(vals))
    bound = _bound_at(ys, ref, state, n, dt, plan_shape(p), norm / np.sqrt(N))
    ratio = np.abs(got - ref) / bound
    assert ratio.max() <= 1.0, (int(ys[np.argmax(ratio)]), float(ratio.max()))
    assert abs(_chunked_norm(state) - norm) <= TOL[dt](n) * norm
    del state, ws
    torch.cuda.empty_cache()


def test_large_sampled_bins_bench_input(oracle_mod):
    """n = 30 complex64 on the benchmark's plan and its own input (seeded
    Gaussian amplitudes drawn on the device): 8 output bins against the
    oracle's O(N) direct sums of the closed-form matrix elements, each within
    the element-wise bound at 1x."""
    n, dt = 30, "c64"
    N = 1 << n
    p = q.Plan(n, -1, q.FORWARD, dt, q.ORDER_NATURAL, tuned=True)
    x = _bench_like(n, dt, 2024)
    xh = x.cpu().numpy().astype(np.complex128)
    ws = p.alloc_workspace()
    p.execute(x, ws, q.SCALE_UNITARY)
    assert p.status(ws) == 0
    ys = np.concatenate([[0, 1, N - 1], np.random.default_rng(30).integers(0, N, size=5)])
    got = x[torch.from_numpy(ys).cuda()].cpu().numpy().astype(np.complex128)
    ref = oracle_mod.aqft_bins(xh, ys, -1, q.FORWARD)
    bound = _bound_at(ys, ref, x, n, dt, plan_shape(p), float(np.linalg.norm(xh)) / np.sqrt(N))
    assert np.max(np.abs(got - ref) / bound) <= 1.0
    del x, ws
    torch.cuda.empty_cache()


@pytest.mark.parametrize("kind", ["gaussian", "tones"])
def test_planted_single_bin_error_is_caught(oracle_mod, kind):
    """n = 24 on the default plan: the GPU output passes both bounds, and the
    same output with one bin moved by 1e-6 ||x|| (at an ordinary bin, and at a
    small bin in the last-pass column of the largest peak) fails the
    element-wise bound although it still meets the L2 target."""
    n = 24
    x = as_dt(qft_inputs.make(kind, n, seed=24), "c64")
    got, _, sh = run(x, n, -1, q.FORWARD, "c64", 0)
    ref, _ = oracle_mod.qft(x, -1, q.FORWARD, q.SCALE_STATE, True)
    assert check_close(got, ref, "c64", n, *sh) is None
    a_last = sh[0]
    rng = np.random.default_rng(5)
    small = np.flatnonzero(np.abs(ref) <= 2.0 / np.sqrt(ref.size))
    peak = int(np.argmax(np.abs(ref)))
    m = 1 << (n - a_last)
    in_col = small[(small % m) == (peak % m)]
    for i in [int(rng.choice(small))] + ([int(in_col[0])] if in_col.size else []):
        bad = got.copy()
        bad[i] += 1e-6 * np.exp(1j * rng.uniform(0, 2 * np.pi))
        assert rel_l2(bad, ref) <= TOL["c64"](n)
        assert check_close(bad, ref, "c64", n, *sh) is not None, i


def _chunked_norm(a, b=None, scale_b=1.0, chunk=1 << 26):
    """||a - scale_b * b|| (or ||a||) in float64 without materialising full-size temporaries."""
    acc = 0.0
    for s in range(0, a.numel(), chunk):
        d = a[s:s + chunk].to(torch.complex128)
        if b is not None:
            d = d - b[s:s + chunk].to(torch.complex128) * scale_b
        acc += float(torch.sum(d.real ** 2 + d.imag ** 2).item())
    return acc ** 0.5


@pytest.mark.parametrize("n,dt", [(33, "c64"), (32, "c128")])
def test_max_size_round_trip(n, dt):
    """Largest sizes (64 GiB states): forward then inverse returns the normalised
    input; the forward result keeps unit norm."""
    free, _ = torch.cuda.mem_get_info()
    need = 3 * (1 << n) * (8 if dt == "c64" else 16) + (4 << 30)
    if free < need:
        pytest.skip(f"needs {need / 2**30:.0f} GiB free")
    x = _bench_like(n, dt, 7)
    pf = q.Plan(n, -1, -1, dt, 0)
    pi = q.Plan(n, -1, +1, dt, 0)
    ws = pf.alloc_workspace()
    state = x.clone()
    pf.execute(state, ws, q.SCALE_STATE)
    assert pf.status(ws) == 0
    assert abs(_chunked_norm(state) - 1.0) < 1e-5
    pi.execute(state, ws, q.SCALE_STATE)
    assert pi.status(ws) == 0
    x_norm = _chunked_norm(x)
    assert _chunked_norm(state, x, 1.0 / x_norm) <= 2 * TOL[dt](n)
    del state, x, ws
    torch.cuda.empty_cache()


# Kernel variants the planner selects from its options: two CTAs per SM
# (complex64 tiles of <= 2^12 amplitudes), the wide pass kernel (2^14-amplitude tiles),
# both together, and small tiles.  Every variant must match the oracle.
VARIANTS = {
    "two_ctas": dict(tile_bits=12),
    "two_ctas_c3": dict(tile_bits=12, coalesce_bits=3),
    "tile11": dict(tile_bits=11),
    "wide": dict(tile_bits=14),
    "t512_blocks3": dict(tile_bits=12, coalesce_bits=4, threads=512, max_stage_bits=3),
    "split_middle": dict(tile_bits=12, coalesce_bits=4, pass_split=1),
}


@pytest.mark.parametrize("variant", sorted(VARIANTS))
@pytest.mark.parametrize("order", [0, 1])
@pytest.mark.parametrize("direction", [-1, 1])
@pytest.mark.parametrize("n,k", [(14, -1), (17, 5), (20, -1), (23, 9)])
def test_kernel_variants(oracle_mod, variant, order, direction, n, k):
    if variant == "wide" and order == q.ORDER_BITREV:
        pytest.skip("the wide pass kernel runs natural-order plans")
    x = qft_inputs.make(qft_inputs.KINDS[(n + direction) % 3], n, seed=n * 7 + order)
    p = q.Plan(n, k, direction, "c64", order, **VARIANTS[variant])
    got, s_in, sh = run(x, n, k, direction, "c64", order, plan=p)
    ref, s_ref = oracle_mod.qft(as_dt(x, "c64"), k, direction, 0, order == 0)
    assert_close(got, ref, "c64", n, sh)
    assert abs(s_in - s_ref) <= 1e-6 * s_ref

