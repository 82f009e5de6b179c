"""GPU parity of the wide pass kernel (complex64, 2^14-amplitude tiles, two
register stages; csrc/qft_wide.cuh) against the CPU FP64 oracle, through the
C ABI.  Plans are made with tile_bits = 14 and checked to run on wide passes
only.  Sizes span several tiles per CTA and ragged passes (blocks of 3..5
wires with extra batch wires); the index maps (natural order) are exercised
by every comparison, and a basis-state input pins them bit for bit through
the argmax of a single-tone output."""
import numpy as np
import pytest

import qft_inputs
from test_gpu_parity import as_dt, assert_close, run

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
q = pytest.importorskip("paper_2606_18981_gb300")
from plan_emulator import parse  # noqa: E402


def wide_plan(n, k=-1, direction=-1):
    p = q.Plan(n, k, direction, "c64", q.ORDER_NATURAL, tile_bits=14)
    info = p.info()
    assert all(parse(p.describe_pass(i))["wide"] == 1 for i in range(info.passes)), "expected wide passes"
    assert info.passes == max(2, (n + 9) // 10)
    return p


@pytest.mark.parametrize("n", [14, 16, 17, 18, 19, 20, 24, 25])
def test_wide_matches_oracle(oracle_mod, n):
    x = as_dt(qft_inputs.gaussian(n, seed=100 + n, normalise=False), "c64")
    for direction in (q.FORWARD, q.INVERSE):
        got, s, sh = run(x, n, plan=wide_plan(n, -1, direction))
        ref, s_ref = oracle_mod.qft(x, -1, direction, 0, True)
        assert abs(s - s_ref) <= 1e-6 * s_ref
        assert_close(got, ref, "c64", n, sh)


@pytest.mark.parametrize("n", [17, 20])
def test_wide_aqft_cutoffs(oracle_mod, n):
    x = as_dt(qft_inputs.tones(n, seed=n), "c64")
    for k in (0, 1, 3, 4, 8, 12):
        for direction in (q.FORWARD, q.INVERSE):
            got, _, sh = run(x, n, plan=wide_plan(n, k, direction))
            ref, _ = oracle_mod.qft(x, k, direction, 0, True)
            assert_close(got, ref, "c64", n, sh)


def test_wide_scale_modes_against_numpy_fft():
    n = 18
    x = as_dt(qft_inputs.gaussian(n, seed=5, normalise=False), "c64")
    N = 1 << n
    F, G = np.fft.fft(x), np.fft.ifft(x)
    for direction, mode, ref in [(-1, q.SCALE_UNNORM, F), (-1, q.SCALE_UNITARY, F / np.sqrt(N)),
                                 (+1, q.SCALE_INV_N, G), (+1, q.SCALE_UNNORM, G * N),
                                 (-1, q.SCALE_STATE, F / (np.linalg.norm(x) * np.sqrt(N)))]:
        got, _, sh = run(x, n, mode=mode, plan=wide_plan(n, -1, direction))
        assert_close(got, ref, "c64", n, sh)


@pytest.mark.parametrize("n", [16, 24])
def test_wide_basis_and_tone_index_maps(n):
    """|j> -> uniform magnitude, exact phases; an on-bin tone -> its bin, argmax exact."""
    N = 1 << n
    rng = np.random.default_rng(n)
    for j in rng.integers(0, N, size=3):
        x = np.zeros(N, dtype=np.complex128)
        x[j] = 1.0
        got, _, sh = run(x, n, plan=wide_plan(n))
        y = np.arange(N, dtype=np.float64)
        ref = np.exp(-2j * np.pi * ((int(j) * y) % N) / N) / np.sqrt(N)
        assert_close(got, ref, "c64", n, sh)
    for k0 in rng.integers(0, N, size=3):
        x = np.exp(2j * np.pi * ((int(k0) * np.arange(N)) % N) / N)
        got, _, sh = run(x, n, plan=wide_plan(n))
        assert int(np.argmax(np.abs(got))) == int(k0)


def test_wide_large_round_trip_and_sampled_bins(oracle_mod):
    """n = 28 (3 passes of 10/9/9 wires): forward then inverse restores a
    Gaussian input; for an input of 2^16 nonzeros at random positions, 32
    output bins equal the oracle's DFT definition summed over the nonzeros,
    within the element-wise bound."""
    n = 28
    N = 1 << n
    pf, pi = wide_plan(n, -1, q.FORWARD), wide_plan(n, -1, q.INVERSE)
    ws = pf.alloc_workspace()
    rng = np.random.default_rng(3)
    idx = np.unique(rng.integers(0, N, size=1 << 16))
    vals = (rng.standard_normal(idx.size) + 1j * rng.standard_normal(idx.size)).astype(np.complex64)
    state = torch.zeros(N, dtype=torch.complex64, device="cuda")
    state[torch.from_numpy(idx).cuda()] = torch.from_numpy(vals).cuda()
    pf.execute(state, ws, q.SCALE_UNITARY)
    bins = rng.integers(0, N, size=32)
    got = state[torch.from_numpy(bins).to("cuda")].cpu().numpy().astype(np.complex128)
    ref = oracle_mod.dft_bins_sparse(idx, vals.astype(np.complex128), n, bins, q.FORWARD) / np.sqrt(N)
    rms = np.linalg.norm(vals.astype(np.complex128)) / np.sqrt(N)
    peak = float(state.abs().max().item())
    bound = 8 * 2.0 ** -24 * n * (np.abs(ref) + rms + peak / np.sqrt(2.0 ** 9))
    assert np.max(np.abs(got - ref) / bound) <= 1.0
    state = qft_inputs.device_gaussian(n, 7, "c64", device="cuda")
    x0 = state.clone()
    pf.execute(state, ws, q.SCALE_UNITARY)
    pi.execute(state, ws, q.SCALE_UNITARY)
    assert pf.status(ws) == 0
    err = (torch.linalg.vector_norm(state - x0) / torch.linalg.vector_norm(x0)).item()
    assert err <= 4e-6, err


def test_wide_timeout_reports_status():
    """A wide pass whose first tile load is never issued: the bounded wait
    expires and the status word reports QFT_ERR_TIMEOUT; the context stays usable."""
    n = 20
    p = q.Plan(n, -1, q.FORWARD, "c64", q.ORDER_NATURAL, tile_bits=14, wait_limit_ms=20, test_skip_first_load=1)
    state = torch.zeros(1 << n, dtype=torch.complex64, device="cuda")
    ws = p.alloc_workspace()
    p.execute(state, ws, q.SCALE_STATE)
    assert p.status(ws) == q.ERR_TIMEOUT
    good = wide_plan(n)
    ws2 = good.alloc_workspace()
    good.execute(state, ws2, q.SCALE_STATE)
    assert good.status(ws2) == 0
