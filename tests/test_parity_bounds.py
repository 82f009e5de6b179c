"""CPU pins of the element-wise parity bound (tests/parity.py) itself.

The wide pass kernel's data flow replayed in complex64 arithmetic
(tests/wide_emulator.py, fp32=True) gives outputs with a realistic FP32
rounding profile.  For Gaussian, tone-mixture, single-tone and basis-state
inputs they must pass the bound (rounding is not flagged), and the same
outputs with one bin moved by 1e-6 * ||x|| must fail it -- at an ordinary
bin of a flat spectrum and at a small bin inside a spectral peak's
last-pass column, where the bound is loosest."""
import numpy as np
import pytest

import qft_inputs
from parity import check_close, elementwise_bound, plan_shape

q = pytest.importorskip("paper_2606_18981_gb300")
from test_wide_host import index_exe  # noqa: E402,F401  (fixture)
from wide_emulator import emulate_wide, thread_maps  # noqa: E402


def inputs(n):
    N = 1 << n
    basis = np.zeros(N, dtype=np.complex128)
    basis[(12345 * 7) % N] = 1.0
    return {"gaussian": qft_inputs.gaussian(n, seed=1, normalise=False),
            "tones": qft_inputs.tones(n, seed=2),
            "tone": np.exp(2j * np.pi * ((7 * np.arange(N)) % N) / N),
            "basis": basis}


@pytest.mark.parametrize("n", [16, 18])
def test_fp32_rounding_passes_and_planted_errors_fail(oracle_mod, index_exe, n):  # noqa: F811
    maps = thread_maps(index_exe)
    rng = np.random.default_rng(n)
    for kind, x in inputs(n).items():
        x = x.astype(np.complex64).astype(np.complex128)
        p = q.Plan(n, -1, q.FORWARD, "c64", q.ORDER_NATURAL, tile_bits=14)
        a_last, natural = plan_shape(p)
        got = emulate_wide(p, x, maps, q.SCALE_STATE, fp32=True)
        ref, _ = oracle_mod.qft(x, -1, q.FORWARD, q.SCALE_STATE, True)
        assert check_close(got, ref, "c64", n, a_last, natural) is None, kind
        bound = elementwise_bound(ref, "c64", n, a_last, natural)
        ratio = np.max(np.abs(got - ref) / bound)
        assert ratio <= 0.25, (kind, ratio)  # the bound's margin over FP32 rounding
        # one bin moved by 1e-6 * ||x|| (the state output has ||ref|| = 1)
        small = np.flatnonzero(np.abs(ref) <= np.sqrt(2.0 / ref.size))
        peak = int(np.argmax(np.abs(ref)))
        in_col = small[(small % (1 << (n - a_last))) == (peak % (1 << (n - a_last)))]
        for i in (int(rng.choice(small)), int(in_col[0]) if in_col.size else None):
            if i is None:
                continue
            bad = got.copy()
            bad[i] += 1e-6 * np.exp(1j * rng.uniform(0, 2 * np.pi))
            assert check_close(bad, ref, "c64", n, a_last, natural) is not None, (kind, i)


def test_bound_margins_at_n24():
    """The numbers quoted in tests/parity.py: at n = 24 (a last pass of 8
    wires), 1e-6 of a unit-norm output exceeds the bound by > 100x at a bin of
    a flat spectrum, and still exceeds it next to a peak that holds the whole
    norm (the loosest case)."""
    n, N = 24, 1 << 24
    flat = np.full(N, 1.0 / np.sqrt(N), dtype=np.complex128)
    assert 1e-6 / elementwise_bound(flat, "c64", n, 8, True)[5] > 100
    peak = np.zeros(N, dtype=np.complex128)
    peak[123] = 1.0
    b = elementwise_bound(peak, "c64", n, 8, True)
    assert 1e-6 / b[123 + (1 << 16)] > 1.3 and 1e-6 / b[124] > 1.3
