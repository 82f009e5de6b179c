"""complex128 on the GPU: the default double-float path and the IEEE FP64
path (QFT_PREC_FP64) against the CPU FP64 oracle, and the double-float
path's range normalisation over the whole FP64 exponent range.

The double-float kernel keeps amplitudes as pairs of FP32 numbers; before
its first pass a pre-pass finds the largest binary exponent of the input and
the input is scaled by that power of two.  The normalised state psi' (scale
mode STATE) does not depend on the input's scale, so an input multiplied by
2^e must give the oracle's psi' of the unscaled input, and scale_in must be
||x|| 2^e, for every e the FP64 range allows.
"""
import numpy as np
import pytest

import qft_inputs

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
q = pytest.importorskip("paper_2606_18981_gb300")


def tol(n):
    return 1e-13 * max(n, 1)


def rel_l2(a, b):
    return float(np.linalg.norm(a - b) / max(np.linalg.norm(b), 1e-300))


def run(x, n, k=-1, direction=-1, order=0, mode=0, precision=0, threads=0, **shape):
    p = q.Plan(n, k, direction, "c128", order, precision=precision, threads=threads, **shape)
    state = torch.empty(1 << n, dtype=torch.complex128, device="cuda")
    p.load(state, torch.from_numpy(np.ascontiguousarray(x)).pin_memory())
    ws = p.alloc_workspace()
    p.execute(state, ws, mode)
    out = state.cpu().numpy()
    assert p.status(ws) == 0
    return out, p.scale_in(ws)


@pytest.mark.parametrize("n", [3, 10, 12, 16, 22])
@pytest.mark.parametrize("precision", [0, 6])
def test_df_and_fp64_against_oracle(oracle_mod, n, precision):
    x = qft_inputs.gaussian(n, seed=100 + n, normalise=False)
    for direction in (-1, +1):
        for k in (-1, 3):
            got, s = run(x, n, k, direction, 0, 0, precision)
            ref, s_ref = oracle_mod.qft(x, k, direction, 0, True)
            assert rel_l2(got, ref) <= tol(n)
            assert np.max(np.abs(got - ref)) <= tol(n) * np.linalg.norm(ref)
            assert abs(s - s_ref) <= 1e-14 * s_ref


@pytest.mark.parametrize("e", [-1000, -600, -100, 0, 100, 600, 1000])
@pytest.mark.parametrize("n", [8, 18])
def test_df_range_normalisation(oracle_mod, n, e):
    x = qft_inputs.gaussian(n, seed=7, normalise=False)
    ref, s_ref = oracle_mod.qft(x, -1, -1, 0, True)
    xs = np.ldexp(x.real, e) + 1j * np.ldexp(x.imag, e)
    got, s = run(xs, n)
    assert rel_l2(got, ref) <= tol(n), (e, rel_l2(got, ref))
    assert abs(s / np.ldexp(s_ref, e) - 1.0) <= 1e-14


def test_df_unnormalised_output_scaled_input():
    """UNNORM output (numpy.fft.fft units) of inputs far from unit scale."""
    n = 14
    x = qft_inputs.gaussian(n, seed=3, normalise=False)
    for e in (-300, 300):
        xs = np.ldexp(x.real, e) + 1j * np.ldexp(x.imag, e)
        got, _ = run(xs, n, mode=q.SCALE_UNNORM)
        ref = np.fft.fft(xs)
        assert rel_l2(got, ref) <= tol(n)


def test_df_wide_dynamic_range(oracle_mod):
    """A basis state plus components 2^-40 and 2^-90 below it: what matters at
    the 2^-48 level of the largest component is kept."""
    n = 16
    rng = np.random.default_rng(5)
    x = np.zeros(1 << n, dtype=np.complex128)
    x[12345] = 1.0 - 0.5j
    idx = rng.integers(0, 1 << n, size=64)
    x[idx[:32]] += np.ldexp(rng.standard_normal(32), -40)
    x[idx[32:]] += 1j * np.ldexp(rng.standard_normal(32), -90)
    got, _ = run(x, n)
    ref, _ = oracle_mod.qft(x, -1, -1, 0, True)
    assert rel_l2(got, ref) <= tol(n)


def test_df_matches_fp64_path():
    """The two complex128 paths agree to the tolerance on a multi-pass transform."""
    n = 21
    x = qft_inputs.tones(n, seed=21)
    a, sa = run(x, n, precision=0)
    b, sb = run(x, n, precision=6)
    assert rel_l2(a, b) <= tol(n)
    assert abs(sa - sb) <= 1e-14 * sb


@pytest.mark.parametrize("n", [10, 15, 20, 23])
@pytest.mark.parametrize("order", [0, 1])
def test_df_512_threads(oracle_mod, n, order):
    """The 512-thread double-float kernel (blocks of <= 3 wires) against the oracle."""
    x = qft_inputs.tones(n, seed=400 + n)
    for direction, k in ((-1, -1), (+1, 5)):
        got, _ = run(x, n, k, direction, order, 0, 0, threads=512)
        ref, _ = oracle_mod.qft(x, k, direction, 0, order == 0)
        assert rel_l2(got, ref) <= tol(n)


@pytest.mark.parametrize("n", [9, 14, 19, 23])
@pytest.mark.parametrize("order", [0, 1])
def test_df_two_ctas_per_sm(oracle_mod, n, order):
    """The double-float kernel with two 256-thread CTAs per SM (2^11-pair
    tiles, blocks of <= 3 wires within 128 registers) against the oracle."""
    x = qft_inputs.tones(n, seed=450 + n)
    shape = dict(threads=256, tile_bits=11, max_stage_bits=3)
    p = q.Plan(n, -1, -1, "c128", order, **shape)
    from plan_emulator import parse
    assert all(parse(p.describe_pass(i))["minb"] == 2 for i in range(p.info().passes))
    for direction, k in ((-1, -1), (+1, 5)):
        for mode in (q.SCALE_STATE, q.SCALE_UNNORM):
            got, _ = run(x, n, k, direction, order, mode, 0, **shape)
            ref, _ = oracle_mod.qft(x, k, direction, mode, order == 0)
            assert rel_l2(got, ref) <= tol(n), (n, order, direction, mode)
