"""Pins for the oracle's Monte Carlo backend (Sec. 6: sum-over-histories
estimates of single output bins with importance-weighted input indices).

The estimator's defining properties fix it without reference to its own code:
exact single-path cases (a basis state, a tone on its own bin: every sample
carries the whole amplitude), unbiasedness of the mean and of the power
estimate (averaged over many independent runs, within a few standard errors
of the exact bins from the DFT definition / closed-form AQFT elements), the
variance of the mean (E|z|^2 - |mean|^2) / M with E|z|^2 known exactly, and
the sampling law (a fine grid of uniforms lands on index j in proportion to
its integer weight q_j, i.e. to max(|Re x_j|, |Im x_j|))."""
import numpy as np
import pytest

import qft_inputs


def _uniforms(rng, m):
    return rng.integers(0, 2 ** 53, size=m, dtype=np.int64).astype(np.float64) / 2.0 ** 53


def _mag(x):
    """The proposal's magnitude of each term: max(|Re x_j|, |Im x_j|)."""
    x = np.asarray(x, dtype=np.complex128)
    return np.maximum(np.abs(x.real), np.abs(x.imag))


def _q(x, n):
    """The proposal's integer weights as the reading defines them: floor(m_j
    2^S / 2^(E+1)) + 1 for m_j > 0, S = min(62 - n, 52), 2^E <= max m < 2^(E+1)
    (formed here with exact float scaling by powers of two)."""
    a = _mag(x)
    S = min(62 - n, 52)
    E = np.frexp(a.max())[1] - 1
    return np.where(a > 0, np.floor(np.ldexp(a, S - E - 1)) + 1, 0).astype(np.uint64)


@pytest.mark.parametrize("sign", [-1, 1])
def test_tone_on_its_bin_is_exact(oracle_mod, sign):
    """A tone at bin N/4 (x_j = i^j, every term of the same magnitude and
    max(|Re|, |Im|)): the proposal is uniform, every path reaches bin N/4 with
    the same phase, so every sample carries the whole amplitude."""
    n = 10
    N = 1 << n
    k0 = N // 4
    x = np.exp(-sign * 2j * np.pi * k0 * np.arange(N) / N)
    idx, w, T = oracle_mod.mc_sample(x, _uniforms(np.random.default_rng(3), 500))
    amp, power, se = oracle_mod.mc_bins(idx, w, n, [k0], -1, sign)
    assert abs(amp[0] - np.sqrt(N)) <= 1e-9 * np.sqrt(N)
    assert abs(power[0] - N) <= 1e-9 * N and se[0] <= 1e-9 * np.sqrt(N)


@pytest.mark.parametrize("k", [-1, 2])
def test_basis_state_is_exact(oracle_mod, k):
    n, j0 = 9, 301
    N = 1 << n
    x = np.zeros(N, complex)
    x[j0] = 0.6 - 0.8j
    ys = np.arange(0, N, 7)
    idx, w, T = oracle_mod.mc_sample(x, _uniforms(np.random.default_rng(4), 64))
    assert np.all(idx == j0)
    amp, power, se = oracle_mod.mc_bins(idx, w, n, ys, k, -1)
    ref = oracle_mod.aqft_bins(x, ys, k, -1)
    assert np.max(np.abs(amp - ref)) <= 1e-12
    # the standard error is the square root of a rounding-level difference
    assert np.max(np.abs(power - np.abs(ref) ** 2)) <= 1e-12 and np.max(se) <= 1e-6 * np.max(np.abs(ref))


def test_zero_input(oracle_mod):
    idx, w, T = oracle_mod.mc_sample(np.zeros(64, complex), [0.5, 0.25])
    assert T == 0 and np.all(w == 0)
    amp, power, se = oracle_mod.mc_bins(idx, w, 6, [0, 5])
    assert np.all(amp == 0) and np.all(power == 0)


def test_sampling_law_on_a_fine_grid(oracle_mod):
    """Uniforms i / K (K = 2^16) land on index j about K q_j / T times (within
    one, since each index owns a contiguous run of targets)."""
    n = 5
    x = qft_inputs.gaussian(n, seed=11, normalise=False)
    x[3] = 0  # a zero amplitude is never drawn
    K = 1 << 16
    idx, w, T = oracle_mod.mc_sample(x, np.arange(K) / K)
    q = _q(x, n)
    assert T == int(q.sum())
    counts = np.bincount(idx, minlength=1 << n)
    assert counts[3] == 0
    assert np.all(np.abs(counts - K * q.astype(np.float64) / float(T)) <= 1.0)
    # weights: x_j T / q_j, i.e. x_j / p_j
    j = idx[K // 3]
    assert np.isclose(w[K // 3], x[j] * float(T) / float(q[j]), rtol=1e-15)


@pytest.mark.parametrize("k", [-1, 3])
def test_unbiased_mean_and_power_and_variance(oracle_mod, k):
    """Gaussian input, n = 8: over R = 400 independent runs of M = 64 samples
    the average estimate of each bin is within 5 standard errors of the exact
    bin (closed-form AQFT elements, which the oracle's pins tie to the DFT
    definition), the average power estimate within 5 standard errors of
    |bin|^2, and the spread of the estimates matches (E|z|^2 - |bin|^2) / M."""
    n, R, M = 8, 400, 64
    N = 1 << n
    x = qft_inputs.gaussian(n, seed=8, normalise=False)
    ys = np.array([0, 1, 17, 128, 200, 255])
    ref = oracle_mod.aqft_bins(x, ys, k, -1)
    q = _q(x, n).astype(np.float64)
    T = q.sum()
    Ez2 = np.sum(np.abs(x) ** 2 * T / q) / N  # E|z|^2 = sum_j p_j |x_j / p_j|^2 / N, the same for every bin
    var = (Ez2 - np.abs(ref) ** 2) / M
    rng = np.random.default_rng(2024)
    amps, pows = [], []
    for _ in range(R):
        idx, w, _T = oracle_mod.mc_sample(x, _uniforms(rng, M))
        a, p, _ = oracle_mod.mc_bins(idx, w, n, ys, k, -1)
        amps.append(a)
        pows.append(p)
    amps, pows = np.array(amps), np.array(pows)
    assert np.all(np.abs(amps.mean(0) - ref) <= 5 * np.sqrt(var / R))
    pstd = pows.std(0, ddof=1)
    assert np.all(np.abs(pows.mean(0) - np.abs(ref) ** 2) <= 5 * pstd / np.sqrt(R))
    emp = np.mean(np.abs(amps - ref) ** 2, axis=0)
    assert np.all((emp > 0.75 * var) & (emp < 1.33 * var))


# ------------------------------------------------- sparse inputs, n up to 62

def test_sparse_bins_equal_dense_and_definition(oracle_mod):
    """The sparse closed-form bins equal the dense ones on the scattered input
    (every cutoff), and at n = 50 the exact ones equal the DFT definition
    summed over the nonzeros with integer phases (an independent formula)."""
    n = 9
    rng = np.random.default_rng(9)
    pos = np.unique(rng.integers(0, 1 << n, size=40))
    vals = rng.standard_normal(pos.size) + 1j * rng.standard_normal(pos.size)
    x = np.zeros(1 << n, complex)
    x[pos] = vals
    ys = np.arange(0, 1 << n, 5)
    for k in (-1, 0, 2, 5):
        assert np.max(np.abs(oracle_mod.aqft_bins_sparse(pos, vals, n, ys, k, -1) -
                             oracle_mod.aqft_bins(x, ys, k, -1))) <= 1e-12
    n = 50
    pos = np.unique(rng.integers(0, 1 << n, size=300, dtype=np.int64))
    vals = rng.standard_normal(pos.size) + 1j * rng.standard_normal(pos.size)
    ys = rng.integers(0, 1 << n, size=20, dtype=np.int64)
    got = oracle_mod.aqft_bins_sparse(pos, vals, n, ys, -1, 1)
    ref = oracle_mod.dft_bins_sparse(pos, vals, n, ys, 1) / np.sqrt(2.0 ** n)
    assert np.max(np.abs(got - ref)) <= 1e-9 * np.max(np.abs(ref))


def test_sparse_single_entry_is_exact(oracle_mod):
    n = 48
    j0 = (1 << 47) + 123456789
    idx, w, T = oracle_mod.mc_sample_sparse([j0], [0.3 - 0.4j], _uniforms(np.random.default_rng(1), 50))
    assert np.all(idx == j0)
    ys = np.array([0, 1, 12345, (1 << 48) - 1])
    amp, power, se = oracle_mod.mc_bins(idx, w, n, ys, 7, -1)
    ref = oracle_mod.aqft_bins_sparse([j0], [0.3 - 0.4j], n, ys, 7, -1)
    assert np.max(np.abs(amp - ref)) <= 1e-12 * 2.0 ** -24


def test_sparse_draw_law_and_unbiased(oracle_mod):
    """n = 40, 64 nonzeros: uniforms on a grid land on entry j in proportion to
    q_j (S from ceil(log2 K)); over 300 runs of 32 samples the estimates of the
    exact and the range-5 bins are unbiased within 5 standard errors."""
    n, K = 40, 64
    rng = np.random.default_rng(40)
    pos = np.unique(rng.integers(0, 1 << n, size=K, dtype=np.int64))
    vals = qft_inputs.gaussian(6, seed=6, normalise=False)[:pos.size]
    G = 1 << 14
    idx, w, T = oracle_mod.mc_sample_sparse(pos, vals, np.arange(G) / G)
    qi = _q(vals, 6)
    assert T == int(qi.sum())
    q = qi.astype(np.float64)
    where = {int(p): i for i, p in enumerate(pos)}
    counts = np.bincount([where[int(j)] for j in idx], minlength=pos.size)
    assert np.all(np.abs(counts - G * q / q.sum()) <= 1.0)
    ys = np.concatenate([[0, 1], rng.integers(0, 1 << n, size=4, dtype=np.int64)])
    for k in (-1, 5):
        ref = oracle_mod.aqft_bins_sparse(pos, vals, n, ys, k, -1)
        amps = []
        for _ in range(300):
            i2, w2, _ = oracle_mod.mc_sample_sparse(pos, vals, _uniforms(rng, 32))
            amps.append(oracle_mod.mc_bins(i2, w2, n, ys, k, -1)[0])
        amps = np.array(amps)
        assert np.all(np.abs(amps.mean(0) - ref) <= 5 * amps.std(0) / np.sqrt(300))
