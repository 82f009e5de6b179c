"""The Monte Carlo backend (Sec. 6, sum over histories) on the GPU against the
oracle: the draws and weights bit for bit for the same uniforms (integer and
correctly rounded FP64 arithmetic on both sides), the per-bin estimates within
the FP32 evaluation's rounding of the oracle's FP64 ones, the exact
single-path cases, and at full size (n = 30, an input with 2^16 nonzeros) the
estimates within five standard errors of the exact bins of the DFT
definition summed over the nonzeros."""
import numpy as np
import pytest

import qft_inputs

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
q = pytest.importorskip("paper_2606_18981_gb300")


def _uniforms(seed, m):
    rng = np.random.default_rng(seed)
    return rng.integers(0, 2 ** 53, size=m, dtype=np.int64).astype(np.float64) / 2.0 ** 53


def _input(kind, n, seed):
    if kind == "tiny":  # magnitudes down to FP32 subnormals and exact zeros
        rng = np.random.default_rng(seed)
        x = (rng.standard_normal(1 << n) + 1j * rng.standard_normal(1 << n)) * 10.0 ** rng.uniform(-44, -30, 1 << n)
        x[rng.integers(0, 1 << n, size=(1 << n) // 8)] = 0
        return x
    if kind == "sparse":  # a few nonzeros, many exact zeros (never drawn)
        rng = np.random.default_rng(seed)
        x = np.zeros(1 << n, complex)
        pos = rng.integers(0, 1 << n, size=max(1, (1 << n) // 16))
        x[pos] = rng.standard_normal(pos.size) + 1j * rng.standard_normal(pos.size)
        return x
    return qft_inputs.make(kind, n, seed)


@pytest.mark.parametrize("dt", ["c64", "c128"])
@pytest.mark.parametrize("n,kind", [(5, "gaussian"), (12, "tones"), (13, "sparse"), (14, "tiny"), (17, "gaussian"),
                                    (20, "sparse")])
def test_draws_and_weights_bitwise(oracle_mod, dt, n, kind):
    td = torch.complex64 if dt == "c64" else torch.complex128
    x = torch.from_numpy(_input(kind, n, 40 + n)).to(td)
    xd = x.cuda()
    u = _uniforms(n, 5000)
    mc = q.MonteCarlo(xd)
    idx, w = mc.sample(torch.from_numpy(u).cuda())
    ridx, rw, T = oracle_mod.mc_sample(x.numpy().astype(np.complex128), u)
    assert np.array_equal(idx.cpu().numpy(), ridx)
    assert np.array_equal(w.cpu().numpy(), rw)


@pytest.mark.parametrize("k,direction", [(-1, -1), (-1, 1), (4, -1), (0, 1)])
def test_bins_match_oracle(oracle_mod, k, direction):
    n, M = 12, 4096
    N = 1 << n
    x = _input("gaussian", n, 7)
    xd = torch.from_numpy(x).cuda()
    u = _uniforms(99, M)
    mc = q.MonteCarlo(xd)
    idx, w = mc.sample(torch.from_numpy(u).cuda())
    ys = np.array(sorted(set([0, 1, N - 1, N // 2] + list(np.random.default_rng(5).integers(0, N, 60)))))
    amp, power, se = (t.cpu().numpy() for t in mc.bins(idx, w, ys, k, direction))
    ridx, rw, _ = oracle_mod.mc_sample(x, u)
    ramp, rpower, rse = oracle_mod.mc_bins(ridx, rw, n, ys, k, direction)
    # FP32 phase and products, FP32 runs of 32 terms: a few units of 2^-24 per term
    scale = np.mean(np.abs(rw)) / np.sqrt(N)
    assert np.max(np.abs(amp - ramp)) <= 64 * 2.0 ** -24 * scale
    assert np.max(np.abs(power - rpower)) <= 4 * np.max(np.abs(ramp)) * 64 * 2.0 ** -24 * scale + 1e-9 * scale ** 2
    assert np.max(np.abs(se - rse)) <= 1e-3 * np.max(rse) + 64 * 2.0 ** -24 * scale


def test_exact_single_path_cases(oracle_mod):
    n = 14
    N = 1 << n
    tone = torch.from_numpy(1j ** np.arange(N)).to(torch.complex64).cuda()  # bin N/4, uniform proposal
    mc = q.MonteCarlo(tone)
    idx, w = mc.sample(torch.from_numpy(_uniforms(1, 1000)).cuda())
    amp, power, se = mc.bins(idx, w, [N // 4, 3], -1, q.FORWARD)
    assert abs(amp[0].item() - np.sqrt(N)) <= 1e-5 * np.sqrt(N)
    assert se[0].item() <= 1e-3 * np.sqrt(N)
    basis = torch.zeros(N, dtype=torch.complex128, device="cuda")
    basis[1234] = 0.6 + 0.8j
    mc = q.MonteCarlo(basis)
    idx, w = mc.sample(torch.from_numpy(_uniforms(2, 100)).cuda())
    assert torch.all(idx == 1234)
    ys = np.arange(0, N, 97)
    amp, power, se = mc.bins(idx, w, ys, 5, q.FORWARD)
    ref = oracle_mod.aqft_bins(basis.cpu().numpy(), ys, 5, q.FORWARD)
    assert np.max(np.abs(amp.cpu().numpy() - ref)) <= 1e-6 / np.sqrt(N)


def test_zero_input_and_argument_checks():
    n = 10
    mc = q.MonteCarlo(torch.zeros(1 << n, dtype=torch.complex64, device="cuda"))
    idx, w = mc.sample(torch.rand(64, dtype=torch.float64, device="cuda"))
    assert torch.all(idx == 0) and torch.all(w == 0)
    amp, power, se = mc.bins(idx, w, [0, 5])
    assert torch.all(amp == 0) and torch.all(power == 0)
    with pytest.raises(q.QftError):
        mc.bins(idx, w, list(range(70000)))  # more than 65536 bins


def test_full_size_sparse_input_within_standard_errors(oracle_mod):
    """n = 30 complex64, 2^16 Gaussian amplitudes at random positions: 2^20
    samples, 64 bins; every estimate within 5 standard errors of the exact bin
    (the DFT definition over the nonzeros), every draw on a nonzero."""
    n = 30
    N = 1 << n
    free, _ = torch.cuda.mem_get_info()
    if free < 3 * N * 8 + (4 << 30):
        pytest.skip("not enough device memory")
    rng = np.random.default_rng(30)
    pos = np.unique(rng.integers(0, N, size=1 << 16))
    vals = (rng.standard_normal(pos.size) + 1j * rng.standard_normal(pos.size)).astype(np.complex64)
    x = torch.zeros(N, dtype=torch.complex64, device="cuda")
    x[torch.from_numpy(pos).cuda()] = torch.from_numpy(vals).cuda()
    mc = q.MonteCarlo(x)
    M = 1 << 20
    gen = torch.Generator(device="cuda").manual_seed(30)
    u = torch.rand(M, dtype=torch.float64, device="cuda", generator=gen)
    idx, w = mc.sample(u)
    drawn = np.unique(idx.cpu().numpy())
    assert np.all(np.isin(drawn, pos))
    ys = np.unique(np.concatenate([[0, 1, N - 1], rng.integers(0, N, size=70)]))[:64]
    amp, power, se = (t.cpu().numpy() for t in mc.bins(idx, w, ys, -1, q.FORWARD))
    ref = oracle_mod.dft_bins_sparse(pos, vals.astype(np.complex128), n, ys, q.FORWARD) / np.sqrt(N)
    assert np.all(se > 0)
    assert np.max(np.abs(amp - ref) / se) <= 5.0
    del x, mc, idx, w, u
    torch.cuda.empty_cache()


# ---------------------------------------------- sparse inputs, beyond a state vector

def _sparse(n, K, seed):
    rng = np.random.default_rng(seed)
    pos = np.unique(rng.integers(0, 1 << n, size=K, dtype=np.int64))
    vals = rng.standard_normal(pos.size) + 1j * rng.standard_normal(pos.size)
    return pos, vals


@pytest.mark.parametrize("dt", ["c64", "c128"])
@pytest.mark.parametrize("n,K", [(50, 1), (50, 3000), (62, 70000)])
def test_sparse_draws_and_weights_bitwise(oracle_mod, dt, n, K):
    td = torch.complex64 if dt == "c64" else torch.complex128
    pos, vals = _sparse(n, K, n + K)
    v = torch.from_numpy(vals).to(td)
    u = _uniforms(K, 4000)
    mc = q.MonteCarlo(v.cuda(), pos=torch.from_numpy(pos).cuda(), n=n)
    idx, w = mc.sample(torch.from_numpy(u).cuda())
    ridx, rw, _ = oracle_mod.mc_sample_sparse(pos, v.numpy().astype(np.complex128), u)
    assert np.array_equal(idx.cpu().numpy(), ridx)
    assert np.array_equal(w.cpu().numpy(), rw)


@pytest.mark.parametrize("k", [-1, 6])
def test_sparse_bins_match_oracle_and_exact(oracle_mod, k):
    """n = 60 (2^60 amplitudes, far beyond a state vector), 512 nonzeros:
    2^16 samples; the GPU's estimates equal the oracle's for the same draws
    within the FP32 evaluation's rounding, and lie within 5 standard errors of
    the exact bins (closed-form elements summed over the nonzeros)."""
    n = 60
    pos, vals = _sparse(n, 512, 60)
    u = _uniforms(60, 1 << 16)
    mc = q.MonteCarlo(torch.from_numpy(vals).cuda(), pos=torch.from_numpy(pos).cuda(), n=n)
    idx, w = mc.sample(torch.from_numpy(u).cuda())
    rng = np.random.default_rng(61)
    ys = np.concatenate([[0, 1, (1 << 60) - 1], rng.integers(0, 1 << 60, size=61, dtype=np.int64)])
    amp, power, se = (t.cpu().numpy() for t in mc.bins(idx, w, ys, k, q.FORWARD))
    ridx, rw, _ = oracle_mod.mc_sample_sparse(pos, vals, u)
    ramp, _, _ = oracle_mod.mc_bins(ridx, rw, n, ys, k, q.FORWARD)
    scale = np.mean(np.abs(rw)) / 2.0 ** 30
    assert np.max(np.abs(amp - ramp)) <= 64 * 2.0 ** -24 * scale
    ref = oracle_mod.aqft_bins_sparse(pos, vals, n, ys, k, q.FORWARD)
    assert np.max(np.abs(amp - ref) / se) <= 5.0
