"""Pins for the CPU oracle: each check ties it to something other than itself.

Sources of truth: the DFT definition and its fast library form (numpy.fft),
the paper's worked examples (Eq. 3 DFT_8 factorisation, the T~ factors of
Sec. 2, Fig. 1 gate list), Table 2 gate counts, textbook special cases (k=0 is
a Walsh-Hadamard transform, basis states, single tones, the shift theorem),
and invariants (unitarity, round trip, symmetry, the AQFT error bound).
"""
import os

import numpy as np
import pytest

import qft_inputs

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


def rel_l2(a, b):
    a = np.asarray(a).ravel()
    b = np.asarray(b).ravel()
    den = np.linalg.norm(b)
    return float(np.linalg.norm(a - b) / (den if den > 0 else 1.0))


# ------------------------------------------------------------ exact QFT == DFT

@pytest.mark.parametrize("n", range(1, 11))
@pytest.mark.parametrize("sign", [-1, +1])
def test_exact_qft_equals_dft_definition(oracle_mod, n, sign):
    """Sec. 3 step 4: scale_in*sqrt(N)*psi' is the unnormalised DFT of x."""
    x = qft_inputs.gaussian(n, seed=100 + n, normalise=False)
    out, s = oracle_mod.qft(x, k=-1, sign=sign, mode=oracle_mod.SCALE_UNNORM)
    ref = oracle_mod.dft(x, sign)
    assert rel_l2(out, ref) < 1e-13 * max(n, 1)


@pytest.mark.parametrize("n", [1, 2, 3, 5, 8, 12, 14])
def test_exact_qft_equals_numpy_fft(oracle_mod, n):
    """Forward = numpy.fft.fft (same e^{-2 pi i/N} sign); inverse = N * numpy.fft.ifft."""
    x = qft_inputs.gaussian(n, seed=7 * n, normalise=False)
    fwd, _ = oracle_mod.qft(x, k=-1, sign=-1, mode=oracle_mod.SCALE_UNNORM)
    assert rel_l2(fwd, np.fft.fft(x)) < 1e-13 * n
    inv, _ = oracle_mod.qft(x, k=-1, sign=+1, mode=oracle_mod.SCALE_UNNORM)
    assert rel_l2(inv, np.fft.ifft(x) * (1 << n)) < 1e-13 * n


@pytest.mark.parametrize("n", [4, 9])
def test_decode_modes(oracle_mod, n):
    """Sec. 3 step 4: unitary = scale_in psi', unnormalised = scale_in sqrt(N) psi',
    1/N convention = scale_in psi'/sqrt(N); state mode has unit norm."""
    x = qft_inputs.gaussian(n, seed=3, normalise=False)
    N = 1 << n
    F = np.fft.fft(x)
    st, s = oracle_mod.qft(x, mode=oracle_mod.SCALE_STATE)
    assert abs(s - np.linalg.norm(x)) < 1e-12 * np.linalg.norm(x)
    assert abs(np.linalg.norm(st) - 1.0) < 1e-13
    assert rel_l2(st, F / (s * np.sqrt(N))) < 1e-13 * n
    un, _ = oracle_mod.qft(x, mode=oracle_mod.SCALE_UNITARY)
    assert rel_l2(un, F / np.sqrt(N)) < 1e-13 * n
    inv_n, _ = oracle_mod.qft(x, mode=oracle_mod.SCALE_INV_N)
    assert rel_l2(inv_n, F / N) < 1e-13 * n


# --------------------------------------------------------------- AQFT pins

@pytest.mark.parametrize("n", range(1, 9))
def test_aqft_circuit_equals_closed_form(oracle_mod, n):
    """Gate-by-gate range-k circuit == closed-form matrix elements, every k, both signs."""
    x = qft_inputs.gaussian(n, seed=200 + n)
    for k in range(0, n):
        for sign in (-1, +1):
            out = oracle_mod.circuit(x, k=k, sign=sign)
            ref = oracle_mod.aqft_direct(x, k=k, sign=sign)
            assert rel_l2(out, ref) < 1e-13 * n, (n, k, sign)


@pytest.mark.parametrize("n", [1, 3, 6, 9])
def test_k_ge_n_minus_1_is_exact(oracle_mod, n):
    """Sec. 2: no cutoff (k = n-1, or larger) is the exact QFT."""
    x = qft_inputs.gaussian(n, seed=11)
    ex = oracle_mod.circuit(x, k=-1)
    for k in (n - 1, n, n + 5):
        assert np.array_equal(oracle_mod.circuit(x, k=k), ex)


@pytest.mark.parametrize("n", [1, 2, 4, 7, 10])
def test_k0_is_walsh_hadamard_then_bit_reversal(oracle_mod, n):
    """k = 0 drops every controlled phase: H on all wires (Sylvester Hadamard
    matrix / sqrt(N)) followed by the qubit-reversal permutation."""
    from scipy.linalg import hadamard

    N = 1 << n
    x = qft_inputs.gaussian(n, seed=5)
    wht = hadamard(N).astype(np.float64) @ x / np.sqrt(N)
    rev = np.array([int(format(i, f"0{n}b")[::-1], 2) for i in range(N)])
    for sign in (-1, +1):
        out = oracle_mod.circuit(x, k=0, sign=sign)
        assert rel_l2(out, wht[rev]) < 1e-13 * n


@pytest.mark.parametrize("n", [3, 5, 7])
def test_aqft_error_bound(oracle_mod, n):
    """||U_k - U||_2 <= sum over dropped controlled-R_{d+1} of ||CP - I||_2
    = sum_{d=k+1}^{n-1} (n-d) * 2 sin(pi/2^{d+1}) (products of unitaries)."""
    N = 1 << n
    I = np.eye(N, dtype=np.complex128)
    U = np.stack([oracle_mod.circuit(I[:, j], k=-1) for j in range(N)], axis=1)
    for k in range(0, n):
        Uk = np.stack([oracle_mod.circuit(I[:, j], k=k) for j in range(N)], axis=1)
        err = np.linalg.norm(Uk - U, 2)
        bound = sum((n - d) * 2 * np.sin(np.pi / 2 ** (d + 1)) for d in range(k + 1, n))
        assert err <= bound + 1e-12
        if k == n - 1:
            assert err < 1e-13


@pytest.mark.parametrize("n", [2, 4, 6])
def test_aqft_matrix_symmetric_and_unitary(oracle_mod, n):
    """With the swaps, <y|U_k|x> depends on x and y symmetrically, so U_k = U_k^T
    and the inverse transform is the conjugate (sign-flipped) circuit."""
    N = 1 << n
    I = np.eye(N, dtype=np.complex128)
    for k in range(0, n):
        Uk = np.stack([oracle_mod.circuit(I[:, j], k=k) for j in range(N)], axis=1)
        assert np.allclose(Uk, Uk.T, atol=1e-14)
        assert np.allclose(Uk.conj().T @ Uk, I, atol=1e-13)
        Vk = np.stack([oracle_mod.circuit(I[:, j], k=k, sign=+1) for j in range(N)], axis=1)
        assert np.allclose(Vk, Uk.conj(), atol=1e-14)


# ---------------------------------------------------------- special inputs

@pytest.mark.parametrize("n", [1, 4, 10])
def test_basis_state(oracle_mod, n):
    """|j> -> uniform magnitude 1/sqrt(N), phases e^{s 2 pi i j y / N}."""
    N = 1 << n
    rng = np.random.default_rng(n)
    for j in [0, 1, N - 1, int(rng.integers(0, N))]:
        for sign in (-1, +1):
            out = oracle_mod.circuit(qft_inputs.basis(n, j), k=-1, sign=sign)
            y = np.arange(N, dtype=np.int64)
            ref = np.exp(sign * 2j * np.pi * ((j * y) % N) / N) / np.sqrt(N)
            assert rel_l2(out, ref) < 1e-13 * n


@pytest.mark.parametrize("n", [3, 8, 12])
def test_single_tone_peaks_at_k0(oracle_mod, n):
    """Sec. 4 correctness check: a unit-norm tone at bin k0=2 lands in bin 2 only."""
    for sign in (-1, +1):
        x = qft_inputs.single_tone(n, k0=2, sign=sign)
        out, s = oracle_mod.qft(x, k=-1, sign=sign)
        assert abs(s - 1.0) < 1e-12
        assert int(np.argmax(np.abs(out))) == 2
        assert abs(abs(out[2]) - 1.0) < 1e-12
        others = np.delete(out, 2)
        assert np.max(np.abs(others)) < 1e-12


@pytest.mark.parametrize("n", [5, 9])
def test_shift_theorem(oracle_mod, n):
    """Circular shift by r multiplies the exact transform by e^{-s 2 pi i r y / N}."""
    N = 1 << n
    x = qft_inputs.gaussian(n, seed=21)
    r = 3
    y = np.arange(N, dtype=np.int64)
    for sign in (-1, +1):
        a = oracle_mod.circuit(x, sign=sign)
        b = oracle_mod.circuit(np.roll(x, r), sign=sign)
        assert rel_l2(b, a * np.exp(sign * 2j * np.pi * ((r * y) % N) / N)) < 1e-12


def test_norm_linearity_roundtrip(oracle_mod):
    n = 9
    x = qft_inputs.gaussian(n, seed=1)
    z = qft_inputs.tones(n, seed=2)
    z = z / np.linalg.norm(z)
    for k in (0, 1, 3, 8):
        a = oracle_mod.circuit(x, k=k)
        b = oracle_mod.circuit(z, k=k)
        assert abs(np.linalg.norm(a) - 1.0) < 1e-13
        ab = oracle_mod.circuit(0.3 * x - 1.7j * z, k=k)
        assert rel_l2(ab, 0.3 * a - 1.7j * b) < 1e-13
        back = oracle_mod.circuit(a, k=k, sign=+1)
        assert rel_l2(back, x) < 1e-13 * n


def test_zero_input(oracle_mod):
    x = np.zeros(16, dtype=np.complex128)
    out, s = oracle_mod.qft(x)
    assert s == 0.0 and np.all(out == 0)


def test_bit_order_and_deferred_swaps(oracle_mod):
    """Sec. 3 step 2: leaving the swaps to the caller gives the output in
    bit-reversed index order; applying the permutation recovers natural order."""
    n = 6
    N = 1 << n
    x = qft_inputs.gaussian(n, seed=9)
    nat = oracle_mod.circuit(x, natural_order=True)
    rev = oracle_mod.circuit(x, natural_order=False)
    perm = np.array([oracle_mod.bit_reverse(i, n) for i in range(N)])
    assert np.array_equal(nat, rev[perm])
    assert oracle_mod.bit_reverse(1, 6) == 32 and oracle_mod.bit_reverse(0b110100, 6) == 0b001011


@pytest.mark.parametrize("n,k", [(10, -1), (12, 3), (12, 0), (11, 7)])
def test_bins_match_circuit(oracle_mod, n, k):
    x = qft_inputs.tones(n, seed=4)
    full = oracle_mod.circuit(x, k=k)
    ys = [0, 1, 2, (1 << n) - 1, 777 % (1 << n), 1234 % (1 << n)]
    for sign in (-1,):
        b = oracle_mod.aqft_bins(x, ys, k=k, sign=sign)
        assert rel_l2(b, full[ys]) < 1e-12


# ----------------------------------------------------- circuit shape pins

def _read_golden(name):
    rows = []
    with open(os.path.join(GOLDEN, name)) as f:
        for line in f:
            line = line.strip()
            if line and not line.startswith("#"):
                rows.append(line)
    return rows


def test_table2_cp_counts(oracle_mod):
    """Table 2: controlled-R_m counts of the 22-qubit circuit per cutoff k."""
    for row in _read_golden("table2_cp_counts.txt"):
        n, k, count = map(int, row.split())
        assert oracle_mod.gate_counts(n, k)[1] == count


def test_exact_counts():
    """Sec. 2: the exact n-wire circuit has n H and n(n-1)/2 controlled phases;
    floor(n/2) swaps reverse the qubit order (n=10: 10 / 45 / 5)."""
    import oracle

    assert oracle.gate_counts(10, -1) == (10, 45, 5)
    for n in range(1, 30):
        assert oracle.gate_counts(n, -1) == (n, n * (n - 1) // 2, n // 2)


def test_fig1_gate_sequence(oracle_mod):
    for row in _read_golden("fig1_qft3_gates.txt"):
        k, seq = row.split("|")
        want = []
        for g in seq.split(";"):
            f = g.split()
            if f[0] == "H":
                want.append(("H", int(f[1])))
            elif f[0] == "CR":
                want.append(("CR", int(f[1]), int(f[2]), int(f[3])))
            else:
                want.append(("SWAP", int(f[1]), int(f[2])))
        assert oracle_mod.gate_list(3, int(k)) == want


# ----------------------------------------------- the paper's DFT_8 example

def _L(N, K):
    """Stride permutation L^{N}_{K} (Sec. 2, Eq. 2): the map i*M + j -> j*K + i
    (i < K, j < M = N/K) read as "output entry i*M + j is input entry j*K + i",
    i.e. the matrix has a one at (i*M + j, j*K + i)."""
    M = N // K
    P = np.zeros((N, N))
    for i in range(K):
        for j in range(M):
            P[i * M + j, j * K + i] = 1.0
    return P


def _T(N, M, sign=-1):
    """Cooley-Tukey twiddle T^{N}_{M}: block diagonal, block i = diag(w_N^{i j}, j<M)."""
    K = N // M
    w = np.exp(sign * 2j * np.pi / N)
    return np.diag([w ** (i * j) for i in range(K) for j in range(M)])


def _dft(N, sign=-1):
    k = np.arange(N)
    return np.exp(sign * 2j * np.pi * np.outer(k, k) / N)


def test_dft8_worked_example(oracle_mod):
    """Eq. 3 (two-level radix-2 DFT_8), the radix-2 block form with the T~
    factors of Sec. 2, and the oracle circuit for n=3 all give DFT_8."""
    H = np.array([[1, 1], [1, -1]], dtype=np.complex128)
    I2, I4 = np.eye(2), np.eye(4)
    dft4 = np.kron(H, I2) @ _T(4, 2) @ np.kron(I2, H) @ _L(4, 2)
    assert np.allclose(dft4, _dft(4))
    dft8 = np.kron(dft4, I2) @ _T(8, 2) @ np.kron(I4, H) @ _L(8, 4)
    assert np.allclose(dft8, _dft(8))

    # radix-2 block form: DFT*_N = (I_2 (x) DFT*_{N/2}) T~_N (H (x) I_{N/2})
    E1, E2 = np.diag([1.0, 0.0]), np.diag([0.0, 1.0])
    R = lambda j: np.diag([1.0, np.exp(-2j * np.pi / 2 ** j)])  # noqa: E731
    I1 = np.eye(2)
    Tt4 = np.kron(I1, E1) + np.kron(R(2), E2)
    Tt8 = (np.kron(np.kron(I1, I1), E1) + np.kron(np.kron(R(3), I1), E2)) @ \
          (np.kron(np.kron(I1, E1), I1) + np.kron(np.kron(R(2), E2), I1))
    dft4s = np.kron(I2, H) @ Tt4 @ np.kron(H, I2)
    dft8s = np.kron(I2, dft4s) @ Tt8 @ np.kron(H, I4)
    rev = [int(format(i, "03b")[::-1], 2) for i in range(8)]
    assert np.allclose(dft8s[rev, :], _dft(8))  # product of L's = bit reversal

    # oracle circuit matrix: natural order == DFT_8/sqrt 8, deferred swaps == DFT*_8/sqrt 8
    I8 = np.eye(8, dtype=np.complex128)
    nat = np.stack([oracle_mod.circuit(I8[:, j], k=2, sign=-1) for j in range(8)], axis=1)
    raw = np.stack([oracle_mod.circuit(I8[:, j], k=2, sign=-1, natural_order=False)
                    for j in range(8)], axis=1)
    assert np.allclose(nat * np.sqrt(8), _dft(8), atol=1e-13)
    assert np.allclose(raw * np.sqrt(8), dft8s, atol=1e-13)


def test_sparse_dft_bins_against_dense_and_numpy(oracle_mod):
    """dft_bins_sparse (Sec. 2 definition over the nonzeros, exact integer
    phases) equals the O(N^2) DFT at n = 10 and numpy.fft at n = 20, in both
    directions; and for n = 34 its integer phase equals Python's exact
    (x * y) mod 2^n."""
    rng = np.random.default_rng(11)
    for n, check in ((10, "dense"), (20, "numpy")):
        N = 1 << n
        idx = rng.choice(N, size=64, replace=False)
        vals = rng.standard_normal(64) + 1j * rng.standard_normal(64)
        x = np.zeros(N, dtype=np.complex128)
        x[idx] = vals
        ys = rng.integers(0, N, size=40)
        for sign in (-1, 1):
            got = oracle_mod.dft_bins_sparse(idx, vals, n, ys, sign)
            if check == "dense":
                ref = oracle_mod.dft(x, sign)[ys]
            else:
                ref = (np.fft.fft(x) if sign < 0 else np.fft.ifft(x) * N)[ys]
            assert np.max(np.abs(got - ref)) <= 1e-9 * np.linalg.norm(vals) * np.sqrt(64)
    n = 34
    a = rng.integers(0, 1 << n, size=1000, dtype=np.uint64)
    b = rng.integers(0, 1 << n, size=1000, dtype=np.uint64)
    got = oracle_mod._mulmod_pow2(a, b, n)
    assert all(int(g) == (int(x) * int(y)) % (1 << n) for g, x, y in zip(got, a, b))


# ------------------------------------------------ Sec. 4 accuracy measures

def test_fidelity_closed_forms(oracle_mod):
    """F = |<a,b>|^2 / (|a|^2 |b|^2) (Sec. 4): 1 under any complex rescaling,
    0 for orthogonal states, cos^2(theta) between unit vectors at angle
    theta, symmetric in its arguments."""
    rng = np.random.default_rng(7)
    a = rng.normal(size=64) + 1j * rng.normal(size=64)
    assert abs(oracle_mod.fidelity(a, (0.3 - 2.1j) * a) - 1.0) < 1e-14
    e0, e1 = np.eye(8)[0], np.eye(8)[1]
    assert oracle_mod.fidelity(e0, e1) == 0.0
    for th in (0.1, 0.7, 1.3):
        b = np.cos(th) * e0 + np.exp(0.4j) * np.sin(th) * e1
        assert abs(oracle_mod.fidelity(e0, b) - np.cos(th) ** 2) < 1e-15
    b = rng.normal(size=64) + 1j * rng.normal(size=64)
    assert abs(oracle_mod.fidelity(a, b) - oracle_mod.fidelity(b, a)) < 1e-15
    # the transform of a basis state |0> has no controlled-phase rotation at
    # any cutoff (every control bit is 0): the range-k result is exact
    x = np.zeros(1 << 8, complex)
    x[0] = 1
    ex, _ = oracle_mod.qft(x, -1, -1, 0, True)
    for k in (0, 2, 5):
        ak, _ = oracle_mod.qft(x, k, -1, 0, True)
        assert abs(oracle_mod.fidelity(ak, ex) - 1.0) < 1e-14


def test_leakage_closed_forms(oracle_mod):
    """Leakage = 1 - |approx[y*]|^2 / |approx|^2 at y* = argmax |exact| (Sec. 4):
    0 for a state on the peak bin, p for weight p moved off it, 1 - 1/N for a
    flat state, and scale invariant."""
    N = 32
    exact = np.zeros(N, complex)
    exact[5] = 1
    assert oracle_mod.leakage(exact, exact) == 0.0
    for p in (1e-3, 0.25, 0.9):
        approx = np.zeros(N, complex)
        approx[5] = np.sqrt(1 - p)
        approx[9] = 1j * np.sqrt(p)
        assert abs(oracle_mod.leakage(approx, exact) - p) < 1e-15
        assert abs(oracle_mod.leakage(3.7 * approx, exact) - p) < 1e-14
    flat = np.exp(1j * np.arange(N)) / np.sqrt(N)
    assert abs(oracle_mod.leakage(flat, exact) - (1 - 1 / N)) < 1e-14
