"""GPU parity of the real-input transforms (R2C forward, C2R inverse) and of
out-of-place execution, against the CPU FP64 oracle.

The oracle for R2C is its own complex transform (the gate-by-gate circuit,
pinned to the DFT definition) applied to the real samples as a complex array,
unnormalised, of which bins 0 .. N/2 are the half spectrum.  For C2R it is the
oracle's inverse transform of the Hermitian extension of the half spectrum,
whose real part is the output.  Tolerances: relative L2 error <= 2e-6
(float32 data) and <= 1e-13 n (float64 data).
"""
import numpy as np
import pytest

import qft_inputs

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
q = pytest.importorskip("paper_2606_18981_gb300")

TOL = {"c64": lambda n: 2e-6, "c128": lambda n: 1e-13 * max(n, 1)}
RDT = {"c64": torch.float32, "c128": torch.float64}
CDT = {"c64": torch.complex64, "c128": torch.complex128}


def rel_l2(a, b):
    return float(np.linalg.norm(np.ravel(a) - np.ravel(b)) / max(np.linalg.norm(np.ravel(b)), 1e-300))


def real_input(n, seed, dt):
    x = np.random.default_rng(seed).standard_normal(1 << n)
    return x.astype(np.float32).astype(np.float64) if dt == "c64" else x


def oracle_rfft(oracle_mod, x):
    N = x.size
    full, _ = oracle_mod.qft(x.astype(np.complex128), -1, -1, oracle_mod.SCALE_UNNORM, True)
    return full[:N // 2 + 1]


def hermitian_full(X, N):
    full = np.zeros(N, dtype=np.complex128)
    full[:N // 2 + 1] = X
    full[0] = X[0].real
    full[N // 2] = X[N // 2].real
    full[N // 2 + 1:] = np.conj(X[1:N // 2][::-1])
    return full


def gpu_rplan(n, direction, dt, inp, out_len, mode):
    p = q.RealPlan(n, direction, dt)
    src = torch.from_numpy(np.ascontiguousarray(inp)).cuda()
    src_copy = src.clone()
    odt = CDT[dt] if direction == q.FORWARD else RDT[dt]
    out = torch.empty(out_len, dtype=odt, device="cuda")
    p.execute(src, out, p.alloc_workspace(), mode)
    torch.cuda.synchronize()
    assert torch.equal(src, src_copy), "input modified"
    return out.cpu().numpy().astype(np.complex128 if direction == q.FORWARD else np.float64)


@pytest.mark.parametrize("dt", ["c64", "c128"])
@pytest.mark.parametrize("n", [2, 3, 4, 6, 11, 13, 14, 17, 21])
def test_rfft_against_oracle(oracle_mod, dt, n):
    x = real_input(n, 10 + n, dt)
    ref = oracle_rfft(oracle_mod, x)
    got = gpu_rplan(n, q.FORWARD, dt, x.astype(np.float32 if dt == "c64" else np.float64), (1 << (n - 1)) + 1,
                    q.SCALE_UNNORM)
    assert rel_l2(got, ref) <= TOL[dt](n)
    assert np.max(np.abs(got - ref)) <= TOL[dt](n) * np.linalg.norm(ref)
    assert abs(got[0].imag) <= TOL[dt](n) * np.linalg.norm(ref) and abs(got[-1].imag) <= TOL[dt](n) * np.linalg.norm(ref)


@pytest.mark.parametrize("dt", ["c64", "c128"])
@pytest.mark.parametrize("n", [2, 3, 5, 10, 13, 16, 20])
def test_irfft_against_oracle(oracle_mod, dt, n):
    N = 1 << n
    rng = np.random.default_rng(50 + n)
    X = rng.standard_normal(N // 2 + 1) + 1j * rng.standard_normal(N // 2 + 1)
    if dt == "c64":
        X = X.astype(np.complex64).astype(np.complex128)
    full, _ = oracle_mod.qft(hermitian_full(X, N), -1, +1, oracle_mod.SCALE_UNNORM, True)
    ref = full.real / N
    got = gpu_rplan(n, q.INVERSE, dt, X.astype(np.complex64 if dt == "c64" else np.complex128), N, q.SCALE_INV_N)
    assert rel_l2(got, ref) <= TOL[dt](n)
    assert np.max(np.abs(got - ref)) <= TOL[dt](n) * np.linalg.norm(ref)


@pytest.mark.parametrize("dt", ["c64", "c128"])
def test_real_scale_modes_and_numpy(dt):
    n = 12
    N = 1 << n
    x = real_input(n, 77, dt)
    xin = x.astype(np.float32 if dt == "c64" else np.float64)
    for mode, f in ((q.SCALE_UNNORM, 1.0), (q.SCALE_UNITARY, N ** -0.5), (q.SCALE_INV_N, 1.0 / N)):
        got = gpu_rplan(n, q.FORWARD, dt, xin, N // 2 + 1, mode)
        assert rel_l2(got, np.fft.rfft(x) * f) <= TOL[dt](n)
    X = np.fft.rfft(x)
    Xin = X.astype(np.complex64 if dt == "c64" else np.complex128)
    for mode, f in ((q.SCALE_INV_N, 1.0), (q.SCALE_UNITARY, N ** 0.5), (q.SCALE_UNNORM, float(N))):
        got = gpu_rplan(n, q.INVERSE, dt, Xin, N, mode)
        assert rel_l2(got, np.fft.irfft(Xin.astype(np.complex128), N) * f) <= 2 * TOL[dt](n)


@pytest.mark.parametrize("dt", ["c64", "c128"])
def test_real_round_trip_and_convenience(dt):
    n = 19
    x = torch.from_numpy(real_input(n, 5, dt)).to(RDT[dt]).cuda()
    X = q.rfft(x)
    y = q.irfft(X)
    err = (torch.linalg.vector_norm((y - x).double()) / torch.linalg.vector_norm(x.double())).item()
    assert err <= 2 * TOL[dt](n)


def test_real_rejects_bad_arguments():
    p = q.RealPlan(8, q.FORWARD, "c64")
    x = torch.zeros(256, dtype=torch.float32, device="cuda")
    out = torch.empty(129, dtype=torch.complex64, device="cuda")
    ws = p.alloc_workspace()
    with pytest.raises(q.QftError):
        p.execute(x, out, ws, q.SCALE_STATE)
    with pytest.raises(q.QftError):
        p.execute(x, x, ws, q.SCALE_UNNORM)
    with pytest.raises(q.QftError):
        q.RealPlan(1, q.FORWARD, "c64")
    zero = gpu_rplan(8, q.FORWARD, "c64", np.zeros(256, dtype=np.float32), 129, q.SCALE_UNNORM)
    assert np.all(zero == 0)


@pytest.mark.parametrize("dt", ["c64", "c128"])
@pytest.mark.parametrize("order", [0, 1])
@pytest.mark.parametrize("n", [9, 16, 22])
def test_out_of_place_equals_in_place(dt, order, n):
    """execute_oop leaves its input unchanged and gives exactly the in-place result."""
    x = torch.from_numpy(qft_inputs.gaussian(n, seed=n, normalise=False)).to(CDT[dt]).cuda()
    p = q.Plan(n, -1, q.FORWARD, dt, order)
    ws = p.alloc_workspace()
    a = x.clone()
    p.execute(a, ws, q.SCALE_STATE)
    b = torch.empty_like(x)
    x0 = x.clone()
    p.execute_oop(x, b, ws, q.SCALE_STATE)
    torch.cuda.synchronize()
    assert p.status(ws) == 0
    assert torch.equal(x, x0)
    assert torch.equal(a, b)


@pytest.mark.parametrize("dt", ["c64", "c128"])
def test_padded_load_is_zero_padded_dft(oracle_mod, dt):
    """Sec. 3 step 1 with n = ceil(log2 len): the transform of the data padded with zeros."""
    n = 10
    N = 1 << n
    p = q.Plan(n, -1, q.FORWARD, dt)
    ws = p.alloc_workspace()
    state = torch.full((N,), 7.0 + 7.0j, dtype=CDT[dt], device="cuda")  # stale values must be overwritten
    for ln in (1, 700, 1000, N):
        x = qft_inputs.gaussian(n, seed=ln, normalise=False)[:ln]
        x = x.astype(np.complex64 if dt == "c64" else np.complex128)
        p.load(state, x, pad=True)
        p.execute(state, ws, q.SCALE_UNNORM)
        got = state.cpu().numpy().astype(np.complex128)
        xp = np.zeros(N, dtype=np.complex128)
        xp[:ln] = x
        ref = oracle_mod.dft(xp, -1)
        assert rel_l2(got, ref) <= TOL[dt](n)
    with pytest.raises(q.QftError):
        p.load(state, np.zeros(N + 1, dtype=np.complex64 if dt == "c64" else np.complex128), pad=True)
