"""GPU parity of QFTs on qubit subsets (multi-dimensional and strided batched
transforms) against the CPU FP64 oracle: every sub-vector along index bits
[w0, w0 + m) of the register transformed independently, for single-pass and
multi-pass plans in both output orders; and the 2-D transform (rows, then
columns) against the oracle applied along each axis and numpy.fft.fft2.
"""
import numpy as np
import pytest

import qft_inputs

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
q = pytest.importorskip("paper_2606_18981_gb300")

TOL = {"c64": lambda n: 2e-6, "c128": lambda n: 1e-13 * max(n, 1)}
CDT = {"c64": torch.complex64, "c128": torch.complex128}


def rel_l2(a, b):
    return float(np.linalg.norm(np.ravel(a) - np.ravel(b)) / max(np.linalg.norm(np.ravel(b)), 1e-300))


def subset_reference(oracle_mod, x, n_addr, w0, m, k, sign, mode, natural):
    a = np.asarray(x, dtype=np.complex128).reshape(1 << (n_addr - w0 - m), 1 << m, 1 << w0)
    out = np.empty_like(a)
    for hi in range(a.shape[0]):
        for lo in range(a.shape[2]):
            out[hi, :, lo], _ = oracle_mod.qft(a[hi, :, lo].copy(), k, sign, mode, natural)
    return out.ravel()


CASES = [(10, 0, 6), (12, 0, 8), (16, 0, 13), (11, 3, 5), (12, 4, 8), (14, 5, 9), (15, 4, 11), (13, 6, 7),
         (12, 2, 6), (18, 4, 14), (23, 0, 16), (24, 0, 18)]


@pytest.mark.parametrize("dt", ["c64", "c128"])
@pytest.mark.parametrize("order", [0, 1])
@pytest.mark.parametrize("n_addr,w0,m", CASES)
def test_subset_against_oracle(oracle_mod, dt, order, n_addr, w0, m):
    x = qft_inputs.gaussian(n_addr, seed=7000 + 31 * w0 + m, normalise=False)
    if dt == "c64":
        x = x.astype(np.complex64).astype(np.complex128)
    for direction, k, mode in ((-1, -1, q.SCALE_UNNORM), (+1, 4, q.SCALE_UNITARY)):
        p = q.Plan(m, k, direction, dt, order, n_addr=n_addr, w0=w0)
        ws = p.alloc_workspace()
        st = torch.from_numpy(x).to(CDT[dt]).cuda()
        p.execute(st, ws, mode)
        got = st.cpu().numpy().astype(np.complex128)
        assert p.status(ws) == 0
        ref = subset_reference(oracle_mod, x, n_addr, w0, m, k, direction, mode, order == 0)
        assert rel_l2(got, ref) <= TOL[dt](m), (rel_l2(got, ref), p.info().passes)


@pytest.mark.parametrize("dt", ["c64", "c128"])
@pytest.mark.parametrize("a,b", [(5, 7), (10, 6), (7, 12), (12, 4), (3, 3), (9, 9)])
def test_fft2_against_oracle_and_numpy(oracle_mod, dt, a, b):
    rng = np.random.default_rng(a * 100 + b)
    x = rng.standard_normal((1 << a, 1 << b)) + 1j * rng.standard_normal((1 << a, 1 << b))
    if dt == "c64":
        x = x.astype(np.complex64).astype(np.complex128)
    got = q.fft2(torch.from_numpy(x).to(CDT[dt]).cuda()).cpu().numpy().astype(np.complex128)
    # oracle along each axis: rows (length 2^b) then columns (length 2^a)
    ref = np.array([oracle_mod.qft(r.copy(), -1, -1, q.SCALE_UNNORM, True)[0] for r in x])
    ref = np.array([oracle_mod.qft(c.copy(), -1, -1, q.SCALE_UNNORM, True)[0] for c in ref.T]).T
    assert rel_l2(got, ref) <= 2 * TOL[dt](a + b)
    assert rel_l2(got, np.fft.fft2(x)) <= 2 * TOL[dt](a + b)
    back = q.fft2(torch.from_numpy(got).to(CDT[dt]).cuda(), inverse=True).cpu().numpy()
    assert rel_l2(back, x) <= 4 * TOL[dt](a + b)


def test_subset_rejects_state_mode_and_batches():
    p = q.Plan(6, -1, q.FORWARD, "c64", n_addr=10, w0=4)
    st = torch.zeros(1 << 10, dtype=torch.complex64, device="cuda")
    ws = p.alloc_workspace()
    with pytest.raises(q.QftError):
        p.execute(st, ws, q.SCALE_STATE)
    with pytest.raises(q.QftError):
        q.Batch([p], [st], q.SCALE_UNNORM)
