"""Quantum phase estimation on the QFT engine (GPU), pinned to textbook
results and to the CPU oracle.

For an eigenphase theta (turns) and m counting qubits, the readout
distribution is the Fejer kernel P(x) = sin^2(pi M d) / (M^2 sin^2(pi d)) with
M = 2^m and d = theta - x/M (Nielsen & Chuang, Sec. 5.2.1); a dyadic theta = x0/M
gives P(x0) = 1; the nearest estimate has probability >= 4/pi^2; a mixture of
eigenvectors gives the |c_j|^2-weighted sum of kernels.  The oracle path
prepares the same state in numpy from its definition and applies the oracle's
transform to each system component.
"""
import math

import numpy as np
import pytest

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
q = pytest.importorskip("paper_2606_18981_gb300")

TOL = {"c64": 2e-6, "c128": 1e-12}


def fejer(theta, m):
    M = 1 << m
    d = theta - np.arange(M) / M
    d = d - np.round(d)
    s = np.sin(np.pi * d)
    with np.errstate(divide="ignore", invalid="ignore"):
        p = np.sin(np.pi * M * d) ** 2 / (M * M * s * s)
    p[np.abs(s) < 1e-300] = 1.0
    return p


@pytest.mark.parametrize("dt", ["c64", "c128"])
@pytest.mark.parametrize("m", [4, 10, 16])
def test_dyadic_phase_is_exact(dt, m):
    M = 1 << m
    for x0 in (0, 1, M // 3, M - 1):
        p = q.qpe([x0 / M], [1.0], m, dtype=dt).cpu().numpy()
        assert int(np.argmax(p)) == x0
        assert abs(p[x0] - 1.0) <= TOL[dt] * m


@pytest.mark.parametrize("dt", ["c64", "c128"])
@pytest.mark.parametrize("m", [6, 12, 18])
def test_fejer_kernel_and_success_bound(dt, m):
    for theta in (math.pi / 10, 0.7071067811865476, 0.123456789):
        p = q.qpe([theta], [1.0], m, dtype=dt).cpu().numpy()
        ref = fejer(theta, m)
        assert np.max(np.abs(p - ref)) <= TOL[dt] * m
        assert abs(p.sum() - 1.0) <= TOL[dt] * m
        nearest = int(round(theta * (1 << m))) % (1 << m)
        assert p[nearest] >= 4 / math.pi ** 2 - TOL[dt]


@pytest.mark.parametrize("dt", ["c64", "c128"])
def test_mixture_against_kernels_and_oracle(oracle_mod, dt):
    m = 11
    M = 1 << m
    thetas = np.array([0.1, 0.37, 0.625, 0.9001])
    c = np.array([0.5, 0.5j, -0.5, 0.5 * np.exp(0.3j)])
    p = q.qpe(thetas, c, m, dtype=dt).cpu().numpy()
    ref = sum(abs(c[j]) ** 2 * fejer(thetas[j], m) for j in range(4))
    assert np.max(np.abs(p - ref)) <= TOL[dt] * m
    # oracle: the prepared state from its definition, then the oracle's transform per component
    y = np.arange(M)
    po = np.zeros(M)
    for j in range(4):
        psi = c[j] * np.exp(2j * np.pi * ((thetas[j] * y) % 1.0)) / np.sqrt(M)
        out, _ = oracle_mod.qft(psi, -1, -1, oracle_mod.SCALE_UNITARY, True)
        po += np.abs(out) ** 2
    assert np.max(np.abs(p - po)) <= TOL[dt] * m


def test_aqft_readout_against_oracle(oracle_mod):
    """The readout with an AQFT cutoff k (fewer controlled phases) against the oracle's AQFT."""
    m, k = 12, 4
    M = 1 << m
    theta = 0.3
    p = q.qpe([theta], [1.0], m, k=k, dtype="c128").cpu().numpy()
    psi = np.exp(2j * np.pi * ((theta * np.arange(M)) % 1.0)) / np.sqrt(M)
    out, _ = oracle_mod.qft(psi, k, -1, oracle_mod.SCALE_UNITARY, True)
    assert np.max(np.abs(p - np.abs(out) ** 2)) <= 1e-12 * m
    assert int(np.argmax(p)) == int(round(theta * M))
