"""Parity bounds shared by the GPU tests: the CUDA path against the FP64 oracle.

Norm-wise (the stated accuracy targets): relative L2 error <= 2e-6 for
complex64 and <= 1e-13 * n for complex128.

Element-wise.  A transform computed by log2 N levels of butterflies with
rounded twiddles commits, at each level, rounding errors of relative size
~eps on the values it touches; each error then travels through the levels
after it, which are unitary.  So the error in output bin i is a sum of
O(log2 N) terms, each bounded by eps times the magnitude of the values that
feed bin i at that level:

  * the bin's own value (rounding of the final values and of the output
    scale): eps * |ref_i|;
  * values spread over the whole output (errors committed early, which the
    later levels spread evenly): eps * ||ref|| / sqrt(N), the RMS amplitude;
  * values concentrated at a spectral peak.  Rounding of the peak's
    partial sums and twiddles leaks (a) into the rest of its last-pass
    column -- the last pass mixes only the 2^a bins that differ in its a
    wires (natural order: the bins equal modulo 2^(n - a); bit-reversed
    order: 2^a consecutive bins), so an error committed there stays in that
    column, spread over its bins -- and (b) into the bins at offsets +-2^k
    from the peak (measured at about 0.3 eps |peak| each, for any n).  Both
    are bounded by eps * max(||ref_col(i)||, ||ref||_inf) / 2^(a/2).

Hence the bound used here,

    |got_i - ref_i| <= C eps log2 N (|ref_i| + RMS + max(||ref_col(i)||, ||ref||_inf) / 2^(a/2)),

with eps = 2^-24 (complex64, FP32 arithmetic) or 2^-46 (complex128: the
double-float pairs' per-operation bound; the FP64 path is tighter), and
C = 8.  Measured on the kernel's data flow replayed in FP32 (n = 14..20):
worst ratios to this bound of 0.03 for Gaussian and 0.02 for basis-state
inputs, and up to 0.25 for single tones and tone mixtures, so the margin
over rounding is at least 4x.  Unlike the max-norm bound implied by the L2
target (||e||_inf <= tol * ||ref||), this one is tight at ordinary bins: at
n = 24 a single bin off by 1e-6 ||x|| exceeds it by more than 100x at a bin
of a flat spectrum and by 1.4x even when one peak holds the whole norm
(tests/test_parity_bounds.py; on the GPU,
tests/test_gpu_parity.py::test_planted_single_bin_error_is_caught).
Index maps (permutations, argmax bins) are compared bit-exactly elsewhere.
"""
from __future__ import annotations

import numpy as np

TOL = {"c64": lambda n: 2e-6, "c128": lambda n: 1e-13 * max(n, 1)}
EPS = {"c64": 2.0 ** -24, "c128": 2.0 ** -46}
C_ELEM = 8.0


def rel_l2(a, b):
    return float(np.linalg.norm(np.ravel(a) - np.ravel(b)) / max(np.linalg.norm(np.ravel(b)), 1e-300))


def elementwise_bound(ref, dt: str, n: int, a_last: int | None = None, natural: bool = True,
                      eps: float | None = None) -> np.ndarray:
    """Per-bin error bound (see the module docstring).  a_last: wires of the
    plan's last pass (None or >= n: one pass, the column is the whole output).
    eps: the arithmetic's unit roundoff when it is not the dtype's (the
    tensor-core tiers: the operand format's)."""
    ref = np.asarray(ref).ravel()
    N = ref.size
    absr = np.abs(ref)
    rms = float(np.linalg.norm(ref)) / np.sqrt(N)
    peak = float(absr.max()) if N else 0.0
    col = np.full(N, float(np.linalg.norm(ref)))
    a = n
    if a_last is not None and 0 < a_last < n and N == (1 << n):
        a = a_last
        e2 = absr.astype(np.float64) ** 2
        if natural:  # the last pass's wires are output bits n-a .. n-1
            colE = e2.reshape(1 << a_last, 1 << (n - a_last)).sum(axis=0)
            col = np.tile(np.sqrt(colE), 1 << a_last)
        else:  # bit-reversed order: its wires are output bits 0 .. a-1
            colE = e2.reshape(1 << (n - a_last), 1 << a_last).sum(axis=1)
            col = np.repeat(np.sqrt(colE), 1 << a_last)
    conc = np.maximum(col, peak) / np.sqrt(float(1 << a)) if N else col
    return C_ELEM * (EPS[dt] if eps is None else eps) * max(n, 1) * (absr + rms + conc)


def plan_shape(plan):
    """(wires of the last pass, natural order?) of a Plan, for elementwise_bound."""
    info = plan.info()
    return int(info.wires_per_pass[info.passes - 1]), info.order == 0


def check_close(got, ref, dt: str, n: int, a_last: int | None = None, natural: bool = True):
    """None if got matches ref within both bounds, else a message."""
    got = np.asarray(got).ravel()
    ref = np.asarray(ref).ravel()
    tol = TOL[dt](n)
    err = rel_l2(got, ref)
    if not err <= tol:
        return f"rel L2 {err:.3e} > {tol:.1e}"
    bound = elementwise_bound(ref, dt, n, a_last, natural)
    ratio = np.abs(got - ref) / bound
    i = int(np.argmax(ratio))
    if not ratio[i] <= 1.0:
        return (f"bin {i}: |error| {abs(got[i] - ref[i]):.3e} > element bound {bound[i]:.3e} "
                f"(|ref| {abs(ref[i]):.3e}, ratio {ratio[i]:.2f})")
    return None


def assert_close(got, ref, dt: str, n: int, a_last: int | None = None, natural: bool = True):
    msg = check_close(got, ref, dt, n, a_last, natural)
    assert msg is None, msg
