"""CPU FP64 oracle for the QFT->FFT method (Markidis et al.).

TEST INFRASTRUCTURE ONLY: the test-suite, ``__graft_entry__.smoke()`` and the
benchmark's ``cpu_baseline`` / ``--impl reference`` legs are the only callers.
The GPU library never imports this package and shares no code with it.

The arithmetic lives in ``qft_oracle.c`` (plain C, FP64, OpenMP parallel-for
over amplitudes).  This module compiles it with gcc on first use (or when
``build()`` is called) and wraps it with ctypes for numpy complex128 arrays.

Conventions (paper Sec. 2-3): qubit q_j is bit j of the array index (LSB q_0);
sign = -1 is the forward transform with omega_N = e^{-2 pi i/N}; the circuit is
the unitary U = DFT_N / sqrt(N); the final swaps give the natural output order.

Functions:
  encode(x)                    Sec. 3 step 1
  circuit(psi, n, k, sign)     Sec. 3 steps 2-3, Fig. 1 (+ Sec. 2 AQFT cutoff)
  decode(psi, scale_in, mode)  Sec. 3 step 4
  qft(x, k, sign, mode)        encode -> circuit -> decode
  dft(x, sign)                 Sec. 2 DFT definition, O(N^2)
  aqft_direct(x, k, sign)      closed-form matrix elements of the range-k AQFT
  aqft_bins(x, ys, k, sign)    a few output bins by O(N) direct summation
  dft_bins_sparse(idx, vals, n, ys, sign)
                               output bins of the Sec. 2 DFT of an input with
                               few nonzeros, summed over the nonzeros only
  mc_sample(x, u)              Sec. 6 Monte Carlo backend: importance-sampled input
                               indices and weights for given uniforms
  mc_sample_sparse(pos, vals, u), aqft_bins_sparse(pos, vals, n, ys, k, sign)
                               the same for an input of few nonzeros in an n-wire
                               register (n <= 62)
  mc_bins(idx, w, n, ys, k, sign)
                               per output bin: the sample mean of the path
                               amplitudes, the unbiased power estimate, the
                               standard error
  gate_counts(n, k)            Table 2
  gate_list(n, k)              Fig. 1
  fidelity(a, b), leakage(...) Sec. 4 accuracy measures
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "qft_oracle.c")
_LIB_PATH = os.path.join(_HERE, "liboracle.so")
_lock = threading.Lock()
_lib = None

SCALE_STATE, SCALE_UNITARY, SCALE_UNNORM, SCALE_INV_N = 0, 1, 2, 3
FORWARD, INVERSE = -1, +1


def build(force: bool = False) -> str:
    """Compile qft_oracle.c into liboracle.so next to it (gcc, OpenMP)."""
    if force or not os.path.exists(_LIB_PATH) or os.path.getmtime(_LIB_PATH) < os.path.getmtime(_SRC):
        tmp = _LIB_PATH + f".{os.getpid()}.tmp"
        cmd = ["gcc", "-O2", "-std=c11", "-ffp-contract=off", "-fopenmp", "-fPIC", "-shared",
               _SRC, "-o", tmp, "-lm"]
        subprocess.run(cmd, check=True)
        os.replace(tmp, _LIB_PATH)
    return _LIB_PATH


def _load():
    global _lib
    with _lock:
        if _lib is not None:
            return _lib
        build()
        lib = ctypes.CDLL(_LIB_PATH)
        dp = ctypes.POINTER(ctypes.c_double)
        i64p = ctypes.POINTER(ctypes.c_int64)
        ip = ctypes.POINTER(ctypes.c_int)
        lib.oracle_encode.argtypes = [ctypes.c_int, dp, dp]
        lib.oracle_encode.restype = ctypes.c_double
        lib.oracle_circuit.argtypes = [ctypes.c_int, ctypes.c_int, ctypes.c_int, ctypes.c_int, dp]
        lib.oracle_circuit.restype = None
        lib.oracle_decode.argtypes = [ctypes.c_int, dp, ctypes.c_double, ctypes.c_int, dp]
        lib.oracle_decode.restype = None
        lib.oracle_dft.argtypes = [ctypes.c_int, ctypes.c_int, dp, dp]
        lib.oracle_dft.restype = None
        lib.oracle_aqft_direct.argtypes = [ctypes.c_int, ctypes.c_int, ctypes.c_int, dp, dp]
        lib.oracle_aqft_direct.restype = None
        lib.oracle_aqft_bins.argtypes = [ctypes.c_int, ctypes.c_int, ctypes.c_int, dp, i64p,
                                         ctypes.c_int, dp]
        lib.oracle_aqft_bins.restype = None
        lib.oracle_gate_counts.argtypes = [ctypes.c_int, ctypes.c_int, i64p, i64p, i64p]
        lib.oracle_gate_counts.restype = None
        lib.oracle_gate_list.argtypes = [ctypes.c_int, ctypes.c_int, ctypes.c_int, ip, ctypes.c_int]
        lib.oracle_gate_list.restype = ctypes.c_int
        lib.oracle_apply_gate.argtypes = [ctypes.c_int, ctypes.c_int, ctypes.c_int, ctypes.c_int,
                                          ctypes.c_int, ctypes.c_int, dp]
        lib.oracle_apply_gate.restype = None
        lib.oracle_bit_reverse.argtypes = [ctypes.c_int64, ctypes.c_int]
        lib.oracle_bit_reverse.restype = ctypes.c_int64
        lib.oracle_mc_sample.argtypes = [ctypes.c_int, dp, dp, ctypes.c_int64, i64p, dp]
        lib.oracle_mc_sample.restype = ctypes.c_uint64
        lib.oracle_mc_bins.argtypes = [ctypes.c_int, ctypes.c_int, ctypes.c_int, i64p, dp, ctypes.c_int64, i64p,
                                       ctypes.c_int, dp]
        lib.oracle_mc_sample_sparse.argtypes = [ctypes.c_int64, i64p, dp, dp, ctypes.c_int64, i64p, dp]
        lib.oracle_mc_sample_sparse.restype = ctypes.c_uint64
        lib.oracle_aqft_bins_sparse.argtypes = [ctypes.c_int, ctypes.c_int, ctypes.c_int, ctypes.c_int64, i64p, dp,
                                                i64p, ctypes.c_int, dp]
        lib.oracle_aqft_bins_sparse.restype = None
        lib.oracle_mc_bins.restype = None
        lib.oracle_num_threads.argtypes = []
        lib.oracle_num_threads.restype = ctypes.c_int
        lib.oracle_set_num_threads.argtypes = [ctypes.c_int]
        lib.oracle_set_num_threads.restype = None
        _lib = lib
        return lib


def _as_c128(x) -> np.ndarray:
    a = np.ascontiguousarray(np.asarray(x, dtype=np.complex128))
    return a


def _dptr(a: np.ndarray):
    return a.ctypes.data_as(ctypes.POINTER(ctypes.c_double))


def _log2_exact(N: int) -> int:
    n = int(N).bit_length() - 1
    if N <= 0 or (1 << n) != N:
        raise ValueError(f"length {N} is not a power of two")
    return n


def num_threads() -> int:
    return _load().oracle_num_threads()


def set_num_threads(t: int) -> None:
    _load().oracle_set_num_threads(int(t))


def encode(x):
    """Sec. 3 step 1: returns (psi = x / ||x||_2, scale_in = ||x||_2)."""
    lib = _load()
    x = _as_c128(x)
    n = _log2_exact(x.size)
    psi = np.empty_like(x)
    s = lib.oracle_encode(n, _dptr(x), _dptr(psi))
    return psi, s


def circuit(psi, k: int = -1, sign: int = FORWARD, natural_order: bool = True) -> np.ndarray:
    """Apply the range-k (A)QFT circuit gate by gate; returns a new array."""
    lib = _load()
    out = _as_c128(psi).copy()
    n = _log2_exact(out.size)
    lib.oracle_circuit(n, int(k), int(sign), 1 if natural_order else 0, _dptr(out))
    return out


def decode(psi, scale_in: float, mode: int = SCALE_STATE) -> np.ndarray:
    """Sec. 3 step 4: rescale the final state to FFT units."""
    lib = _load()
    psi = _as_c128(psi)
    n = _log2_exact(psi.size)
    out = np.empty_like(psi)
    lib.oracle_decode(n, _dptr(psi), float(scale_in), int(mode), _dptr(out))
    return out


def qft(x, k: int = -1, sign: int = FORWARD, mode: int = SCALE_STATE, natural_order: bool = True):
    """encode -> circuit -> decode.  Returns (output, scale_in)."""
    psi, s = encode(x)
    return decode(circuit(psi, k, sign, natural_order), s, mode), s


def dft(x, sign: int = FORWARD) -> np.ndarray:
    """Unnormalised DFT by its definition (Sec. 2), O(N^2)."""
    lib = _load()
    x = _as_c128(x)
    n = _log2_exact(x.size)
    out = np.empty_like(x)
    lib.oracle_dft(n, int(sign), _dptr(x), _dptr(out))
    return out


def aqft_direct(x, k: int = -1, sign: int = FORWARD) -> np.ndarray:
    """U_k x (natural order, swaps included) from closed-form matrix elements, O(N^2)."""
    lib = _load()
    x = _as_c128(x)
    n = _log2_exact(x.size)
    out = np.empty_like(x)
    lib.oracle_aqft_direct(n, int(k), int(sign), _dptr(x), _dptr(out))
    return out


def aqft_bins(x, ys, k: int = -1, sign: int = FORWARD) -> np.ndarray:
    """Selected output bins <y|U_k|x> by O(N) direct summation each."""
    lib = _load()
    x = _as_c128(x)
    n = _log2_exact(x.size)
    ys = np.ascontiguousarray(np.asarray(ys, dtype=np.int64))
    out = np.empty(ys.size, dtype=np.complex128)
    lib.oracle_aqft_bins(n, int(k), int(sign), _dptr(x),
                         ys.ctypes.data_as(ctypes.POINTER(ctypes.c_int64)), int(ys.size), _dptr(out))
    return out


def _mulmod_pow2(a, b, n: int):
    """(a * b) mod 2^n exactly for uint64 arrays with a, b < 2^n <= 2^34:
    b is split into 17-bit halves so that no partial product reaches 2^64."""
    a = np.asarray(a, dtype=np.uint64)
    b = np.asarray(b, dtype=np.uint64)
    mask = np.uint64((1 << n) - 1)
    lo = b & np.uint64((1 << 17) - 1)
    hi = b >> np.uint64(17)
    t = ((a * hi) & mask) << np.uint64(17)
    return (t + a * lo) & mask


def dft_bins_sparse(idx, vals, n: int, ys, sign: int = FORWARD) -> np.ndarray:
    """Bins y of the unnormalised DFT (Sec. 2) X[y] = sum_x v_x e^{sign 2 pi i x y / N}
    of a length-N = 2^n input that is zero except v_m at indices idx_m: the
    definition summed over the nonzeros only, with the phase x*y mod N formed
    exactly in integers.  For large-n checks where an O(N) sum per bin is too slow."""
    idx = np.asarray(idx, dtype=np.uint64)
    vals = np.asarray(vals, dtype=np.complex128)
    out = np.empty(len(ys), dtype=np.complex128)
    N = float(1 << n)
    for i, y in enumerate(np.asarray(ys, dtype=np.uint64)):
        ph = _mulmod_pow2(idx, np.full(idx.shape, y, dtype=np.uint64), n).astype(np.float64) / N
        out[i] = np.sum(vals * np.exp(sign * 2j * np.pi * ph))
    return out


def gate_counts(n: int, k: int = -1):
    """(n_H, n_CP, n_swap) of the range-k circuit (Table 2)."""
    lib = _load()
    a, b, c = ctypes.c_int64(), ctypes.c_int64(), ctypes.c_int64()
    lib.oracle_gate_counts(int(n), int(k), ctypes.byref(a), ctypes.byref(b), ctypes.byref(c))
    return a.value, b.value, c.value


def gate_list(n: int, k: int = -1, natural_order: bool = True):
    """The gate sequence (Fig. 1): list of ('H', t) / ('CR', control, target, m) / ('SWAP', a, b)."""
    lib = _load()
    cap = n + n * n + n
    buf = (ctypes.c_int * (4 * cap))()
    g = lib.oracle_gate_list(int(n), int(k), 1 if natural_order else 0, buf, cap)
    out = []
    for i in range(g):
        kind, a, b, m = buf[4 * i: 4 * i + 4]
        if kind == 0:
            out.append(("H", a))
        elif kind == 1:
            out.append(("CR", a, b, m))
        else:
            out.append(("SWAP", a, b))
    return out


def apply_gate(psi: np.ndarray, kind: str, a: int = 0, b: int = 0, m: int = 0, sign: int = FORWARD) -> None:
    """In place on a complex128 array: 'H' on q_a, 'CR' (control a, target b, R_m), or 'SWAPS'."""
    lib = _load()
    n = _log2_exact(psi.size)
    assert psi.dtype == np.complex128 and psi.flags.c_contiguous
    code = {"H": 0, "CR": 1, "SWAPS": 2}[kind]
    lib.oracle_apply_gate(n, code, int(a), int(b), int(m), int(sign), _dptr(psi))


def bit_reverse(i: int, n: int) -> int:
    return _load().oracle_bit_reverse(int(i), int(n))


def fidelity(a, b) -> float:
    """Sec. 4: squared, normalised inner product |<a,b>|^2 / (||a||^2 ||b||^2)."""
    a = np.asarray(a, dtype=np.complex128).ravel()
    b = np.asarray(b, dtype=np.complex128).ravel()
    num = abs(np.vdot(a, b)) ** 2
    den = np.vdot(a, a).real * np.vdot(b, b).real
    return float(num / den) if den > 0 else 1.0


def leakage(approx, exact) -> float:
    """Sec. 4 top-bin leakage: 1 - |approx[y*]|^2 / ||approx||^2, y* = argmax |exact|."""
    approx = np.asarray(approx, dtype=np.complex128).ravel()
    ystar = int(np.argmax(np.abs(np.asarray(exact).ravel())))
    tot = np.vdot(approx, approx).real
    return float(1.0 - abs(approx[ystar]) ** 2 / tot) if tot > 0 else 0.0


def mc_sample(x, u):
    """Sec. 6 Monte Carlo backend, sampling step: for each uniform u_m in [0, 1)
    (a multiple of 2^-53) the input index j_m drawn with probability
    q_j / T (q_j = ceil(m_j 2^(62-n) / max m), m_j = max(|Re x_j|, |Im x_j|),
    T = sum q) and its weight w_m = x_j T / q_j.  Returns (idx int64,
    w complex128, T)."""
    lib = _load()
    x = _as_c128(x)
    n = _log2_exact(x.size)
    u = np.ascontiguousarray(np.asarray(u, dtype=np.float64))
    idx = np.empty(u.size, dtype=np.int64)
    w = np.empty(u.size, dtype=np.complex128)
    T = lib.oracle_mc_sample(n, _dptr(x), u.ctypes.data_as(ctypes.POINTER(ctypes.c_double)), int(u.size),
                             idx.ctypes.data_as(ctypes.POINTER(ctypes.c_int64)), _dptr(w))
    return idx, w, int(T)


def mc_sample_sparse(pos, vals, u):
    """mc_sample for a sparse input: amplitude vals[j] at input index pos[j] of
    an n-wire register (any n <= 62); the proposal runs over the list (S from
    ceil(log2 K)); returns (input indices int64, w complex128, T)."""
    lib = _load()
    pos = np.ascontiguousarray(np.asarray(pos, dtype=np.int64))
    vals = _as_c128(vals)
    u = np.ascontiguousarray(np.asarray(u, dtype=np.float64))
    idx = np.empty(u.size, dtype=np.int64)
    w = np.empty(u.size, dtype=np.complex128)
    T = lib.oracle_mc_sample_sparse(int(pos.size), pos.ctypes.data_as(ctypes.POINTER(ctypes.c_int64)), _dptr(vals),
                                    u.ctypes.data_as(ctypes.POINTER(ctypes.c_double)), int(u.size),
                                    idx.ctypes.data_as(ctypes.POINTER(ctypes.c_int64)), _dptr(w))
    return idx, w, int(T)


def aqft_bins_sparse(pos, vals, n: int, ys, k: int = -1, sign: int = FORWARD) -> np.ndarray:
    """<y|U_k|x> (closed-form elements, natural order) for an input with
    amplitudes vals at indices pos of an n-wire register (n <= 62), summed
    over the nonzeros only."""
    lib = _load()
    pos = np.ascontiguousarray(np.asarray(pos, dtype=np.int64))
    vals = _as_c128(vals)
    ys = np.ascontiguousarray(np.asarray(ys, dtype=np.int64))
    out = np.empty(ys.size, dtype=np.complex128)
    lib.oracle_aqft_bins_sparse(int(n), int(k), int(sign), int(pos.size),
                                pos.ctypes.data_as(ctypes.POINTER(ctypes.c_int64)), _dptr(vals),
                                ys.ctypes.data_as(ctypes.POINTER(ctypes.c_int64)), int(ys.size), _dptr(out))
    return out


def mc_bins(idx, w, n: int, ys, k: int = -1, sign: int = FORWARD):
    """Sec. 6 Monte Carlo backend, estimation step: per output bin y of the
    range-k transform (natural order) the mean of z_m = w_m e^{sign 2 pi i
    phase(j_m, y)/N} / sqrt(N) (an unbiased estimate of <y|U_k|x>), the
    unbiased power estimate (|sum z|^2 - sum |z|^2) / (M (M-1)) and the
    standard error of the mean.  Returns (amp complex128, power, stderr)."""
    lib = _load()
    idx = np.ascontiguousarray(np.asarray(idx, dtype=np.int64))
    w = _as_c128(w)
    ys = np.ascontiguousarray(np.asarray(ys, dtype=np.int64))
    out = np.empty(4 * ys.size, dtype=np.float64)
    lib.oracle_mc_bins(int(n), int(k), int(sign), idx.ctypes.data_as(ctypes.POINTER(ctypes.c_int64)), _dptr(w),
                       int(idx.size), ys.ctypes.data_as(ctypes.POINTER(ctypes.c_int64)), int(ys.size),
                       out.ctypes.data_as(ctypes.POINTER(ctypes.c_double)))
    out = out.reshape(-1, 4)
    return out[:, 0] + 1j * out[:, 1], out[:, 2], out[:, 3]
