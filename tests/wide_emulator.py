"""numpy replay of the wide pass kernel's data flow (csrc/qft_wide.cuh), for
checks on the CPU before the kernel runs on a GPU.

It follows the kernel step by step with the kernel's own thread maps (read
from tests/native/wide_index_check.cu --dump): stage 0 reads register j of
thread t at tile index wide_x0(t) | j << 9, forms each cross twiddle as the
kernel does -- the per-tile table UA (tile coordinates + batch bits x0..x3),
the per-kernel table VB (the thread's other five fixed bits) and the extra
batch bits' table W -- applies the diagonal and the block circuit to each
group, exchanges the values to wide_x1(t) | j << 4, runs stage 1 the same
way and stores through the kernel's offsets out_tile + othr(t) + oj(j).
Arithmetic is float64 by default, so a mismatch against the oracle means a
map or table mistake, not rounding.  With fp32=True every twiddle and every
intermediate value is rounded to complex64 as in the kernel (the operation
order differs in detail: no fused multiply-adds), which gives a realistic
rounding-error profile for checking the parity bounds themselves.  Test
helper only.
"""
from __future__ import annotations

import os
import subprocess

import numpy as np

from plan_emulator import _block_circuit, _brev, _gather_tma, check_structure, parse

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def thread_maps(exe: str):
    out = subprocess.run([exe, "--dump"], capture_output=True, text=True, check=True).stdout.split()
    a = np.array(out, dtype=np.int64).reshape(-1, 4)
    return {"x0": a[:, 1], "x1": a[:, 2], "x1top": a[:, 3]}


_FP32 = False


def _phase(beta, n, sign):
    w = np.exp(sign * 2j * np.pi * np.asarray(beta, dtype=np.float64) / float(1 << n))
    return w.astype(np.complex64) if _FP32 else w


def _block_circuit32(v, R, kk, sign):
    """The block's butterflies and controlled phases in complex64 arithmetic."""
    v = v.astype(np.complex64)
    for t in range(R - 1, -1, -1):
        bit = 1 << t
        js = [j for j in range(1 << R) if not (j & bit)]
        a = v[..., js].copy()
        b = v[..., [j | bit for j in js]].copy()
        v[..., js] = a + b
        v[..., [j | bit for j in js]] = a - b
        lo = max(0, t - kk)
        mask = (bit - 1) & ~((1 << lo) - 1)
        for j in range(1 << R):
            if j & bit:
                v[..., j] *= np.complex64(np.exp(sign * 2j * np.pi * (j & mask) / (2 * bit)))
    return v


def _cross_beta(I, n, hi, c, kk):
    """Integer cross phase of block wire c (units of 2^-n turns) from the logical bits I above hi."""
    I = np.asarray(I, dtype=np.uint64)
    rh = _brev(I, n) & np.uint64((1 << (n - 1 - hi)) - 1)
    lowcut = n - 1 - c - kk
    if lowcut > 0:
        rh &= ~np.uint64((1 << lowcut) - 1)
    return (rh << np.uint64(c)) & np.uint64((1 << n) - 1)


def _bits_to_wires(vals, positions, p_wire):
    """Logical bits (uint64) of values whose bit k sits at tile bit positions[k]."""
    vals = np.asarray(vals, dtype=np.int64)
    I = np.zeros(vals.shape, dtype=np.uint64)
    for k, pos in enumerate(positions):
        I |= ((vals >> k) & 1).astype(np.uint64) << np.uint64(p_wire[pos])
    return I


def _stage(v, P, S, ia, ib, vb_pos, w_pos, I_tile, sign, cross):
    """One register stage on v (T, 512, 32) in place, as the kernel does it."""
    n, kk, p_wire = P["n"], P["kk"], P["p_wire"]
    R = S["r"]
    E = 5 - R
    hi = S["wlo"] + R - 1
    Ia = _bits_to_wires(np.arange(16), range(4), p_wire)        # batch bits x0..x3
    Ib = _bits_to_wires(np.arange(32), vb_pos, p_wire)          # the other fixed bits
    Iw = _bits_to_wires(np.arange(1 << E), w_pos, p_wire)       # extra batch bits
    uv, Wt = [], []
    for e in range(R):
        c = S["wlo"] + e
        UA = _phase(_cross_beta(I_tile[:, None] | Ia[None, :], n, hi, c, kk), n, sign)  # (T, 16)
        VB = _phase(_cross_beta(Ib, n, hi, c, kk), n, sign) if cross else np.ones(32)
        uv.append(UA[:, ia] * VB[ib][None, :])                                           # (T, 512)
        Wt.append(_phase(_cross_beta(Iw, n, hi, c, kk), n, sign) if cross else np.ones(1 << E))
    jb = np.arange(1 << R)
    for js in range(1 << E):
        idx = js + (jb << E)
        g = v[:, :, idx]
        if cross:
            for e in range(R):
                tau = uv[e] * (Wt[e][js] if js else 1.0)
                sel = (jb >> e) & 1 == 1
                g[:, :, sel] *= tau[:, :, None]
        g = (_block_circuit32 if _FP32 else _block_circuit)(g, R, kk, sign)
        v[:, :, idx] = g


def run_wide_pass(P, src, dst, sign, scale_mode, norm_sq, maps):
    n = P["n"]
    T = P["num_tiles"]
    tiles = np.arange(T, dtype=np.int64)
    A = src[_gather_tma(P, src.size, tiles)]  # (T, 2^14) in tile-bit order x
    I_tile = np.zeros(T, dtype=np.uint64)
    out_tile = np.zeros(T, dtype=np.int64)
    for s in P["seg"]:
        c = ((tiles >> s["src"]) & ((1 << s["len"]) - 1)).astype(np.uint64)
        I_tile |= c << np.uint64(s["wire"])
        if s["out_rev"]:
            out_tile += (_brev(c, s["len"]) << np.uint64(s["out"] - s["len"] + 1)).astype(np.int64)
        else:
            out_tile += (c << np.uint64(s["out"])).astype(np.int64)
    S0, S1 = P["st"]
    top = P["first"] == 1
    x0, x1 = maps["x0"], maps["x1top" if top else "x1"]
    j = np.arange(32, dtype=np.int64)
    # stage 0
    v = A[:, x0[:, None] | (j[None, :] << 9)]
    cross0 = S0["wlo"] + S0["r"] - 1 < n - 1
    _stage(v, P, S0, x0 & 15, (x0 >> 4) & 31, [4 + k for k in range(5)], [9 + i for i in range(5 - S0["r"])],
           I_tile, sign, cross0)
    # exchange
    full = np.empty_like(A)
    full[:, x0[:, None] | (j[None, :] << 9)] = v
    v = full[:, x1[:, None] | (j[None, :] << 4)]
    # stage 1
    _stage(v, P, S1, x1 & 15, x1 >> 9, [9 + k for k in range(5)], [4 + i for i in range(5 - S1["r"])],
           I_tile, sign, True)
    # store
    p_out = P["p_out"]
    othr = np.zeros(512, dtype=np.int64)
    for b in range(14):
        othr += ((x1 >> b) & 1) << p_out[b]
    oj = np.zeros(32, dtype=np.int64)
    for e in range(5):
        oj += ((j >> e) & 1) << p_out[4 + e]
    inv_root_n = 2.0 ** (-n / 2)
    scale_in = np.sqrt(norm_sq)
    factor = {0: (inv_root_n / scale_in if scale_in > 0 else 0.0), 1: inv_root_n, 2: 1.0,
              3: inv_root_n * inv_root_n}[scale_mode]
    oaddr = out_tile[:, None, None] + othr[None, :, None] + oj[None, None, :]
    assert oaddr.min() >= 0 and oaddr.max() < dst.size
    if _FP32:
        dst[oaddr] = (v * np.float32(factor if P["last"] else 1.0)).astype(np.complex64)
    else:
        dst[oaddr] = v * (factor if P["last"] else 1.0)
    return oaddr.ravel()


def emulate_wide(plan, x, maps, scale_mode=0, fp32=False):
    """Replay every pass of a plan whose passes are all wide passes (fp32: in
    complex64 arithmetic, see the module docstring)."""
    global _FP32
    _FP32 = fp32
    info = plan.info()
    N = 1 << info.n_addr
    state = np.asarray(x, dtype=np.complex64 if fp32 else np.complex128).copy()
    work = np.zeros(N, dtype=state.dtype)
    bufs = [state, work]
    norm_sq = float(np.sum(np.abs(state.astype(np.complex128)) ** 2))
    for i in range(info.passes):
        P = parse(plan.describe_pass(i))
        assert P["wide"] == 1
        check_structure(P, 8)
        src, dst = bufs[P["in_buf"]], bufs[P["out_buf"]]
        written = run_wide_pass(P, src.copy(), dst, plan.direction, scale_mode, norm_sq, maps)
        assert np.array_equal(np.sort(written), np.arange(N)), "output map of a pass must be a bijection"
    _FP32 = False
    return bufs[0].astype(np.complex128)
