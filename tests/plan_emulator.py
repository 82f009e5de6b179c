"""CPU emulation of libqftfft's pass plans, for index checks before any kernel runs.

Reads each pass record (``qft_plan_describe_pass``) and replays it in numpy:
the TMA box gather (or the 1D bulk load), every register stage (group index ->
tile index, cross twiddle from exact integer phases, the block's butterflies
and controlled-phase rotations), the final store through the output address
map, and the norm / decode scale.  It mirrors the kernel's arithmetic in
float64 so that planner mistakes (a wrong wire map, stride, box coordinate,
lane map or stage split) show up as a mismatch against the oracle, and it
asserts that every index it forms is in bounds and that each map is a
bijection.  Test helper only.
"""
from __future__ import annotations

import numpy as np

K_MAX_STAGES, K_MAX_TILE_BITS, K_MAX_SEGS, K_MAX_DIMS, K_MAX_R = 8, 14, 8, 5, 7


def parse(rec):
    it = iter(rec)
    nx = lambda: int(next(it))  # noqa: E731
    P = {k: nx() for k in ("n", "kk", "tb", "nstages", "first", "last", "load_mode", "num_tiles")}
    st = []
    for _ in range(K_MAX_STAGES):
        s = {k: nx() for k in ("wlo", "r", "q", "cross", "ngbits", "tile_above", "uoff")}
        s["img"] = [nx() for _ in range(K_MAX_R)]
        s["lo_tw"] = nx()
        s["hi_tw"] = nx()
        s["gpos"] = [nx() for _ in range(K_MAX_TILE_BITS)]
        st.append(s)
    P["st"] = st[:P["nstages"]]
    P["p_wire"] = [nx() for _ in range(K_MAX_TILE_BITS)]
    P["p_out"] = [nx() for _ in range(K_MAX_TILE_BITS)]
    P["nseg"] = nx()
    segs = [{k: nx() for k in ("src", "len", "wire", "out", "out_rev")} for _ in range(K_MAX_SEGS)]
    P["seg"] = segs[:P["nseg"]]
    P["ndims"] = nx()
    P["dim_src"] = [nx() for _ in range(K_MAX_DIMS)]
    P["dim_len"] = [nx() for _ in range(K_MAX_DIMS)]
    P["gdim"] = [nx() for _ in range(K_MAX_DIMS)]
    P["gstride"] = [nx() for _ in range(4)]
    P["box"] = [nx() for _ in range(K_MAX_DIMS)]
    for k in ("grid", "smem", "in_buf", "out_buf", "npartials", "run_bits", "paired", "minb", "n_addr", "wide"):
        P[k] = nx()
    return P


def _groups(P, S):
    """Group bits of a stage as the emulation enumerates them: a paired stage's
    thread also covers tile bit 0 (its SIMD lane), so it is one more group bit."""
    gpos = list(S["gpos"][:S["ngbits"]])
    return gpos + [0] if P["paired"] else gpos


def _brev(v, length):
    v = np.asarray(v, dtype=np.uint64)
    r = np.zeros_like(v)
    for b in range(length):
        r |= ((v >> np.uint64(b)) & np.uint64(1)) << np.uint64(length - 1 - b)
    return r


def check_structure(P, esize):
    """Bijection checks that need no data: tile bits + tile-coordinate bits cover
    the input and the output address bits exactly once, TMA boxes fit, stage
    blocks are contiguous runs of wires and tile bits, lane maps are permutations."""
    n, tb, na = P["n"], P["tb"], P["n_addr"]  # transform wires; address bits (> n for subset plans)
    wires = sorted(P["p_wire"][:tb] + [s["wire"] + i for s in P["seg"] for i in range(s["len"])])
    assert wires == list(range(na)), "tile + segment wires must be a permutation of the wires"
    outs = list(P["p_out"][:tb])
    for s in P["seg"]:
        outs += [s["out"] - i if s["out_rev"] else s["out"] + i for i in range(s["len"])]
    assert sorted(outs) == list(range(na)), "output address bits must be a permutation"
    assert sum(s["len"] for s in P["seg"]) == na - tb
    assert P["num_tiles"] == 1 << (na - tb)
    pb0 = 1 if P["paired"] else 0
    if P["paired"]:
        assert esize == 8 and not (P["first"] and P["last"])
        assert all(s["q"] >= 1 and s["r"] <= 4 for s in P["st"]), "tile bit 0 is the pair lane, blocks <= 4 wires"
    for s in P["st"]:
        assert 1 <= s["r"] <= K_MAX_R and s["ngbits"] == tb - s["r"] - pb0
        assert 0 <= s["q"] and s["q"] + s["r"] <= tb
        for e in range(s["r"]):
            assert P["p_wire"][s["q"] + e] == s["wlo"] + e, "stage block must be consecutive wires on consecutive tile bits"
        others = sorted(s["gpos"][:s["ngbits"]])
        assert others == [p for p in range(pb0, tb) if not (s["q"] <= p < s["q"] + s["r"])]
    seg_wires = [s["wire"] + i for s in P["seg"] for i in range(s["len"])]
    uoff = 0
    for s in P["st"]:
        hi = s["wlo"] + s["r"] - 1
        above = lambda w: hi < w < n  # noqa: E731  (batch wires of subset plans carry no phase)
        assert s["tile_above"] == int(any(above(w) for w in seg_wires)), "per-tile twiddle flag"
        assert s["uoff"] == uoff
        lanes_above = any(above(P["p_wire"][s["gpos"][i]]) for i in range(min(5, s["ngbits"])))
        lanes_above = lanes_above or (P["paired"] and above(P["p_wire"][0]))
        high_above = any(above(P["p_wire"][s["gpos"][i]]) for i in range(5, s["ngbits"]))
        assert s["lo_tw"] == int(lanes_above) and s["hi_tw"] == int(high_above or not lanes_above)
        uoff += s["r"]
    # blocks processed top-down and covering each wire once
    blocks = [(s["wlo"], s["r"]) for s in P["st"]]
    for a, b in zip(blocks, blocks[1:]):
        assert b[0] + b[1] == a[0], "blocks must be consecutive, top-down"
    if P["load_mode"] == 0:
        mult = esize // 8
        elems = 1
        for d in range(K_MAX_DIMS):
            elems *= P["box"][d]
            assert 1 <= P["box"][d] <= 256
            if P["dim_len"][d]:
                assert P["box"][d] == 1
                assert P["gdim"][d] == 1 << P["dim_len"][d]
        assert elems == (1 << tb) * mult, "box must hold exactly one tile"
        assert (P["box"][0] * 8) % 16 == 0, "TMA inner box extent must be a multiple of 16 bytes"
        for d in range(1, K_MAX_DIMS):
            assert P["gstride"][d - 1] % 16 == 0 and P["gstride"][d - 1] < (1 << 40)
    assert P["smem"] <= 227 * 1024
    if P["minb"] == 2:  # two CTAs per SM: both fit in shared memory, stages within the 128-register kernel
        assert 2 * (P["smem"] + 3 * 1024) <= 228 * 1024
        assert max(s["r"] for s in P["st"]) <= (3 if P["paired"] else 4)


def _gather_tma(P, src_u64, tiles):
    """Box gather for a batch of tiles -> (len(tiles), box elems) UINT64 element addresses."""
    box = P["box"]
    strides = [1] + [g // 8 for g in P["gstride"]]
    # box linear index -> per-dim offsets
    lin = np.arange(int(np.prod(box)), dtype=np.int64)
    off = np.zeros_like(lin)
    rem = lin.copy()
    for d in range(K_MAX_DIMS):
        b = rem % box[d]
        rem //= box[d]
        off += b * strides[d]
    base = np.zeros(len(tiles), dtype=np.int64)
    for d in range(K_MAX_DIMS):
        if P["dim_len"][d]:
            c = (tiles >> P["dim_src"][d]) & ((1 << P["dim_len"][d]) - 1)
            assert np.all(c + box[d] <= P["gdim"][d])
            base += c * strides[d]
    addr = base[:, None] + off[None, :]
    assert addr.min() >= 0 and addr.max() < src_u64
    return addr


def _block_circuit(v, R, kk, sign):
    """v: (..., 2^R) complex; the block's H (unnormalised) + controlled phases."""
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
                v[..., j] *= np.exp(sign * 2j * np.pi * (j & mask) / (2 * bit))
    return v


def run_pass(P, src, dst, esize, sign, scale_mode, norm_sq):
    """Replay one pass from src (complex128 array) into dst; returns the set of
    output addresses written (as a sorted array) for the bijection check."""
    n, tb, kk = P["n"], P["tb"], P["kk"]
    T = P["num_tiles"]
    tiles = np.arange(T, dtype=np.int64)
    ntile = 1 << tb
    if P["load_mode"] == 1:
        A = src.reshape(T, ntile).copy()
    else:
        mult = esize // 8
        addr = _gather_tma(P, src.size * mult, tiles)
        if mult == 1:
            A = src[addr]
        else:
            assert np.all(addr[:, 0::2] % 2 == 0) and np.all(addr[:, 1::2] == addr[:, 0::2] + 1)
            A = src[addr[:, 0::2] // 2]
    # tile coordinate -> logical bits / output offset
    I_tile = np.zeros(T, dtype=np.uint64)
    out_tile = np.zeros(T, dtype=np.int64)
    for s in P["seg"]:
        v = ((tiles >> s["src"]) & ((1 << s["len"]) - 1)).astype(np.uint64)
        I_tile |= v << np.uint64(s["wire"])
        if s["out_rev"]:
            out_tile += (_brev(v, s["len"]) << np.uint64(s["out"] - s["len"] + 1)).astype(np.int64)
        else:
            out_tile += (v << np.uint64(s["out"])).astype(np.int64)
    inv_root_n = 2.0 ** (-n / 2)
    scale_in = np.sqrt(norm_sq)
    factor = {0: (inv_root_n / scale_in if scale_in > 0 else 0.0), 1: inv_root_n, 2: 1.0,
              3: inv_root_n * inv_root_n}[scale_mode]
    Bbuf = A.copy()
    written = None
    for si, S in enumerate(P["st"]):
        gpos = _groups(P, S)
        R, q, ng = S["r"], S["q"], 1 << len(gpos)
        g = np.arange(ng, dtype=np.int64)
        pb = np.zeros(ng, dtype=np.int64)
        iw = np.zeros(ng, dtype=np.uint64)
        ob = np.zeros(ng, dtype=np.int64)
        for i in range(len(gpos)):
            bit = (g >> i) & 1
            p = gpos[i]
            pb |= bit << p
            iw |= bit.astype(np.uint64) << np.uint64(P["p_wire"][p])
            ob += bit << P["p_out"][p]
        j = np.arange(1 << R, dtype=np.int64)
        pidx = pb[:, None] | (j[None, :] << q)
        assert pidx.max() < ntile and np.array_equal(np.sort(pidx.ravel()), np.arange(ntile))
        v = (A if si == 0 else Bbuf)[:, pidx]  # (T, ng, 2^R)
        if S["cross"]:
            I = I_tile[:, None] | iw[None, :]
            hi = S["wlo"] + R - 1
            rh = (_brev(I, n)) & np.uint64((1 << (n - 1 - hi)) - 1)
            for e in range(R):
                c = S["wlo"] + e
                m = rh.copy()
                lowcut = n - 1 - c - kk
                if lowcut > 0:
                    m &= ~np.uint64((1 << lowcut) - 1)
                beta = (m << np.uint64(c)) & np.uint64((1 << n) - 1)
                tau = np.exp(sign * 2j * np.pi * beta.astype(np.float64) / float(1 << n))
                sel = (j & (1 << e)) != 0
                v[:, :, sel] *= tau[:, :, None]
        v = _block_circuit(v, R, kk, sign)
        if si == len(P["st"]) - 1:
            oj = np.zeros(1 << R, dtype=np.int64)
            for e in range(R):
                oj += ((j >> e) & 1) << P["p_out"][q + e]
            oaddr = out_tile[:, None, None] + ob[None, :, None] + oj[None, None, :]
            assert oaddr.min() >= 0 and oaddr.max() < dst.size
            dst[oaddr] = v * (factor if P["last"] else 1.0)
            written = oaddr.ravel()
        else:
            Bbuf[:, pidx] = v
    return written


def emulate(plan, x, scale_mode=0):
    """Replay every pass of a Plan on input x (numpy complex); returns the output."""
    esize = 8 if plan.dtype == 0 else 16
    info = plan.info()
    N = 1 << info.n_addr
    state = np.asarray(x, dtype=np.complex128).copy()
    work = np.zeros(N, dtype=np.complex128)
    bufs = [state, work]
    norm_sq = float(np.sum(np.abs(state) ** 2))
    first_grid = parse(plan.describe_pass(0))["grid"]
    last = parse(plan.describe_pass(info.passes - 1))
    if info.passes > 1:
        assert last["npartials"] == first_grid, "the last pass sums one norm partial per first-pass CTA"
    for i in range(info.passes):
        P = parse(plan.describe_pass(i))
        check_structure(P, esize)
        src, dst = bufs[P["in_buf"]], bufs[P["out_buf"]]
        src_copy = src.copy()  # in-place passes read the pre-pass values of their own tile
        written = run_pass(P, src_copy, dst, esize, plan.direction, scale_mode, norm_sq)
        assert np.array_equal(np.sort(written), np.arange(N)), "output map of a pass must be a bijection"
    return bufs[0]
