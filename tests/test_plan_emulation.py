"""Planner checks on the CPU: index maps, TMA boxes and the pass arithmetic.

Each plan built by libqftfft is replayed by tests/plan_emulator.py (numpy,
float64) and compared with the oracle; the emulator also asserts that every
index is in bounds and every map is a bijection.  Large plans (up to n = 34)
get the data-free structural checks.  No GPU is needed: plan creation is host
code.
"""
import numpy as np
import pytest

import qft_inputs

q = pytest.importorskip("paper_2606_18981_gb300")
from plan_emulator import check_structure, emulate, parse  # noqa: E402


def rel_l2(a, b):
    return float(np.linalg.norm(np.ravel(a) - np.ravel(b)) / max(np.linalg.norm(np.ravel(b)), 1e-300))


CASES = []
for dt in ("c64", "c128"):
    for order in (q.ORDER_NATURAL, q.ORDER_BITREV):
        for n in (1, 2, 3, 5, 8, 12):
            CASES.append((n, -1, dt, order, 0))
        for n, tbits in ((9, 5), (12, 5), (13, 6), (14, 7), (15, 6), (16, 8), (8, 4), (14, 5)):
            CASES.append((n, -1, dt, order, tbits))
        CASES.append((14, 0, dt, order, 0))
        CASES.append((15, 2, dt, order, 6))
        CASES.append((13, 4, dt, order, 5))


@pytest.mark.parametrize("n,k,dt,order,tbits", CASES)
def test_emulated_plan_matches_oracle(oracle_mod, n, k, dt, order, tbits):
    x = qft_inputs.gaussian(n, seed=1000 + n, normalise=False)
    for direction in (q.FORWARD, q.INVERSE):
        p = q.Plan(n, k, direction, dt, order, tile_bits=tbits)
        for mode in (q.SCALE_STATE, q.SCALE_UNNORM):
            got = emulate(p, x, mode)
            ref, _ = oracle_mod.qft(x, k=k, sign=direction, mode=mode, natural_order=(order == q.ORDER_NATURAL))
            assert rel_l2(got, ref) < 1e-12, (n, k, dt, order, tbits, direction, mode)


@pytest.mark.parametrize("dt", ["c64", "c128"])
@pytest.mark.parametrize("order", [0, 1])
def test_structure_all_sizes(dt, order):
    nmax = 34 if dt == "c64" else 33
    esize = 8 if dt == "c64" else 16
    for n in range(1, nmax + 1):
        for k in (-1, 0, 4):
            p = q.Plan(n, k, q.FORWARD, dt, order)
            inf = p.info()
            assert inf.n_h == n and inf.n_swap == n // 2
            for i in range(inf.passes):
                P = parse(p.describe_pass(i))
                check_structure(P, esize)
                if P["load_mode"] == 0:
                    assert P["run_bits"] >= (2 if dt == "c64" else 1), "HBM runs must be >= 32 bytes"


@pytest.mark.parametrize("n", [3, 6, 7, 10, 13, 16])
@pytest.mark.parametrize("prec", [1, 5])
def test_emulated_tensor_tier_plans(oracle_mod, n, prec):
    """Tensor-core tier plans: one block of <= 6 wires per pass, 12-bit tiles."""
    x = qft_inputs.gaussian(n, seed=300 + n, normalise=False)
    for order in (q.ORDER_NATURAL, q.ORDER_BITREV):
        p = q.Plan(n, -1 if n % 2 else 3, q.FORWARD, "c64", order, precision=prec)
        for i in range(p.info().passes):
            P = parse(p.describe_pass(i))
            assert P["nstages"] == 1 and P["st"][0]["r"] <= 6 and P["tb"] - P["st"][0]["r"] <= 8
        got = emulate(p, x, q.SCALE_STATE)
        ref, _ = oracle_mod.qft(x, k=p.k, sign=-1, mode=0, natural_order=(order == q.ORDER_NATURAL))
        assert rel_l2(got, ref) < 1e-12


@pytest.mark.parametrize("f,n", [(4, 9), (4, 13), (5, 13), (5, 16), (7, 7), (7, 12), (7, 13), (7, 14), (7, 16),
                                 (7, 20), (7, 21)])
@pytest.mark.parametrize("prec", [1, 5])
def test_emulated_tensor_tier_block_widths(oracle_mod, f, n, prec):
    """Tier plans of fused blocks of <= f wires (max_stage_bits = f): every pass
    is one block of <= f wires, f = 7 plans do run 7-wire blocks where n
    allows, and the replayed plan matches the oracle in both orders."""
    x = qft_inputs.gaussian(n, seed=400 + n, normalise=False)
    for order in (q.ORDER_NATURAL, q.ORDER_BITREV):
        p = q.Plan(n, -1 if n % 2 else 5, q.FORWARD, "c64", order, precision=prec, max_stage_bits=f)
        rs = []
        for i in range(p.info().passes):
            P = parse(p.describe_pass(i))
            assert P["nstages"] == 1 and P["st"][0]["r"] <= f
            assert P["tb"] == (11 if f in (4, 7) else 12) or P["tb"] == n
            rs.append(P["st"][0]["r"])
        if f == 7 and n in (13, 14, 20, 21):
            assert 7 in rs
        got = emulate(p, x, q.SCALE_STATE)
        ref, _ = oracle_mod.qft(x, k=p.k, sign=-1, mode=0, natural_order=(order == q.ORDER_NATURAL))
        assert rel_l2(got, ref) < 1e-12


def test_tensor_tier_block_width_range():
    for f in (1, 3, 8):
        with pytest.raises(q.QftError) as e:
            q.Plan(20, precision=q.PREC_FP16X3, max_stage_bits=f)
        assert e.value.code == q.ERR_BAD_ARG


def test_tensor_tier_rejects_complex128():
    with pytest.raises(q.QftError) as e:
        q.Plan(20, dtype="c128", precision=q.PREC_FP16X3)
    assert e.value.code == q.ERR_UNSUPPORTED


def test_plan_counters_table2():
    """Pre-fusion counters of the plan reproduce Table 2 for n = 22."""
    for k, cnt in ((21, 231), (16, 216), (12, 186), (10, 165), (8, 140), (6, 111), (4, 78)):
        assert q.Plan(22, k).info().n_cp == cnt


def test_plan_argument_errors():
    with pytest.raises(q.QftError) as e:
        q.Plan(0)
    assert e.value.code == q.ERR_BAD_ARG
    with pytest.raises(q.QftError):
        q.Plan(35, dtype="c64")
    with pytest.raises(q.QftError):
        q.Plan(34, dtype="c128")
    with pytest.raises(q.QftError):
        q.Plan(10, direction=2)
    with pytest.raises(ValueError):
        q.Plan(10, dtype="c32")


def test_variant_plans_use_the_intended_kernels():
    """The planner selects two CTAs per SM for 2^12-amplitude complex64 tiles;
    the removed paired stages are refused."""
    import plan_emulator as pe
    descs = lambda p: [pe.parse(p.describe_pass(i)) for i in range(p.info().passes)]  # noqa: E731
    d = descs(q.Plan(26, -1, q.FORWARD, "c64", 0, tile_bits=12))
    assert all(P["minb"] == 2 and not P["paired"] and not P["wide"] for P in d)
    with pytest.raises(q.QftError) as e:
        q.Plan(26, -1, q.FORWARD, "c64", 0, paired=1)
    assert e.value.code == q.ERR_UNSUPPORTED


@pytest.mark.parametrize("dt", ["c64", "c128"])
@pytest.mark.parametrize("n,tbits", [(14, 6), (17, 7), (16, 6), (19, 8), (13, 5)])
def test_pass_split_plans(oracle_mod, dt, n, tbits):
    """pass_split = 1 (left-over wires on the middle passes): same transform,
    first and last passes with at least as many batch wires as the default."""
    x = qft_inputs.gaussian(n, seed=3000 + n, normalise=False)
    p0 = q.Plan(n, -1, q.FORWARD, dt, q.ORDER_NATURAL, tile_bits=tbits)
    p1 = q.Plan(n, -1, q.FORWARD, dt, q.ORDER_NATURAL, tile_bits=tbits, pass_split=1)
    i0, i1 = p0.info(), p1.info()
    assert i0.passes == i1.passes
    assert sum(list(i1.wires_per_pass)[:i1.passes]) == n
    if i1.passes >= 3:
        assert i1.wires_per_pass[0] <= i0.wires_per_pass[0]
    for i in range(i1.passes):
        check_structure(parse(p1.describe_pass(i)), 8 if dt == "c64" else 16)
    got = emulate(p1, x, q.SCALE_STATE)
    ref, _ = oracle_mod.qft(x, k=-1, sign=q.FORWARD, mode=q.SCALE_STATE, natural_order=True)
    assert rel_l2(got, ref) < 1e-12


def subset_reference(oracle_mod, x, n_addr, w0, m, k, sign, mode, natural):
    """The oracle's m-wire transform applied to every sub-vector along index
    bits [w0, w0 + m) (the other bits fixed)."""
    a = np.asarray(x, dtype=np.complex128).reshape(1 << (n_addr - w0 - m), 1 << m, 1 << w0)
    out = np.empty_like(a)
    for hi in range(a.shape[0]):
        for lo in range(a.shape[2]):
            out[hi, :, lo], _ = oracle_mod.qft(a[hi, :, lo].copy(), k=k, sign=sign, mode=mode, natural_order=natural)
    return out.ravel()


SUBSET_CASES = []
for dt in ("c64", "c128"):
    for order in (q.ORDER_NATURAL, q.ORDER_BITREV):
        for n_addr, w0, m, tbits in ((10, 0, 6, 0), (12, 0, 8, 0), (11, 3, 5, 0), (12, 4, 8, 0), (14, 5, 9, 6),
                                     (15, 4, 11, 7), (13, 6, 7, 0), (12, 2, 6, 0), (15, 0, 11, 6),
                                     (16, 0, 13, 7)):
            SUBSET_CASES.append((n_addr, w0, m, dt, order, tbits))


@pytest.mark.parametrize("n_addr,w0,m,dt,order,tbits", SUBSET_CASES)
def test_subset_plans_match_oracle(oracle_mod, n_addr, w0, m, dt, order, tbits):
    """QFTs on qubit subsets: every sub-vector along bits [w0, w0 + m) transformed
    independently (single-pass and multi-pass plans, both orders)."""
    x = qft_inputs.gaussian(n_addr, seed=5000 + n_addr + w0, normalise=False)
    for direction, k in ((q.FORWARD, -1), (q.INVERSE, 3)):
        p = q.Plan(m, k, direction, dt, order, tile_bits=tbits, n_addr=n_addr, w0=w0)
        inf = p.info()
        assert inf.n_addr == n_addr and inf.w0 == w0 and inf.n == m
        for i in range(inf.passes):
            check_structure(parse(p.describe_pass(i)), 8 if dt == "c64" else 16)
        got = emulate(p, x, q.SCALE_UNNORM)
        ref = subset_reference(oracle_mod, x, n_addr, w0, m, k, direction, q.SCALE_UNNORM,
                               order == q.ORDER_NATURAL)
        assert rel_l2(got, ref) < 1e-12, (n_addr, w0, m, dt, order, direction)


def test_subset_plan_rejections():
    with pytest.raises(q.QftError):
        q.Plan(20, -1, q.FORWARD, "c64", n_addr=22, w0=1)  # multi-pass with fewer than 4 low batch bits
    with pytest.raises(q.QftError):
        q.Plan(8, -1, q.FORWARD, "c64", n_addr=10, w0=4)   # does not fit the array
    with pytest.raises(q.QftError):
        q.Plan(8, -1, q.FORWARD, "c64", n_addr=12, w0=2, precision=q.PREC_FP16X3)


@pytest.mark.parametrize("dt", ["c64", "c128"])
@pytest.mark.parametrize("order", [0, 1])
@pytest.mark.parametrize("n", [13, 14, 15, 16])
def test_headline_plan_shape_scaled_down(oracle_mod, dt, order, n):
    """The plan shape the planner uses for large complex64 states (tiles of
    TB bits with cmin coalescing bits, left-over wires on the middle passes,
    blocks of <= 4 wires), scaled down to TB = 6, cmin = 2, blocks <= 2 so
    that natural order takes the same 4 passes at emulation sizes; both
    directions, against the oracle."""
    x = qft_inputs.gaussian(n, seed=4000 + n, normalise=False)
    for direction in (q.FORWARD, q.INVERSE):
        p = q.Plan(n, -1, direction, dt, order, tile_bits=6, coalesce_bits=2, max_stage_bits=2, pass_split=1)
        inf = p.info()
        # natural order: 4 passes of <= TB - cmin wires; bit-reversed order: the
        # last pass (contiguous, no batch wires) may take a whole tile
        assert inf.passes == 4 if order == q.ORDER_NATURAL else inf.passes == 1 + -(-(n - 6) // 4)
        assert sum(list(inf.wires_per_pass)[:inf.passes]) == n
        for i in range(inf.passes):
            check_structure(parse(p.describe_pass(i)), 8 if dt == "c64" else 16)
        got = emulate(p, x, q.SCALE_STATE)
        ref, _ = oracle_mod.qft(x, k=-1, sign=direction, mode=q.SCALE_STATE, natural_order=(order == q.ORDER_NATURAL))
        assert rel_l2(got, ref) < 1e-12, (n, dt, order, direction)


def test_default_large_complex64_plans_are_the_tuned_shape():
    """Default complex64 plans of 2^27 amplitudes and more: natural order runs
    on wide passes (2^14-amplitude tiles, ceil(n / 10) passes); bit-reversed
    order keeps the shape measured fastest on GB300 for the 2^12 / 2^13-tile
    kernel: 2^12-amplitude tiles with 4 coalescing bits, blocks of <= 4 wires,
    two CTAs per SM."""
    for n in (27, 28, 30, 32):
        p = q.Plan(n, -1, q.FORWARD, "c64", q.ORDER_NATURAL)
        inf = p.info()
        ds = [parse(p.describe_pass(i)) for i in range(inf.passes)]
        assert inf.passes == (n + 9) // 10
        assert all(P["wide"] == 1 and P["tb"] == 14 for P in ds)
        assert all(P["run_bits"] >= 4 for P in ds)  # >= 128-byte HBM runs
        p = q.Plan(n, -1, q.FORWARD, "c64", q.ORDER_BITREV)
        ds = [parse(p.describe_pass(i)) for i in range(p.info().passes)]
        assert all(P["wide"] == 0 and P["tb"] == 12 and P["minb"] == 2 for P in ds)
        assert all(s["r"] <= 4 for P in ds for s in P["st"])
    w = list(q.Plan(30, -1, q.FORWARD, "c64", q.ORDER_NATURAL).info().wires_per_pass)[:3]
    assert w == [10, 10, 10]


@pytest.mark.parametrize("dt", ["c64", "c128"])
@pytest.mark.parametrize("order", [0, 1])
@pytest.mark.parametrize("n", [9, 13, 16])
def test_512_thread_plans_match_oracle(oracle_mod, dt, order, n):
    """Plans for 512-thread CTAs: blocks of <= 4 wires (complex64) or <= 3
    (double-float complex128), replayed against the oracle."""
    x = qft_inputs.gaussian(n, seed=5000 + n, normalise=False)
    p = q.Plan(n, -1, q.FORWARD, dt, order, threads=512)
    rmax = 4 if dt == "c64" else 3
    for i in range(p.info().passes):
        P = parse(p.describe_pass(i))
        check_structure(P, 8 if dt == "c64" else 16)
        assert all(s["r"] <= rmax for s in P["st"])
    got = emulate(p, x, q.SCALE_UNITARY)
    ref, _ = oracle_mod.qft(x, k=-1, sign=q.FORWARD, mode=q.SCALE_UNITARY, natural_order=(order == q.ORDER_NATURAL))
    assert rel_l2(got, ref) < 1e-12


@pytest.mark.parametrize("order", [0, 1])
@pytest.mark.parametrize("n", [9, 14, 19])
def test_df_two_cta_plans_match_oracle(oracle_mod, order, n):
    """Double-float plans for two 256-thread CTAs per SM: 2^11-pair tiles,
    blocks of <= 3 wires, the stage-minimising pass widths; replayed against
    the oracle."""
    x = qft_inputs.gaussian(n, seed=5100 + n, normalise=False)
    p = q.Plan(n, -1, q.FORWARD, "c128", order, threads=256, tile_bits=11, max_stage_bits=3)
    for i in range(p.info().passes):
        P = parse(p.describe_pass(i))
        check_structure(P, 16)
        assert P["minb"] == 2 and P["tb"] <= 11 and all(s["r"] <= 3 for s in P["st"])
    got = emulate(p, x, q.SCALE_UNITARY)
    ref, _ = oracle_mod.qft(x, k=-1, sign=q.FORWARD, mode=q.SCALE_UNITARY, natural_order=(order == q.ORDER_NATURAL))
    assert rel_l2(got, ref) < 1e-12


def test_default_double_float_plan_shapes():
    """Default double-float complex128 plans from n = 21 (512 threads, blocks of
    <= 3 wires): the fewest register stages in all, and one coalescing bit less
    only where that saves a pass without adding a stage (n = 28 alone up to 33)."""
    expect = {21: (3, 7), 24: (3, 8), 27: (3, 9), 28: (3, 10), 29: (4, 10), 30: (4, 10), 33: (4, 11)}
    for n in range(21, 34):
        p = q.Plan(n, -1, q.FORWARD, "c128", q.ORDER_NATURAL)
        ds = [parse(p.describe_pass(i)) for i in range(p.info().passes)]
        for P in ds:
            check_structure(P, 16)
            assert all(s["r"] <= 3 for s in P["st"][:P["nstages"]])
        stages = sum(P["nstages"] for P in ds)
        # every pass but the last (the contiguous one) keeps >= 2 coalescing bits (64-byte runs)
        assert all(P["run_bits"] >= 2 for P in ds), n
        assert min(P["run_bits"] for P in ds[:-1]) == (2 if n == 28 else 3), n
        assert stages >= -(-n // 3)  # blocks of <= 3 wires
        if n in expect:
            assert (len(ds), stages) == expect[n], (n, len(ds), stages)


def test_plan_info_fused_blocks():
    """Sec. 3.1's plan record: the fused blocks (register stages of all passes)
    cover every wire once, and max_fused_size is the widest block."""
    for n, dt in ((10, "c64"), (20, "c64"), (30, "c64"), (33, "c64"), (22, "c128"), (30, "c128")):
        p = q.Plan(n, -1, q.FORWARD, dt)
        info = p.info()
        recs = [parse(p.describe_pass(i)) for i in range(info.passes)]
        rs = [s["r"] for P in recs for s in P["st"]]
        assert info.fused_blocks == len(rs) == sum(info.stages_per_pass[:info.passes])
        assert info.max_fused_size == max(rs) and sum(rs) == n
