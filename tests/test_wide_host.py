"""CPU checks of the wide pass kernel (csrc/qft_wide.cuh) before it runs on a
GPU: its index maps exhaustively (tests/native/wide_index_check.cu: thread
maps, shared-memory layouts, bank conflicts, store runs), the planner's wide
pass records (structure, pass counts), and a float64 numpy replay of the
kernel's data flow against the oracle (tests/wide_emulator.py)."""
import os
import shutil
import subprocess

import numpy as np
import pytest

import qft_inputs

q = pytest.importorskip("paper_2606_18981_gb300")
from plan_emulator import check_structure, parse  # noqa: E402
from wide_emulator import emulate_wide, thread_maps  # noqa: E402

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def index_exe(tmp_path_factory):
    nvcc = next((c for c in (shutil.which("nvcc"), "/usr/local/cuda/bin/nvcc") if c and os.path.exists(c)), None)
    if nvcc is None:
        pytest.skip("nvcc not available")
    exe = str(tmp_path_factory.mktemp("wide") / "wide_index_check")
    src = os.path.join(ROOT, "tests", "native", "wide_index_check.cu")
    inc = [f"-I{os.path.join(ROOT, 'paper_2606_18981_gb300', 'csrc')}", f"-I{os.path.join(ROOT, 'include')}"]
    r = subprocess.run([nvcc, "-std=c++17", "-O2", "--expt-relaxed-constexpr", *inc, "-o", exe, src],
                       capture_output=True, text=True)
    assert r.returncode == 0, r.stdout + r.stderr
    return exe


def test_index_maps_and_bank_conflicts(index_exe):
    r = subprocess.run([index_exe], capture_output=True, text=True, timeout=300)
    print(r.stdout)
    assert r.returncode == 0 and "ALL OK" in r.stdout, r.stdout + r.stderr


def wide_ns():
    return [n for n in range(14, 35) if n not in (21, 22)]


def test_wide_plan_records():
    """Every wide plan: ceil(n/10) passes (2 at least), records that pass the
    structural checks, and the default planner picks wide passes from n = 23."""
    for n in wide_ns():
        for k in (-1, 0, 5):
            p = q.Plan(n, k, q.FORWARD, "c64", q.ORDER_NATURAL, tile_bits=14)
            info = p.info()
            assert info.passes == max(2, (n + 9) // 10), n
            for i in range(info.passes):
                P = parse(p.describe_pass(i))
                assert P["wide"] == 1 and P["tb"] == 14 and P["nstages"] == 2
                check_structure(P, 8)
        d = q.Plan(n, -1, q.FORWARD, "c64")
        assert all(parse(d.describe_pass(i))["wide"] == int(n >= 23) for i in range(d.info().passes)), n
    for n in (21, 22):  # no wide shape: the default planner keeps the 2^13 / 2^12 tiles
        with pytest.raises(q.QftError):
            q.Plan(n, -1, q.FORWARD, "c64", q.ORDER_NATURAL, tile_bits=14)
        d = q.Plan(n, -1, q.FORWARD, "c64")
        assert all(parse(d.describe_pass(i))["wide"] == 0 for i in range(d.info().passes))


@pytest.mark.parametrize("n", [14, 15, 16, 17, 18, 19, 20])
def test_wide_dataflow_matches_oracle(oracle_mod, index_exe, n):
    maps = thread_maps(index_exe)
    x = qft_inputs.gaussian(n, seed=50 + n, normalise=False)
    for k in (-1, 0, 3):
        for direction in (q.FORWARD, q.INVERSE):
            p = q.Plan(n, k, direction, "c64", q.ORDER_NATURAL, tile_bits=14)
            for mode in (q.SCALE_STATE, q.SCALE_UNNORM, q.SCALE_INV_N):
                got = emulate_wide(p, x, maps, mode)
                ref, _ = oracle_mod.qft(x, k=k, sign=direction, mode=mode, natural_order=True)
                err = np.linalg.norm(got - ref) / np.linalg.norm(ref)
                assert err < 1e-12, (n, k, direction, mode, err)


def _subset_reference(oracle_mod, x, n_addr, m, k, sign, mode):
    """The oracle's m-wire transform of every length-2^m run of x (index bits
    m .. n_addr-1 fixed)."""
    a = np.asarray(x, dtype=np.complex128).reshape(1 << (n_addr - m), 1 << m)
    return np.concatenate([oracle_mod.qft(r.copy(), k=k, sign=sign, mode=mode, natural_order=True)[0] for r in a])


@pytest.mark.parametrize("n_addr,m", [(17, 16), (18, 16), (19, 17), (20, 18)])
def test_wide_subset_plans_match_oracle(oracle_mod, index_exe, n_addr, m):
    """Wide passes for a transform on the low m of n_addr index bits: the upper
    bits keep their addresses in every layout (a batch index, no phases)."""
    maps = thread_maps(index_exe)
    x = qft_inputs.gaussian(n_addr, seed=70 + n_addr + m, normalise=False)
    for k, direction in ((-1, q.FORWARD), (3, q.INVERSE)):
        p = q.Plan(m, k, direction, "c64", q.ORDER_NATURAL, tile_bits=14, n_addr=n_addr)
        assert p.info().passes == max(2, (m + 9) // 10)
        for mode in (q.SCALE_UNNORM, q.SCALE_INV_N):
            got = emulate_wide(p, x, maps, mode)
            ref = _subset_reference(oracle_mod, x, n_addr, m, k, direction, mode)
            err = np.linalg.norm(got - ref) / np.linalg.norm(ref)
            assert err < 1e-12, (n_addr, m, k, direction, mode, err)


def test_default_subset_plans_take_wide_passes():
    """Default complex64 natural-order plans on the low bits of an array of
    >= 2^23 amplitudes run on wide passes; other subsets, and transforms of 14 or
    15 wires under further index bits (six TMA dimensions), keep the 2^12 / 2^13 tiles."""
    for n_addr, m in ((23, 16), (28, 24), (30, 20), (34, 30)):
        d = q.Plan(m, -1, q.FORWARD, "c64", n_addr=n_addr)
        assert d.info().passes == max(2, (m + 9) // 10)
        assert all(parse(d.describe_pass(i))["wide"] == 1 for i in range(d.info().passes)), (n_addr, m)
        for i in range(d.info().passes):
            check_structure(parse(d.describe_pass(i)), 8)
    for args in ((20, dict(n_addr=22)), (24, dict(n_addr=28, w0=4)), (13, dict(n_addr=28)), (14, dict(n_addr=28))):
        d = q.Plan(args[0], -1, q.FORWARD, "c64", **args[1])
        assert all(parse(d.describe_pass(i))["wide"] == 0 for i in range(d.info().passes))


def test_subset_plans_on_large_arrays_are_well_formed():
    """Every default complex64 plan for the low m bits of a 2^23..2^34 array:
    well-formed pass records (the address maps are permutations of all n_addr
    bits, the TMA boxes fit); wide passes, ceil(m / 10) of them, except where
    the upper wires would need a sixth TMA dimension (m = 14, 15, 21..23, 31)."""
    for n_addr in range(23, 35):
        for m in range(14, n_addr + 1):
            p = q.Plan(m, -1, q.FORWARD, "c64", n_addr=n_addr)
            ds = [parse(p.describe_pass(i)) for i in range(p.info().passes)]
            for P in ds:
                check_structure(P, 8)
            if all(P["wide"] == 1 for P in ds):
                assert p.info().passes == max(2, (m + 9) // 10), (n_addr, m)
            else:
                assert m in (14, 15, 21, 22, 23, 31), (n_addr, m)
