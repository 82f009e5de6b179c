"""The N > 1 bench path (independent replicas, one per GPU): whole-job time is
the slowest rank's and the rate counts every rank's work.  Runs as two gloo
ranks on CPU."""
import os
import socket
import sys

import pytest

torch = pytest.importorskip("torch")
import torch.distributed as dist  # noqa: E402
import torch.multiprocessing as mp  # noqa: E402

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank(rank, world, port, out):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    sys.path.insert(0, ROOT)
    import bench

    ms, rate = bench.whole_job_rate(10.0 + 5.0 * rank, 1000, world)
    dist.barrier()
    out[rank] = (ms, rate)
    dist.destroy_process_group()


def test_whole_job_rate_two_gloo_ranks():
    port = _free_port()
    with mp.Manager() as m:
        out = m.dict()
        mp.spawn(_rank, args=(2, port, out), nprocs=2, join=True)
        res = dict(out)
    for r in (0, 1):
        ms, rate = res[r]
        assert ms == pytest.approx(15.0)  # the slower rank's time, on every rank
        assert rate == pytest.approx(2 * 1000 / 0.015)  # both ranks' units


def test_whole_job_rate_single_rank():
    sys.path.insert(0, ROOT)
    import bench

    ms, rate = bench.whole_job_rate(4.0, 1 << 20, 1)
    assert ms == 4.0 and rate == pytest.approx((1 << 20) / 0.004)


def test_clock_record_rejection_rules():
    """The bench re-measures once when its timed region saw a hardware or
    thermal slowdown, or SM clocks far below maximum with no reason given;
    the power cap alone is kept."""
    sys.path.insert(0, ROOT)
    import bench

    ok = {"sm_mhz": 2070.0, "sm_max_mhz": 2070.0, "reasons": []}
    assert not bench.clocks_rejected(ok)
    assert not bench.clocks_rejected({**ok, "sm_mhz": 1440.0, "reasons": ["sw_power_cap"]})
    for r in ("hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown"):
        assert bench.clocks_rejected({**ok, "reasons": [r]})
    assert bench.clocks_rejected({**ok, "sm_mhz": 990.0})
    assert not bench.clocks_rejected({"sm_mhz": None, "sm_max_mhz": None, "reasons": ["unsampled"]})


def test_copy_overlap_of_the_end_to_end_pipeline():
    """The e2e record's copy timeline: mean copy times and how long each input
    copy ran alongside the previous step's read-back (serial copies give 0)."""
    sys.path.insert(0, ROOT)
    import bench

    serial = [(0, 40, 50, 95), (95, 135, 145, 190), (190, 230, 240, 285)]
    r = bench.copy_overlap(serial)
    assert r["h2d_ms_mean"] == 40 and r["d2h_ms_mean"] == 45 and r["h2d_next_during_d2h_ms_mean"] == 0
    overlapped = [(0, 41, 50, 105), (41, 95, 105, 160), (95, 150, 160, 215)]
    r = bench.copy_overlap(overlapped)
    # step 2's input copy [41, 95] against step 1's read-back [50, 105]: 45 ms; then [95, 150] vs [105, 160]: 45
    assert r["h2d_next_during_d2h_ms_mean"] == 45
