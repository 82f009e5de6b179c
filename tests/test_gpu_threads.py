"""Kernel launches from several host threads (the serving loop's worker and the
caller, or any multi-threaded user): a kernel's dynamic shared-memory limit is
one attribute per device, so a thread that launches the same kernel with a
smaller tile must not lower it under another thread's larger launch."""
import threading

import numpy as np
import pytest

import qft_inputs

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
q = pytest.importorskip("paper_2606_18981_gb300")


def test_two_threads_same_kernel_different_tiles(oracle_mod):
    n = 16
    x = torch.from_numpy(qft_inputs.gaussian(n, seed=9)).to(torch.complex64).cuda()
    ref, _ = oracle_mod.qft(x.cpu().numpy().astype(np.complex128), -1, -1, oracle_mod.SCALE_STATE, True)
    big = q.Plan(n, -1, q.FORWARD, "c64", tile_bits=12, coalesce_bits=4, max_stage_bits=4)    # 3 x 32 KiB tiles
    small = q.Plan(n, -1, q.FORWARD, "c64", tile_bits=10, coalesce_bits=3, max_stage_bits=4)  # 3 x 8 KiB tiles
    wb, ws = big.alloc_workspace(), small.alloc_workspace()

    def run(p, w):
        st = x.clone()
        p.execute(st, w, q.SCALE_STATE)
        torch.cuda.synchronize()
        assert p.status(w) == 0
        got = st.cpu().numpy().astype(np.complex128)
        assert np.linalg.norm(got - ref) / np.linalg.norm(ref) <= 2e-6

    run(big, wb)
    errors = []

    def worker():
        try:
            run(small, ws)
        except Exception as e:  # reported on the main thread
            errors.append(e)

    t = threading.Thread(target=worker)
    t.start()
    t.join()
    assert not errors, errors
    run(big, wb)  # the larger launch still has its shared memory
