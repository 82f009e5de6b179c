"""Autotuner for the pass planner: per (dtype, n), time a few plan shapes on the
GPU and keep the fastest.

The knobs are the planner options of ``qft_opts``: tile bits (amplitudes per CTA
tile, i.e. how many wires one HBM pass can fuse), coalesce bits (minimum HBM run
length), the widest register stage, and the CTA size of the pass kernel.  A
candidate can win only if its output agrees with the default plan's to the
parity tolerance of its dtype (relative L2).  Results go to a JSON cache
(``autotune_cache.json`` next to this file by default) that ``best_opts`` reads;
``Plan(..., tuned=True)`` and the batched / serving helpers use it.  The
environment variable ``QFTFFT_TUNING_CACHE`` overrides the cache file (a path),
or turns tuned shapes off (``off``: the planner's defaults everywhere).

    python -m paper_2606_18981_gb300.autotune --dtype c64 --nmin 8 --nmax 33
"""
from __future__ import annotations

import json
import os
import statistics

CACHE = os.path.join(os.path.dirname(os.path.abspath(__file__)), "autotune_cache.json")

# candidate plan shapes (qft_opts fields; 0 = planner default).  Complex64
# tiles of 2^12 amplitudes run two CTAs per SM; tile bits 14 is the wide pass
# kernel (2^14-amplitude tiles); double-float tiles of 2^11 pairs with 256
# threads and blocks of <= 3 wires run two CTAs per SM.
_KEYS = ("tile_bits", "coalesce_bits", "max_stage_bits", "threads", "paired", "pass_split")
CANDIDATES = {
    "c64": [dict(zip(_KEYS, c)) for c in (
        (0, 0, 0, 0, 0, 0), (14, 0, 0, 0, 0, 0), (13, 4, 5, 256, 0, 0), (13, 3, 5, 256, 0, 0),
        (13, 5, 5, 256, 0, 0), (13, 4, 4, 512, 0, 0), (12, 4, 4, 256, 0, 0), (12, 3, 4, 256, 0, 0),
        (12, 5, 4, 256, 0, 0), (12, 4, 3, 256, 0, 0), (11, 4, 4, 256, 0, 0), (12, 4, 4, 256, 0, 1),
        (13, 4, 5, 256, 0, 1))],
    "c128": [dict(zip(_KEYS, c)) for c in (
        (0, 0, 0, 0, 0, 0), (12, 3, 4, 256, 0, 0), (11, 3, 4, 256, 0, 0), (12, 2, 4, 256, 0, 0),
        (12, 4, 4, 256, 0, 0), (12, 3, 4, 256, 0, 1), (12, 3, 3, 256, 0, 0), (12, 3, 3, 512, 0, 0),
        (12, 4, 3, 512, 0, 0), (11, 3, 3, 512, 0, 0), (11, 3, 3, 256, 0, 0))],
}

_cache: dict | None = None
ENV = "QFTFFT_TUNING_CACHE"


def cache_path() -> str | None:
    """The cache file in effect: ``$QFTFFT_TUNING_CACHE`` if set (None when it
    says ``off``, ``none``, ``0`` or is empty), else the package's file."""
    v = os.environ.get(ENV)
    if v is None:
        return CACHE
    if v.strip().lower() in ("", "off", "none", "0"):
        return None
    return v


def load_cache(path: str | None = None) -> dict:
    """The tuning cache at ``path`` (default: the file in effect; the package's
    file is read once)."""
    global _cache
    if path is None:
        path = cache_path()
        if path is None:
            return {}
    if path != CACHE:
        return _read(path)
    if _cache is None:
        _cache = _read(CACHE)
    return _cache


def _read(path: str) -> dict:
    try:
        with open(path) as f:
            return json.load(f)
    except (OSError, ValueError):
        return {}


def best_opts(n: int, dtype: str = "c64") -> dict:
    """Plan keyword arguments the cache holds for (dtype, n) ({} if none); zero
    fields (planner defaults) are left out."""
    entry = load_cache().get(dtype, {}).get(str(int(n)))
    if not entry:
        return {}
    return {k: int(v) for k, v in entry["opts"].items() if int(v) != 0}


def _time_plan(q, torch, plan, state, ws, reps):
    torch.cuda.synchronize()  # state was written on the current stream
    s = torch.cuda.Stream()
    plan.execute(state, ws, q.SCALE_STATE, stream=s)
    torch.cuda.synchronize()
    times = []
    for _ in range(reps):
        a = torch.cuda.Event(enable_timing=True)
        b = torch.cuda.Event(enable_timing=True)
        a.record(s)
        plan.execute(state, ws, q.SCALE_STATE, stream=s)
        b.record(s)
        torch.cuda.synchronize()
        times.append(a.elapsed_time(b))
    return statistics.median(times)


def tune(ns, dtype: str = "c64", reps: int = 5, path: str | None = None, verbose: bool = True) -> dict:
    """Time every candidate for each n (exact forward QFT, natural order) and
    store the fastest in the cache.  Needs a CUDA device."""
    import torch

    import paper_2606_18981_gb300 as q

    td = torch.complex64 if dtype == "c64" else torch.complex128
    tol = 2e-6 if dtype == "c64" else 4e-12
    path = path or cache_path() or CACHE
    cache = dict(load_cache(path))
    cache.setdefault(dtype, {})
    for n in ns:
        g = torch.Generator(device="cuda")
        g.manual_seed(n)
        x = torch.randn(1 << n, dtype=td, device="cuda", generator=g)
        ref = None
        results = []
        for cand in CANDIDATES[dtype]:
            try:
                p = q.Plan(n, -1, q.FORWARD, dtype, q.ORDER_NATURAL, **cand)
            except q.QftError:
                continue
            ws = p.alloc_workspace()
            st = x.clone()
            p.execute(st, ws, q.SCALE_STATE)
            torch.cuda.synchronize()
            if ref is None:
                ref = st.clone()
            else:
                err = float(torch.linalg.vector_norm((st - ref).to(torch.complex128)) /
                            torch.linalg.vector_norm(ref.to(torch.complex128)))
                if err > tol:
                    continue
            ms = _time_plan(q, torch, p, x.clone(), ws, reps)
            results.append((ms, cand, p.info().passes))
            del ws, st
        ms, i_best, passes = min((m, i, ps) for i, (m, _, ps) in enumerate(results))
        cand = results[i_best][1]
        cache[dtype][str(n)] = {"opts": dict(cand), "ms": ms, "passes": passes,
                                "candidates": {",".join(str(cand_v) for cand_v in c.values()): m
                                               for m, c, _ in results}}
        if verbose:
            print(f"{dtype} n={n}: best {tuple(cand.values())} {ms:.4f} ms ({passes} passes)", flush=True)
        del x, ref
        torch.cuda.empty_cache()
    with open(path, "w") as f:
        json.dump(cache, f, indent=1, sort_keys=True)
    global _cache
    if path == CACHE:
        _cache = cache
    return cache


if __name__ == "__main__":
    import argparse

    ap = argparse.ArgumentParser()
    ap.add_argument("--dtype", default="c64", choices=["c64", "c128"])
    ap.add_argument("--nmin", type=int, default=8)
    ap.add_argument("--nmax", type=int, default=30)
    ap.add_argument("--reps", type=int, default=5)
    ap.add_argument("--out", default=None)
    a = ap.parse_args()
    tune(range(a.nmin, a.nmax + 1), a.dtype, a.reps, a.out)
