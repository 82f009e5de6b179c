"""Autotuner cache handling (CPU) and a small tuning run (GPU)."""
import json

import pytest

q = pytest.importorskip("paper_2606_18981_gb300")
from paper_2606_18981_gb300 import autotune  # noqa: E402


def test_best_opts_reads_cache(tmp_path, monkeypatch):
    path = tmp_path / "cache.json"
    path.write_text(json.dumps({"c64": {"20": {"opts": {"tile_bits": 12, "coalesce_bits": 4, "max_stage_bits": 4,
                                                       "threads": 512}}}}))
    monkeypatch.setattr(autotune, "CACHE", str(path))
    monkeypatch.setattr(autotune, "_cache", None)
    assert autotune.best_opts(20, "c64") == {"tile_bits": 12, "coalesce_bits": 4, "max_stage_bits": 4, "threads": 512}
    assert autotune.best_opts(21, "c64") == {}
    p = q.Plan(20, tuned=True)
    assert list(p.info().tile_bits)[0] == 12


def test_cache_override_from_the_environment(tmp_path, monkeypatch):
    path = tmp_path / "mine.json"
    path.write_text(json.dumps({"c64": {"18": {"opts": {"tile_bits": 11, "coalesce_bits": 3}}}}))
    monkeypatch.setenv(autotune.ENV, str(path))
    assert autotune.cache_path() == str(path)
    assert autotune.best_opts(18, "c64") == {"tile_bits": 11, "coalesce_bits": 3}
    assert list(q.Plan(18, tuned=True).info().tile_bits)[0] == 11
    monkeypatch.setenv(autotune.ENV, "off")
    assert autotune.cache_path() is None and autotune.best_opts(30, "c64") == {}
    monkeypatch.delenv(autotune.ENV)
    assert autotune.cache_path() == autotune.CACHE


def test_every_candidate_is_a_valid_plan():
    for dt, cands in autotune.CANDIDATES.items():
        for cand in cands:
            for n in (8, 14, 20, 26, 30):
                q.Plan(n, -1, q.FORWARD, dt, **cand)


@pytest.mark.gpu
def test_tune_small_range(tmp_path):
    cache = autotune.tune([14, 18], "c64", reps=2, path=str(tmp_path / "c.json"), verbose=False)
    assert set(cache["c64"]) == {"14", "18"}
    for e in cache["c64"].values():
        assert e["ms"] > 0 and e["passes"] >= 1
