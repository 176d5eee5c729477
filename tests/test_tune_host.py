"""Host logic of the tile autotuner (no GPU): workload buckets, the JSON cache, and that a cached
choice is installed without tuning while a miss tunes."""
import json

import pytest

from paper_2104_04582_gb300 import fewsum as F
from paper_2104_04582_gb300 import tune


def test_buckets_round_slots_and_samples_up():
    assert tune.bucket(F.FEW_MIXED, 1281, 3155760) == "mixed:2048:4194304"
    assert tune.bucket(F.FEW_MIXED, 1024, 4 ** 10) == "mixed:1024:1048576"
    assert tune.bucket(F.FEW_MIXED, 1025, 4 ** 10 + 1) == "mixed:2048:4194304"
    assert tune.bucket(F.FEW_FP64, 1, 1) == "fp64:1:1"
    assert tune.bucket(F.FEW_FP64, 0, 0) == "fp64:1:1"


def test_cache_roundtrip(tmp_path):
    p = str(tmp_path / "sub" / "tiles.json")
    assert tune._load(p) == {}
    tune._save(p, {"a": {"R": 4}})
    assert tune._load(p) == {"a": {"R": 4}}
    assert not (tmp_path / "sub" / "tiles.json.tmp").exists()


def test_cached_choice_is_installed_without_tuning(tmp_path, monkeypatch):
    p = str(tmp_path / "tiles.json")
    key = tune.bucket(F.FEW_MIXED, 1281, 3155760)
    with open(p, "w") as fh:
        json.dump({key: {"R": 8, "threads": 128, "stage_slots": 512, "ms": 1.0}}, fh)
    installed = []
    monkeypatch.setattr(tune, "install", lambda h, prec, c: installed.append((prec, c)))
    monkeypatch.setattr(tune, "tune", lambda *a, **k: pytest.fail("tuned despite a cache hit"))
    choice, tuned = tune.ensure(0, None, F.FEW_MIXED, 1281, 3155760, p)
    assert (choice, tuned) == ((8, 128, 512), False)
    assert installed == [(F.FEW_MIXED, (8, 128, 512))]


def test_a_miss_or_an_old_entry_tunes(tmp_path, monkeypatch):
    p = str(tmp_path / "tiles.json")
    key = tune.bucket(F.FEW_FP64, 500, 10 ** 5)
    with open(p, "w") as fh:  # an entry without stage_slots (an older tile format) is a miss
        json.dump({key: {"R": 1, "threads": 256, "ms": 1.0}}, fh)
    calls = []
    monkeypatch.setattr(tune, "install", lambda *a: pytest.fail("installed an old entry"))

    def fake_tune(h, run, prec, n_slots, n_samples, **kw):
        calls.append((prec, n_slots, n_samples, kw.get("cache_path")))
        return (2, 256, 256), {}
    monkeypatch.setattr(tune, "tune", fake_tune)
    choice, tuned = tune.ensure(0, None, F.FEW_FP64, 500, 10 ** 5, p)
    assert (choice, tuned) == ((2, 256, 256), True)
    assert calls == [(F.FEW_FP64, 500, 10 ** 5, p)]


def test_candidates_are_valid_tiles():
    for prec, cands in tune.CANDIDATES.items():
        assert cands and len(set(cands)) == len(cands)
        for R, T, S in cands:
            assert T in (128, 256) and S % 16 == 0 and 16 <= S <= 4096
            assert R in ((1, 2) if prec == F.FEW_FP64 else (2, 4, 8))
