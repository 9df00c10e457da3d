"""Host logic of the autotuner: cache keys and the JSON cache (no GPU needed)."""
import json

import pytest

pytest.importorskip("torch")

from paper_2103_00405_gb300 import autotune as A
from paper_2103_00405_gb300 import workloads as W


@pytest.fixture
def fake_gpu(monkeypatch, tmp_path):
    monkeypatch.setattr(A, "_gpu", lambda: "GB300-test")
    monkeypatch.setenv("RANDTIME_AUTOTUNE_CACHE", str(tmp_path / "cache" / "autotune.json"))
    return tmp_path


def test_batch_key_depends_on_the_size_multiset_not_the_order(fake_gpu):
    specs = [W.random_mass_action(3, m, seed=m) for m in (5, 40, 300)]
    k1 = A.batch_key(specs, 1)
    k2 = A.batch_key(list(reversed(specs)), 1)
    assert k1 == k2
    assert A.batch_key(specs, 2) != k1
    assert A.batch_key(specs[:2], 1) != k1
    assert "GB300-test" in k1


def test_single_key_names_the_shape(fake_gpu):
    spec = W.random_mass_action(7, 90, seed=1)
    assert A.single_key(spec, 64) == "single|GB300-test|M=90|N=7|traj=64"


def test_cache_round_trip_and_cached_choice_is_returned_without_timing(fake_gpu, monkeypatch):
    specs = [W.random_mass_action(3, m, seed=m) for m in (5, 40)]
    key = A.batch_key(specs, 1)
    A._store(key, {"policy": {"thread_max_m": 4, "warp_max_m": 64, "block_threads": 256}})
    A._store("other", {"policy": {}})
    with open(A.cache_path()) as f:
        data = json.load(f)
    assert set(data) == {key, "other"}

    def no_timing(*a, **k):
        raise AssertionError("a cached choice must not be re-timed")

    monkeypatch.setattr(A, "_time", no_timing)
    got = A.tune_batch(specs, None, None, 1)
    assert got == {"thread_max_m": 4, "warp_max_m": 64, "block_threads": 256}


def test_candidates_respect_the_library_limits():
    for c in A.BATCH_CANDIDATES:
        assert 0 <= c["thread_max_m"] <= 8
        assert 0 <= c["warp_max_m"] <= 256
        assert c["block_threads"] in (128, 256, 512)
