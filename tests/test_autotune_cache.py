"""Autotuner bookkeeping on the CPU: cache keys, storage and the choice rule."""
from paper_2406_02720_b300 import autotune


def test_cache_key_buckets_and_sizes():
    a = autotune.cache_key("B300", 1_000_000, [(640, 360), (1920, 1080), (640, 360)], True)
    b = autotune.cache_key("B300", 1_048_000, [(1920, 1080), (640, 360), (640, 360)], True)
    assert a == b                                   # same bucket, same multiset of sizes
    assert autotune.cache_key("B300", 3_000_000, [(640, 360)], True) != a
    assert autotune.cache_key("B300", 1_000_000, [(640, 360), (1920, 1080), (640, 360)], False) != a
    assert autotune.n_bucket(3_000_000) == 1 << 22 and autotune.n_bucket(1) == 1


def test_store_load_and_pick(tmp_path):
    path = str(tmp_path / "tune.json")
    timings = [([16, 16], 256, 3.0), ([8, 8], 64, 2.5), ([32, 8], 128, 2.7)]
    assert autotune.pick(timings) == ((8, 8), 64)
    autotune.store(path, "k", {"tile": [8, 8], "batch": 64, "timings": timings})
    autotune.store(path, "k2", {"tile": [16, 16], "batch": 256, "timings": timings})
    data = autotune.load(path)
    assert data["k"]["batch"] == 64 and data["k2"]["tile"] == [16, 16]
    assert autotune.load(str(tmp_path / "missing.json")) == {}
