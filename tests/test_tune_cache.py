"""The batch autotuner's cache (host logic, no GPU): keys by device and size class, a
store/fetch round trip, rewriting, and an unreadable file treated as empty."""
import json
import os

from paper_1610_07279_gb300 import tune_cache as tc


def test_bucket_is_the_power_of_two_below():
    assert [tc.bucket(v) for v in (0, 1, 2, 3, 4, 5, 1000, 1024, 1025)] == [0, 1, 2, 2, 4, 4, 512, 1024, 1024]


def test_key_classes_sizes_and_search_space():
    k = tc.make_key("GB300", 152, [4096, 5000], (8, 16), (32,), (8192,), 3)
    # same device, same size class (2 systems, 9096 particles -> 8192), same candidates
    assert k == tc.make_key("GB300", 152, [3000, 6000], (8, 16), (32,), (8192,), 3)
    assert k == tc.make_key("GB300", 152, [3000, 6000, 10], (8, 16), (32,), (8192,), 3)  # 3 systems: class 2
    assert k != tc.make_key("GB300", 152, [3000, 6000, 10, 10], (8, 16), (32,), (8192,), 3)  # 4 systems
    assert k != tc.make_key("GB300", 152, [9000, 9000], (8, 16), (32,), (8192,), 3)   # 16384 particles
    assert k != tc.make_key("GB300", 132, [4096, 5000], (8, 16), (32,), (8192,), 3)   # another device
    assert k != tc.make_key("GB300", 152, [4096, 5000], (8, 16, 32), (32,), (8192,), 3)  # another search
    assert k != tc.make_key("GB300", 152, [4096, 5000], (8, 16), (32,), (8192,), 5)


def test_store_fetch_and_rewrite(tmp_path):
    path = str(tmp_path / "sub" / "tune.json")
    c = tc.TuneCache(path)
    assert c.get("a") is None
    c.put("a", {"leaf_max": 16, "group_max": 32, "walk_queue": 8192, "best_ms": 8.2, "ms": [1.0, 2.0]})
    c.put("b", {"leaf_max": 8, "group_max": 64, "walk_queue": 16384, "best_ms": 3.0})
    assert c.get("a") == {"leaf_max": 16, "group_max": 32, "walk_queue": 8192, "best_ms": 8.2}
    c.put("a", {"leaf_max": 32, "group_max": 16, "walk_queue": 8192, "best_ms": 7.0})
    assert tc.TuneCache(path).get("a")["leaf_max"] == 32 and tc.TuneCache(path).get("b")["group_max"] == 64
    assert [f for f in os.listdir(os.path.dirname(path)) if f.startswith(".tune")] == []  # no temporaries left


def test_unreadable_or_malformed_entries(tmp_path):
    path = str(tmp_path / "tune.json")
    with open(path, "w") as f:
        f.write("{not json")
    c = tc.TuneCache(path)
    assert c.get("a") is None
    c.put("a", {"leaf_max": 16, "group_max": 32, "walk_queue": 8192, "best_ms": 1.0})
    assert c.get("a")["walk_queue"] == 8192
    with open(path, "w") as f:
        json.dump({"a": {"leaf_max": "16"}, "b": [1, 2]}, f)
    assert c.get("a") is None and c.get("b") is None
