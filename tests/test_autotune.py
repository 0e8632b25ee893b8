"""Autotuner cache logic (no GPU)."""
from paper_2404_07183_gb300 import autotune


def test_input_class_buckets_sizes():
    a = autotune.input_class(20000, 275.0, 500, ["l1", "gram"], "f32c", "full", "GB300")
    b = autotune.input_class(30000, 300.0, 510, ["gram", "l1"], "f32c", "full", "GB300")
    c = autotune.input_class(20000, 275.0, 500, ["l1", "gram"], "f64", "full", "GB300")
    assert a == b          # same power-of-two buckets, metric order irrelevant
    assert a != c


def test_cache_roundtrip_and_choice(tmp_path):
    path = str(tmp_path / "tune.json")
    assert autotune.load_cache(path) == {}
    autotune.store("k1", {"schedule": "tile512x2", "timings_ms": {"tile512x2": 1.0}}, path)
    autotune.store("k2", {"schedule": "mergepath", "timings_ms": {}}, path)
    c = autotune.load_cache(path)
    assert c["k1"]["schedule"] == "tile512x2" and c["k2"]["schedule"] == "mergepath"
    assert autotune.choose({"tile1024": 3.0, "tile512x2": 2.5, "mergepath": 9.0}) == "tile512x2"
