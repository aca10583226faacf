"""The autotuner's host logic (no GPU): workload classes and the cache."""
from paper_2405_07122_gb300 import autotune


def test_workload_key_classes():
    assert autotune.workload_key("keys", 10**8) == "keys:f64:keys:2^26"
    assert autotune.workload_key("segmented", 2**30 + 5, "u64", pairs=True) == \
        "segmented:u64:pairs:2^30"
    # one class per power of two
    assert autotune.workload_key("keys", 2**20) == autotune.workload_key("keys", 2**21 - 1)
    assert autotune.workload_key("keys", 2**20) != autotune.workload_key("keys", 2**21)
    assert autotune.workload_key("keys", 0) == "keys:f64:keys:2^0"


def test_cache_round_trip(tmp_path):
    path = str(tmp_path / "sub" / "tune.json")
    assert autotune.load_cache(path) == {}  # missing file: empty cache
    c = {"keys:f64:keys:2^26": {"max_digit_bits": 11, "tile_log2": 14, "leaf_cap": 4096}}
    autotune.save_cache(c, path)
    assert autotune.load_cache(path) == c
    (tmp_path / "bad.json").write_text("{not json")
    assert autotune.load_cache(str(tmp_path / "bad.json")) == {}


def test_default_grid_is_speed_only():
    # only pcf_tuning knobs: none of them changes alpha..delta, tau or the output
    assert set(autotune.DEFAULT_GRID) == {"max_digit_bits", "tile_log2", "leaf_cap"}
    for v in autotune.DEFAULT_GRID["leaf_cap"]:
        assert 64 <= v <= 8192 and v & (v - 1) == 0
