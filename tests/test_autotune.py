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
    assert set(autotune.DEFAULT_GRID) == {"max_digit_bits", "tile_log2", "leaf_cap", "leaf_mode"}
    for v in autotune.DEFAULT_GRID["leaf_cap"]:
        assert 64 <= v <= 8192 and v & (v - 1) == 0
    assert set(autotune.DEFAULT_GRID["leaf_mode"]) <= {1, 2}


class _FakeContext:
    made = []

    def __init__(self, device=0, tuning=None, **kw):
        self.tuning_ = dict(tuning or {})
        _FakeContext.made.append(self.tuning_)

    def close(self):
        pass


def test_tune_and_cache_logic_without_a_gpu(monkeypatch, tmp_path):
    # every grid point is tried once; the fastest is kept and cached; a
    # cached class is served without tuning again
    cost = {(10, 1024): 3.0, (10, 4096): 1.5, (11, 1024): 2.0, (11, 4096): 2.5}
    monkeypatch.setattr(autotune.pcfsort, "Context", _FakeContext)
    monkeypatch.setattr(autotune, "_time",
                        lambda run, reps: (run(), cost[_FakeContext.cur])[1])

    def runner(ctx):
        _FakeContext.cur = (ctx.tuning_["max_digit_bits"], ctx.tuning_["leaf_cap"])

    _FakeContext.made = []
    grid = {"max_digit_bits": (10, 11), "leaf_cap": (1024, 4096)}
    best, res = autotune.tune(runner, grid=grid)
    assert best == {"max_digit_bits": 10, "leaf_cap": 4096}
    assert res == cost and len(_FakeContext.made) == 4
    path = str(tmp_path / "t.json")
    c = autotune.tuned_context("k", runner, grid=grid, cache_path=path)
    assert c.tuning_ == best and autotune.load_cache(path) == {"k": best}

    def no_tuning(ctx):
        raise AssertionError("a cached class is not tuned again")

    c = autotune.tuned_context("k", no_tuning, grid=grid, cache_path=path)
    assert c.tuning_ == best
    # an unknown class without a runner gets the library's defaults
    c = autotune.tuned_context("other", None, grid=grid, cache_path=path)
    assert c.tuning_ == {}
