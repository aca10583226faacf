"""The autotuner on the GPU: it times every knob setting of its grid on a
sample of the workload, keeps the fastest in its cache, and the tuned
context still sorts bit for bit like the oracle (the knobs are speed only)."""
import numpy as np
import pytest

import oracle
from paper_2405_07122_gb300 import workloads as W

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")


@pytest.fixture(scope="module")
def A():
    from paper_2405_07122_gb300 import build as pcf_build
    pcf_build.build()
    from paper_2405_07122_gb300 import autotune
    return autotune


def test_tune_picks_a_setting_of_its_grid(A):
    keys, offs, _ = W.batched_f64(64, seed=3, lo_exp=10.0, hi_exp=17.0)
    t = torch.from_numpy(keys).cuda()
    o = torch.empty_like(t)
    grid = {"leaf_cap": (1024, 4096), "tile_log2": (14,)}
    best, res = A.tune(lambda c: c.sort_segmented(t, offs, keys_out=o, key_type="f64"),
                       grid=grid, reps=2)
    assert set(res) == {(1024, 14), (4096, 14)}
    assert all(ms > 0 for ms in res.values())
    assert best == min(({"leaf_cap": k[0], "tile_log2": k[1]} for k in res),
                       key=lambda d: res[(d["leaf_cap"], d["tile_log2"])])


def test_tuned_context_caches_and_sorts(A, tmp_path):
    cache = str(tmp_path / "tune.json")
    x = W.f64_keys("mixture", 2**21 + 9, 4)
    t = torch.from_numpy(x).cuda()
    o = torch.empty_like(t)
    key = A.workload_key("keys", x.size)
    grid = {"leaf_cap": (2048, 4096), "max_digit_bits": (10, 11)}
    ctx = A.tuned_context(key, lambda c: c.sort_keys(t, o, key_type="f64"), grid=grid,
                          cache_path=cache)
    tuned = A.load_cache(cache)[key]
    assert tuned["leaf_cap"] in (2048, 4096) and tuned["max_digit_bits"] in (10, 11)
    got = ctx.tuning()
    assert got["leaf_cap"] == tuned["leaf_cap"]
    assert got["max_digit_bits"] == tuned["max_digit_bits"]
    ctx.close()

    def must_not_run(c):
        raise AssertionError("a cached key is not tuned again")

    ctx = A.tuned_context(key, must_not_run, grid=grid, cache_path=cache)
    o.zero_()
    ctx.sort_keys(t, o, key_type="f64", seed=2)
    torch.cuda.synchronize()
    ref, _ = oracle.sort(x, seed=2)
    assert np.array_equal(o.cpu().numpy().view(np.uint64), ref.view(np.uint64))
    ctx.close()
