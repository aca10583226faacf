"""Autotuner for the speed-only knobs of the library (pcf_tuning).

The knobs are the widest bucket-id digit scattered per global pass
(max_digit_bits), the keys per count tile (tile_log2), the largest bucket
finished on chip (leaf_cap) and how keys-only sorts finish it (leaf_mode: a
block-local sort, or the remaining Learned-Sort steps).  None of them
changes alpha, beta, gamma, delta, tau or the output, so the tuner may pick
any of them; it times each candidate on a sample of the caller's workload
with CUDA events and keeps the fastest.  Results are cached in a JSON file keyed by workload class.
"""
import itertools
import json
import os

from . import pcfsort

DEFAULT_GRID = {
    "max_digit_bits": (10, 11),
    "tile_log2": (13, 14),
    "leaf_cap": (2048, 8192),
    "leaf_mode": (1, 2),
}

CACHE = os.path.join(os.path.dirname(os.path.abspath(__file__)), "_build", "autotune.json")


def workload_key(kind, n, key_type="f64", pairs=False):
    """Workload class: kind ('keys'|'segmented'), size class log2(n), type."""
    return "%s:%s:%s:2^%d" % (kind, key_type, "pairs" if pairs else "keys", max(0, int(n).bit_length() - 1))


def load_cache(path=CACHE):
    try:
        with open(path) as f:
            return json.load(f)
    except Exception:
        return {}


def save_cache(cache, path=CACHE):
    os.makedirs(os.path.dirname(path), exist_ok=True)
    tmp = path + ".tmp"
    with open(tmp, "w") as f:
        json.dump(cache, f, indent=1, sort_keys=True)
    os.replace(tmp, path)


def _time(run, reps):
    import torch
    run()  # warm (allocations, first launch)
    torch.cuda.synchronize()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    best = float("inf")
    for _ in range(reps):
        e0.record()
        run()
        e1.record()
        torch.cuda.synchronize()
        best = min(best, e0.elapsed_time(e1))
    return best


def tune(sample_runner, grid=None, reps=3, device=0):
    """sample_runner(ctx) sorts one sample with context ctx.  Returns
    (best_tuning_dict, {tuning_tuple: ms})."""
    grid = grid or DEFAULT_GRID
    names = list(grid)
    results = {}
    best, best_ms = None, float("inf")
    for combo in itertools.product(*(grid[k] for k in names)):
        t = dict(zip(names, combo))
        ctx = pcfsort.Context(device, tuning=t)
        try:
            ms = _time(lambda: sample_runner(ctx), reps)
        finally:
            ctx.close()
        results[combo] = ms
        if ms < best_ms:
            best, best_ms = t, ms
    return best, results


def tuned_context(key, sample_runner=None, device=0, grid=None, cache_path=CACHE, **ctx_kw):
    """A Context with the cached tuning of `key`; tunes (and caches) first
    when the key is new and a sample_runner is given."""
    cache = load_cache(cache_path)
    if key not in cache and sample_runner is not None:
        best, _ = tune(sample_runner, grid=grid, device=device)
        cache[key] = best
        save_cache(cache, cache_path)
    return pcfsort.Context(device, tuning=cache.get(key), **ctx_kw)
