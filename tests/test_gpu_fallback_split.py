"""GPU parity of the standard sort on duplicate-heavy buckets.

A bucket that the failure guard (|c| >= delta) sends to the standard sort
and that one value dominates is split stably into below / equal / above
that value, round after round, before the merge sort takes what is left.
These inputs put many heavy values into one bucket, so that several rounds
(and more than the round limit) run; outputs are compared bit for bit with
the oracle, values included (stability).
"""
import numpy as np
import pytest

import oracle
from paper_2405_07122_gb300 import workloads as W

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")


@pytest.fixture(scope="module")
def P():
    from paper_2405_07122_gb300 import build as pcf_build
    pcf_build.build()
    from paper_2405_07122_gb300 import pcfsort
    return pcfsort


@pytest.fixture(scope="module")
def ctx(P):
    c = P.Context(0)
    yield c
    c.close()


def _dev(x):
    return torch.from_numpy(x if x.dtype == np.float64 else x.view(np.int64)).cuda()


def _kt(x):
    return "f64" if x.dtype == np.float64 else "u64"


def _sort(ctx, x, v=None, seed=0):
    t = _dev(x)
    ko = torch.empty_like(t)
    if v is None:
        ctx.sort_keys(t, ko, key_type=_kt(x), seed=seed)
        torch.cuda.synchronize()
        k = ko.cpu().numpy()
        return (k if x.dtype == np.float64 else k.view(np.uint64)), None
    tv = torch.from_numpy(v.view(np.int32)).cuda()
    vo = torch.empty_like(tv)
    ctx.sort_pairs(t, tv, ko, vo, key_type=_kt(x), seed=seed)
    torch.cuda.synchronize()
    k = ko.cpu().numpy()
    return (k if x.dtype == np.float64 else k.view(np.uint64)), vo.cpu().numpy().view(np.uint32)


def _bits(a):
    return np.ascontiguousarray(a).view(np.uint64)


def geometric_u64(n, seed, heavy=24):
    """Heavy value k (adjacent integers near 2^63) holds n >> (k + 1) keys;
    the rest are uniform 64-bit noise.  All heavy values share one bucket."""
    g = np.random.Generator(np.random.PCG64(seed))
    parts, used = [], 0
    for k in range(heavy):
        c = n >> (k + 1)
        parts.append(np.full(c, (1 << 63) + 3 * k, dtype=np.uint64))
        used += c
    parts.append(g.integers(0, 2**64 - 1, size=n - used, dtype=np.uint64, endpoint=True))
    x = np.concatenate(parts)
    g.shuffle(x)
    return x


def signed_zeros_f64(n, seed):
    """Half -0.0, a quarter +0.0 (distinct keys in the total order), an
    eighth the next double above +0.0, the rest normal noise."""
    g = np.random.Generator(np.random.PCG64(seed))
    a, b, c = n // 2, n // 4, n // 8
    x = np.concatenate([np.full(a, -0.0), np.full(b, 0.0), np.full(c, 5e-324),
                        g.normal(0.0, 1.0, size=n - a - b - c)])
    g.shuffle(x)
    return x


@pytest.mark.parametrize("n", [1 << 20, 3 * 10**5 + 7])
def test_geometric_heavy_values_pairs(ctx, n):
    x = geometric_u64(n, seed=n)
    v = np.arange(n, dtype=np.uint32)[::-1].copy()
    rk, rv = oracle.sort(x, v)
    k, vv = _sort(ctx, x, v)
    assert np.array_equal(k, rk)
    assert np.array_equal(vv, rv)
    st = ctx.last_stats()
    assert st["fallback_splits"] >= 8  # the round limit was reached


def test_geometric_heavy_values_keys(ctx):
    x = geometric_u64(1 << 20, seed=3)
    rk, _ = oracle.sort(x)
    k, _ = _sort(ctx, x)
    assert np.array_equal(k, rk)
    assert ctx.last_stats()["fallback_splits"] >= 8


@pytest.mark.parametrize("pairs", [False, True])
def test_signed_zeros_are_distinct_pivots(ctx, pairs):
    n = 400001
    x = signed_zeros_f64(n, seed=9)
    v = np.arange(n, dtype=np.uint32) if pairs else None
    rk, rv = oracle.sort(x, v)
    k, vv = _sort(ctx, x, v)
    assert np.array_equal(_bits(k), _bits(rk))
    if pairs:
        assert np.array_equal(vv, rv)
    assert ctx.last_stats()["fallback_splits"] >= 1


@pytest.mark.parametrize("n", [5000, 70001, 262144])
def test_injected_duplicates_ragged_sizes(ctx, n):
    # the appendix input at sizes that leave a ragged last tile
    x = W.inject_duplicates(W.f64_keys("lognormal", n // 2, n), seed=n)
    v = np.arange(x.size, dtype=np.uint32)
    rk, rv = oracle.sort(x, v)
    k, vv = _sort(ctx, x, v)
    assert np.array_equal(_bits(k), _bits(rk))
    assert np.array_equal(vv, rv)
    k2, _ = _sort(ctx, x)
    assert np.array_equal(_bits(k2), _bits(rk))


def test_segmented_several_split_items(ctx):
    # several arrays, each with its own dominant value: several items per round
    g = np.random.Generator(np.random.PCG64(21))
    arrs = []
    for s in range(7):
        m = int(g.integers(3000, 90000))
        arrs.append(W.inject_duplicates(W.f64_keys("normal", m, 100 + s), seed=200 + s))
    offs = np.zeros(len(arrs) + 1, dtype=np.uint64)
    offs[1:] = np.cumsum([a.size for a in arrs])
    x = np.concatenate(arrs)
    v = np.arange(x.size, dtype=np.uint32)
    t, tv = _dev(x), torch.from_numpy(v.view(np.int32)).cuda()
    ko, vo = torch.empty_like(t), torch.empty_like(tv)
    ctx.sort_segmented(t, offs, vals_in=tv, keys_out=ko, vals_out=vo, key_type="f64", seed=4)
    torch.cuda.synchronize()
    k, vv = ko.cpu().numpy(), vo.cpu().numpy().view(np.uint32)
    for s in range(len(arrs)):
        a, b = int(offs[s]), int(offs[s + 1])
        rk, rv = oracle.sort(x[a:b], v[a:b])
        assert np.array_equal(_bits(k[a:b]), _bits(rk)), s
        assert np.array_equal(vv[a:b], rv), s
    assert ctx.last_stats()["fallback_splits"] >= len(arrs)
