"""GPU parity of the block-local leaf sort (tuning leaf_mode 1, keys only)
and of the on-chip Learned-Sort steps it replaces by default (leaf_mode 2).

A bucket that fits in shared memory is finished by a Standard-Sort, which
Alg. 1 leaves open (Sec. 3.1: any sort): one equal-width split of the
bucket's range into about n parts, ranks inside the parts, and a warp sort
of the parts that hold more than 16 keys.  The output is the unique
ascending order, so every case is compared bit for bit with the oracle.
The inputs aim at the split's hard cases: outliers that put most keys in
one part, few distinct values, the extremes of the u64 and binary64 orders.
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


@pytest.fixture(scope="module", params=[(1, 8192), (1, 4096), (2, 4096)],
                ids=["sort-8192", "sort-4096", "learned-4096"])
def ctx(P, request):
    mode, cap = request.param
    c = P.Context(0, tuning=dict(leaf_mode=mode, leaf_cap=cap))
    assert c.tuning()["leaf_mode"] == mode
    yield c
    c.close()


def _dev(x):
    return torch.from_numpy(np.ascontiguousarray(x if x.dtype == np.float64
                                                 else x.view(np.int64))).cuda()


def _sort(ctx, x, seed=0):
    t = _dev(x)
    out = torch.empty_like(t)
    ctx.sort_keys(t, out, key_type="f64" if x.dtype == np.float64 else "u64", seed=seed)
    torch.cuda.synchronize()
    return out.cpu().numpy().view(np.uint64)


def _check(ctx, x, seed=0):
    ref, _ = oracle.sort(x, seed=seed)
    got = _sort(ctx, x, seed)
    assert np.array_equal(got, np.ascontiguousarray(ref).view(np.uint64))


def _skewed(n, seed):
    """n keys: a tight cluster plus a few far outliers, so that one part of
    an equal-width split of the range holds almost every key."""
    g = np.random.Generator(np.random.PCG64(seed))
    x = 1.0 + g.random(n) * 1e-6
    k = max(1, n // 200)
    x[g.integers(0, n, size=k)] = 1e6 * (1.0 + g.random(k))
    return x


SIZES = [2, 3, 17, 33, 65, 100, 255, 256, 257, 700, 1024, 1025, 2048, 3000, 4096, 6000, 8192]


@pytest.mark.parametrize("n", SIZES)
def test_skewed_parts(ctx, n):
    _check(ctx, _skewed(n, n))


@pytest.mark.parametrize("n", SIZES)
@pytest.mark.parametrize("values", [2, 3, 7, 40])
def test_few_distinct_values(ctx, n, values):
    g = np.random.Generator(np.random.PCG64(n * 100 + values))
    x = g.normal(size=values)[g.integers(0, values, size=n)]
    _check(ctx, x)


@pytest.mark.parametrize("n", [64, 1000, 4096, 8192])
def test_u64_extremes(ctx, n):
    g = np.random.Generator(np.random.PCG64(n + 3))
    x = g.integers(0, 2**64 - 1, size=n, dtype=np.uint64, endpoint=True)
    x[: n // 8] = np.uint64(2**64 - 1)
    x[n // 8: n // 4] = 0
    _check(ctx, g.permutation(x))
    # a narrow range: every key its own part (no shift)
    y = np.uint64(2**63) + g.integers(0, n // 2 + 1, size=n, dtype=np.uint64)
    _check(ctx, y)


@pytest.mark.parametrize("n", [100, 1500, 8000])
def test_special_binary64(ctx, n):
    g = np.random.Generator(np.random.PCG64(n + 9))
    pool = np.array([0.0, -0.0, 5e-324, -5e-324, np.inf, -np.inf, 1e308, -1e308,
                     2.2250738585072014e-308, 1.0, -1.0])
    x = np.concatenate([pool[g.integers(0, pool.size, size=n // 2)],
                        g.normal(size=n - n // 2)])
    _check(ctx, g.permutation(x))


@pytest.mark.parametrize("dist", ["uniform", "normal", "exponential", "lognormal", "mixture"])
def test_level_buckets(ctx, dist):
    # a global level, then its buckets finished on chip
    _check(ctx, W.f64_keys(dist, 2 * 10**6 + 5, 41), seed=3)


def test_segmented_classes(ctx):
    g = np.random.Generator(np.random.PCG64(77))
    lens = g.integers(0, 8193, size=300)
    lens[:8] = [0, 1, 2, 256, 257, 4096, 4097, 8192]
    offs = np.zeros(lens.size + 1, dtype=np.uint64)
    offs[1:] = np.cumsum(lens)
    x = W.f64_keys("normal", int(offs[-1]), 5)
    x[::7] = np.round(x[::7], 1)  # duplicates inside every array
    t = _dev(x)
    out = torch.empty_like(t)
    ctx.sort_segmented(t, offs, keys_out=out, key_type="f64", seed=8)
    torch.cuda.synchronize()
    got = out.cpu().numpy().view(np.uint64)
    for s in range(lens.size):
        a, b = int(offs[s]), int(offs[s + 1])
        ref, _ = oracle.sort(x[a:b], seed=8 + s)
        assert np.array_equal(got[a:b], ref.view(np.uint64)), s


def test_modes_agree_and_pairs_unaffected(P):
    x = W.f64_keys("lognormal", 3 * 10**6, 12)
    outs = []
    for mode in (1, 2):
        c = P.Context(0, tuning=dict(leaf_mode=mode))
        outs.append(_sort(c, x))
        c.close()
    assert np.array_equal(outs[0], outs[1])
    # key-value sorts keep the stable on-chip Learned-Sort steps
    c = P.Context(0, tuning=dict(leaf_mode=1))
    v = np.arange(x.size, dtype=np.uint32)
    t, tv = _dev(x), torch.from_numpy(v.view(np.int32)).cuda()
    ko, vo = torch.empty_like(t), torch.empty_like(tv)
    c.sort_pairs(t, tv, ko, vo, key_type="f64")
    torch.cuda.synchronize()
    rk, rv = oracle.sort(x, v)
    assert np.array_equal(ko.cpu().numpy().view(np.uint64), rk.view(np.uint64))
    assert np.array_equal(vo.cpu().numpy().view(np.uint32), rv)
    c.close()


def test_bad_leaf_mode(P):
    c = P.Context(0)
    with pytest.raises(Exception):
        c.set_tuning(leaf_mode=3)
    c.close()
