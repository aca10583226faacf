"""GPU parity of the large on-chip size classes (buckets of 1025-8192 keys,
one CTA of 128-512 threads per bucket, keys only) against the oracle.

With leaf_cap above 1024 a bucket (or a whole array) of up to leaf_cap keys
runs its remaining Learned-Sort recursion in shared memory instead of at
another global level; key-value sorts keep 1024.  The output must not
change: every case is compared bit for bit with the oracle.
"""
import numpy as np
import pytest

import oracle
from paper_2405_07122_gb300 import workloads as W

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")

CAPS = [2048, 4096, 8192]


@pytest.fixture(scope="module")
def P():
    from paper_2405_07122_gb300 import build as pcf_build
    pcf_build.build()
    from paper_2405_07122_gb300 import pcfsort
    return pcfsort


@pytest.fixture(scope="module", params=CAPS)
def ctx(P, request):
    c = P.Context(0, tuning=dict(leaf_cap=request.param))
    yield c
    c.close()


def _dev(x):
    return torch.from_numpy(x if x.dtype == np.float64 else x.view(np.int64)).cuda()


def _sort(ctx, x, seed=0):
    t = _dev(x)
    out = torch.empty_like(t)
    ctx.sort_keys(t, out, key_type="f64" if x.dtype == np.float64 else "u64", seed=seed)
    torch.cuda.synchronize()
    return out.cpu().numpy().view(np.uint64)


def _bits(a):
    return np.ascontiguousarray(a).view(np.uint64)


@pytest.mark.parametrize("n", [1025, 2047, 2048, 2049, 3001, 4095, 4096, 4097, 6000, 8191, 8192,
                               8193])
@pytest.mark.parametrize("dist", ["uniform", "normal", "lognormal", "mixture"])
def test_whole_arrays_on_chip(ctx, n, dist):
    x = W.f64_keys(dist, n, n * 7 + 1)
    ref, _ = oracle.sort(x, seed=2)
    assert np.array_equal(_sort(ctx, x, seed=2), _bits(ref))


@pytest.mark.parametrize("dist", ["exponential", "lognormal", "mixture"])
def test_level0_buckets_in_large_classes(ctx, dist):
    # heavy-tailed and clustered inputs: many level-0 buckets of 1025-8192 keys
    x = W.f64_keys(dist, 3 * 10**6 + 11, 5)
    ref, _ = oracle.sort(x)
    assert np.array_equal(_sort(ctx, x), _bits(ref))


def test_u64_keys(ctx):
    g = np.random.Generator(np.random.PCG64(17))
    x = g.integers(0, 2**40, size=2 * 10**6, dtype=np.uint64) << np.uint64(3)
    ref, _ = oracle.sort(x)
    assert np.array_equal(_sort(ctx, x), ref)


@pytest.mark.parametrize("n", [1500, 5000, 8192])
def test_degenerate_calls(ctx, n):
    g = np.random.Generator(np.random.PCG64(n))
    # infinite keys: a degenerate range, the whole call goes to Standard-Sort
    x = g.normal(size=n)
    x[::97] = np.inf
    x[5::101] = -np.inf
    ref, _ = oracle.sort(x)
    assert np.array_equal(_sort(ctx, x), _bits(ref))
    # few distinct values: sub-buckets of at least delta keys
    y = np.round(g.normal(size=n) * 2.0)
    ref, _ = oracle.sort(y)
    assert np.array_equal(_sort(ctx, y), _bits(ref))
    # one value, and a signed-zero mix
    z = np.full(n, 3.5)
    assert np.array_equal(_sort(ctx, z), _bits(z))
    zz = np.where(g.random(n) < 0.5, -0.0, 0.0)
    ref, _ = oracle.sort(zz)
    assert np.array_equal(_sort(ctx, zz), _bits(ref))


def test_segmented_mixed_lengths(ctx):
    g = np.random.Generator(np.random.PCG64(23))
    lens = g.integers(0, 8193, size=400)
    lens[:6] = [0, 1, 1024, 1025, 4096, 8192]
    offs = np.zeros(lens.size + 1, dtype=np.uint64)
    offs[1:] = np.cumsum(lens)
    x = W.f64_keys("lognormal", int(offs[-1]), 29)
    t = _dev(x)
    out = torch.empty_like(t)
    ctx.sort_segmented(t, offs, keys_out=out, key_type="f64", seed=4)
    torch.cuda.synchronize()
    got = out.cpu().numpy().view(np.uint64)
    for s in range(lens.size):
        a, b = int(offs[s]), int(offs[s + 1])
        ref, _ = oracle.sort(x[a:b], seed=4 + s)
        assert np.array_equal(got[a:b], _bits(ref)), s


def test_pairs_keep_their_cap(ctx):
    # key-value sorts run with at most 1024 keys on chip, and stay stable
    x = np.round(W.f64_keys("exponential", 10**6, 31) * 50.0) / 50.0
    v = np.arange(x.size, dtype=np.uint32)
    rk, rv = oracle.sort(x, v)
    t, tv = _dev(x), torch.from_numpy(v.view(np.int32)).cuda()
    ko, vo = torch.empty_like(t), torch.empty_like(tv)
    ctx.sort_pairs(t, tv, ko, vo, key_type="f64")
    torch.cuda.synchronize()
    assert np.array_equal(ko.cpu().numpy().view(np.uint64), _bits(rk))
    assert np.array_equal(vo.cpu().numpy().view(np.uint32), rv)
