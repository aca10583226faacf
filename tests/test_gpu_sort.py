"""GPU parity: the CUDA library (through its C ABI) against the CPU oracle.

Sorting has one correct output (ascending, IEEE total order; stable for
pairs), so every comparison is bit-exact.  Level-0 intermediates (range,
parameters and the bucket table T) are compared too, since both sides
follow the same reading of Sec. 3.3.
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


def to_dev(x):
    if x.dtype == np.float64:
        return torch.from_numpy(np.ascontiguousarray(x)).cuda()
    return torch.from_numpy(np.ascontiguousarray(x).view(np.int64)).cuda()


def from_dev(t, like):
    a = t.cpu().numpy()
    return a if like.dtype == np.float64 else a.view(np.uint64)


def kt_of(x):
    return "f64" if x.dtype == np.float64 else "u64"


def gpu_sort(ctx, x, seed=0, in_place=False):
    t = to_dev(x)
    out = t if in_place else torch.empty_like(t)
    ctx.sort_keys(t, out, key_type=kt_of(x), seed=seed)
    torch.cuda.synchronize()
    return from_dev(out, x)


def gpu_sort_pairs(ctx, x, v, seed=0):
    t = to_dev(x)
    tv = torch.from_numpy(v.view(np.int32)).cuda()
    ko, vo = torch.empty_like(t), torch.empty_like(tv)
    ctx.sort_pairs(t, tv, ko, vo, key_type=kt_of(x), seed=seed)
    torch.cuda.synchronize()
    return from_dev(ko, x), vo.cpu().numpy().view(np.uint32)


def same_bits(a, b):
    return np.array_equal(np.asarray(a).view(np.uint64), np.asarray(b).view(np.uint64))


EDGE = [
    np.array([1.5]),
    np.array([2.0, 1.0]),
    np.full(700, 3.25),
    np.full(5000, -1.0),
    np.array([1.0, 2.0] * 3000),
    np.array([0.0, -0.0] * 2500 + [-0.0]),
    np.array([5e-324, -5e-324, 0.0, -0.0, 2.2250738585072014e-308] * 800),
    np.array([np.inf, -np.inf, 1.0, 0.0] * 50),
    np.array([np.inf, -np.inf, 1.0, 0.0] * 5000),
    np.arange(100000, dtype=np.float64),
    np.arange(100000, dtype=np.float64)[::-1].copy(),
    np.arange(100000, dtype=np.float64) * 0.25,
    np.array([0, 2**64 - 1, 1, 2**63] * 2000, dtype=np.uint64),
    np.array([1e308, -1e308] * 3000 + [0.0]),
]


@pytest.mark.parametrize("i", range(len(EDGE)))
def test_edge_cases(ctx, i):
    x = EDGE[i]
    ref, _ = oracle.sort(x)
    assert same_bits(gpu_sort(ctx, x), ref)


@pytest.mark.parametrize("n", [0, 1, 2, 3, 31, 99, 100, 101, 511, 512, 513, 1023, 1024, 1025,
                               4097, 32768, 32769, 100003])
@pytest.mark.parametrize("dist", ["uniform", "normal", "lognormal"])
def test_sizes(ctx, n, dist):
    x = W.f64_keys(dist, n, n + 1)
    ref, _ = oracle.sort(x, seed=5)
    assert same_bits(gpu_sort(ctx, x, seed=5), ref)


@pytest.mark.parametrize("dist", W.DISTRIBUTIONS)
def test_config1_scale(ctx, dist):
    # n = 10^6 (the small configuration; several tiles and a ragged tail)
    x = W.f64_keys(dist, 10**6 + 17, 0)
    ref, _ = oracle.sort(x)
    assert same_bits(gpu_sort(ctx, x), ref)


def test_in_place_equals_out_of_place(ctx):
    x = W.f64_keys("mixture", 300001, 3)
    a = gpu_sort(ctx, x)
    b = gpu_sort(ctx, x, in_place=True)
    assert same_bits(a, b)


def test_injected_duplicates(ctx):
    # the paper's appendix input: n extra copies of one value in [min, max]
    x = W.inject_duplicates(W.f64_keys("normal", 200000, 4), seed=4)
    ref, _ = oracle.sort(x)
    assert same_bits(gpu_sort(ctx, x), ref)


@pytest.mark.parametrize("n", [5000, 300000])
def test_u64_pairs_stable(ctx, n):
    x = W.zipf_u64(n, seed=5, n_values=max(10, n // 50))
    v = np.arange(n, dtype=np.uint32)
    rk, rv = oracle.sort(x, v)
    k, vv = gpu_sort_pairs(ctx, x, v)
    assert same_bits(k, rk)
    assert np.array_equal(vv, rv)


def test_f64_pairs_stable(ctx):
    x = np.round(W.f64_keys("normal", 400000, 8) * 20.0) / 20.0  # many duplicates
    v = np.arange(x.size, dtype=np.uint32)[::-1].copy()
    rk, rv = oracle.sort(x, v)
    k, vv = gpu_sort_pairs(ctx, x, v)
    assert same_bits(k, rk)
    assert np.array_equal(vv, rv)


def test_level0_intermediates_match_oracle(ctx):
    for dist, n in [("uniform", 10**6), ("normal", 300000), ("lognormal", 123457)]:
        x = W.f64_keys(dist, n, 0)
        ref = oracle.level0(x, seed=11)
        got = ctx.debug_level0(to_dev(x), key_type="f64", seed=11)
        for k in ("alpha", "beta", "gamma", "delta", "lo_bits", "hi_bits", "status"):
            assert got[k] == ref[k], (dist, k)
        assert np.array_equal(got["T"].astype(np.uint64), ref["T"]), dist


def test_segmented_equals_separate(ctx):
    keys, offs, _ = W.batched_f64(40, seed=6, lo_exp=1.0, hi_exp=16.0)
    t = to_dev(keys)
    out = torch.empty_like(t)
    ctx.sort_segmented(t, offs, keys_out=out, key_type="f64", seed=9)
    torch.cuda.synchronize()
    got = out.cpu().numpy()
    for s in range(40):
        seg = keys[offs[s]:offs[s + 1]]
        ref, _ = oracle.sort(seg, seed=9 + s)
        assert same_bits(got[offs[s]:offs[s + 1]], ref), s


def test_segmented_pairs(ctx):
    keys, offs, _ = W.batched_f64(25, seed=7, lo_exp=3.0, hi_exp=15.0)
    keys = np.round(keys, 1)
    v = np.arange(keys.size, dtype=np.uint32)
    t, tv = to_dev(keys), torch.from_numpy(v.view(np.int32)).cuda()
    ko, vo = torch.empty_like(t), torch.empty_like(tv)
    ctx.sort_segmented(t, offs, vals_in=tv, keys_out=ko, vals_out=vo, key_type="f64")
    torch.cuda.synchronize()
    k, vv = ko.cpu().numpy(), vo.cpu().numpy().view(np.uint32)
    for s in range(25):
        a, b = offs[s], offs[s + 1]
        rk, rv = oracle.sort(keys[a:b], v[a:b], seed=s)
        assert same_bits(k[a:b], rk) and np.array_equal(vv[a:b], rv), s


def test_tuning_does_not_change_output(P):
    x = W.f64_keys("exponential", 500000, 12)
    ref, _ = oracle.sort(x)
    for tu in (dict(max_digit_bits=6, tile_log2=12, leaf_cap=128),
               dict(max_digit_bits=11, tile_log2=16, leaf_cap=1024),
               dict(max_digit_bits=8, tile_log2=14, leaf_cap=256)):
        c = P.Context(0, tuning=tu)
        assert same_bits(gpu_sort(c, x), ref), tu
        c.close()


def test_other_policy(P):
    # alpha = n^{3/4}, beta = n^{1/2}, gamma = n^{1/2}, delta = n^{3/4}, tau = 32
    x = W.f64_keys("lognormal", 200000, 13)
    ref, _ = oracle.sort(x, seed=3, policy=oracle.Policy(3, 2, 2, 3, 4, 32))
    c = P.Context(0, policy=(3, 2, 2, 3, 4, 32))
    assert same_bits(gpu_sort(c, x, seed=3), ref)
    c.close()


def test_nan_rejected_and_output_untouched(ctx, P):
    x = W.f64_keys("normal", 100000, 1)
    x[777] = np.nan
    t = to_dev(x)
    out = torch.full_like(t, 7.0)
    with pytest.raises(P.PcfError) as e:
        ctx.sort_keys(t, out, key_type="f64")
    assert e.value.code == 2
    torch.cuda.synchronize()
    assert bool((out == 7.0).all())
    small = torch.tensor([1.0, float("nan"), 0.0], dtype=torch.float64, device="cuda")
    out = torch.full_like(small, 7.0)
    with pytest.raises(P.PcfError):
        ctx.sort_keys(small, out, key_type="f64")
    assert bool((out == 7.0).all())


def test_scan_matches_cumsum(ctx):
    g = np.random.Generator(np.random.PCG64(2))
    for n in (1, 4095, 4096, 4097, 1 << 20, 3000001):
        a = g.integers(0, 1000, n).astype(np.uint32)
        t = torch.from_numpy(a.view(np.int32)).cuda()
        assert ctx.debug_scan(t) == 0
        ex = np.concatenate([[0], np.cumsum(a.astype(np.uint64))[:-1]]).astype(np.uint32)
        assert np.array_equal(t.cpu().numpy().view(np.uint32), ex)


def test_bounded_wait_times_out_without_fault(ctx):
    # a tile that never publishes: its successor gives up after the bounded
    # spin and reports a timeout; the context stays usable afterwards
    a = torch.ones(4096 * 8, dtype=torch.int32, device="cuda")
    rc = ctx.debug_scan(a, withhold_tile=3, spin_limit=2000)
    assert rc == 5
    x = W.f64_keys("uniform", 50000, 3)
    ref, _ = oracle.sort(x)
    assert same_bits(gpu_sort(ctx, x), ref)


def test_invalid_arguments(ctx, P):
    t = torch.zeros(10, dtype=torch.float64, device="cuda")
    L = P.lib()
    assert L.pcf_sort_keys(ctx._h, t.data_ptr(), t.data_ptr(), 10, 7, 0, None) == 1
    assert L.pcf_sort_keys(ctx._h, None, t.data_ptr(), 10, 0, 0, None) == 1
    assert L.pcf_sort_keys(ctx._h, t.data_ptr() + 4, t.data_ptr(), 2, 0, 0, None) == 1
    with pytest.raises(P.PcfError):
        ctx.set_policy(3, 3, 3, 4, 4, 100)  # delta exponent must be < 1
    with pytest.raises(P.PcfError):
        ctx.set_policy(model=2)             # no such CDF model
    with pytest.raises(P.PcfError):
        ctx.set_policy(range_mode=5)        # no such range mode
    # the bucketing-only entry: arrays of fewer than 2 keys, bad parameters
    k = torch.from_numpy(W.f64_keys("normal", 1000, 1)).cuda()
    for offs, abc in [([0, 1, 1000], (10, 10, 10)), ([0, 500, 400, 1000], (10, 10, 10)),
                      ([0, 1000], (0, 10, 10)), ([0, 1000], (10, 10, 1 << 24))]:
        with pytest.raises(P.PcfError) as ei:
            ctx.bucket_sizes(k, offs, *abc)
        assert ei.value.code == 1
    x = W.f64_keys("normal", 1000, 2)
    x[500] = np.nan
    with pytest.raises(P.PcfError) as ei:
        ctx.bucket_sizes(to_dev(x), [0, 1000], 30, 30, 30)
    assert ei.value.code == 2
    ctx.set_policy()  # back to the default for the tests that follow


def test_host_batch_error_leaves_no_copy_in_flight(ctx, P):
    # a NaN in the second of three arrays: the call fails, returns with its
    # copies drained, and the context sorts normally afterwards
    xs = [W.f64_keys("uniform", 200000, 60 + i) for i in range(3)]
    xs[1][1234] = np.nan
    hs = [torch.from_numpy(x.copy()).pin_memory() for x in xs]
    with pytest.raises(P.PcfError) as ei:
        ctx.sort_keys_host_batch(hs, key_type="f64")
    assert ei.value.code == 2
    ref, _ = oracle.sort(xs[0])
    assert same_bits(hs[0].numpy(), ref)       # the array before the failure is done
    h = torch.from_numpy(xs[2].copy()).pin_memory()
    ctx.sort_keys_host_batch([h], key_type="f64")
    ref, _ = oracle.sort(xs[2])
    assert same_bits(h.numpy(), ref)


def test_injected_allocation_failure(P):
    # a device allocation fails (injected on the host, as an exhausted
    # device would report it) at every point of a fresh context's first
    # sort: the call returns PCF_ERR_OOM with nothing in flight, and the
    # same context then sorts correctly
    x = W.f64_keys("lognormal", 300000, 77)
    ref, _ = oracle.sort(x)
    L = P.lib()
    failures = 0
    for k in range(64):
        c = P.Context(0)
        L.pcf_debug_fail_alloc_after(k)
        try:
            got = gpu_sort(c, x)
            L.pcf_debug_fail_alloc_after(-1)
            assert same_bits(got, ref)
            c.close()
            break  # k is past the last allocation of the call
        except P.PcfError as e:
            assert e.code == 3, (k, e.code)
            failures += 1
        finally:
            L.pcf_debug_fail_alloc_after(-1)
        assert same_bits(gpu_sort(c, x), ref), k
        c.close()
    assert failures >= 5


def test_copy_bandwidth_probe(ctx, P):
    src = torch.randint(-2**62, 2**62, (1 << 24,), dtype=torch.int64, device="cuda")
    dst = torch.zeros_like(src)
    gbs = ctx.copy_bandwidth(src, dst, reps=3)
    torch.cuda.synchronize()
    assert torch.equal(src, dst) and gbs > 0
    with pytest.raises(P.PcfError):
        ctx.copy_bandwidth(src[:-2], src[2:], reps=1)  # overlapping buffers


def test_host_end_to_end(ctx):
    x = W.f64_keys("normal", 1 << 20, 21)
    h = torch.from_numpy(x.copy()).pin_memory()
    ctx.sort_keys_host(h, key_type="f64")
    ref, _ = oracle.sort(x)
    assert same_bits(h.numpy(), ref)


@pytest.mark.parametrize("pinned", [True, False])
def test_host_batch_pipelined(ctx, pinned):
    # more arrays than the three device slots, sizes from empty to 2^21,
    # each sorted in place exactly as the single-array host call would
    sizes = [1 << 21, 0, 1, 5000, 300001, 1 << 20, 99, 777777]
    xs = [W.f64_keys(W.DISTRIBUTIONS[i % len(W.DISTRIBUTIONS)], n, 40 + i)
          for i, n in enumerate(sizes)]
    hs = [torch.from_numpy(x.copy()) for x in xs]
    if pinned:
        hs = [h.pin_memory() for h in hs]
    ctx.sort_keys_host_batch(hs, key_type="f64", seed=3)
    for i, (x, h) in enumerate(zip(xs, hs)):
        ref, _ = oracle.sort(x, seed=3 + i)
        assert same_bits(h.numpy(), ref), i
    # u64 keys, and a second call on the same context (slots reused)
    us = [W.zipf_u64(n, seed=50 + n % 7, n_values=1000) for n in (123457, 4096, 1 << 19, 2, 65536)]
    hu = [torch.from_numpy(u.view(np.int64).copy()).pin_memory() for u in us]
    ctx.sort_keys_host_batch(hu, key_type="u64")
    for u, h in zip(us, hu):
        ref, _ = oracle.sort(u)
        assert same_bits(h.numpy().view(np.uint64), ref)


@pytest.mark.parametrize("start", [0, 1, 3])
def test_buffers_at_any_8_byte_offset(ctx, start):
    # key buffers that start 8 bytes past a 16-byte boundary (a slice at an
    # odd index): the vector loads must begin at the first aligned key
    x = W.f64_keys("normal", 3 * 10**5 + 7, 30 + start)
    t = to_dev(x)
    src = t[start:]
    out = torch.empty(src.numel() + 1, dtype=torch.float64, device="cuda")[1:]
    ctx.sort_keys(src, out, key_type="f64")
    torch.cuda.synchronize()
    ref, _ = oracle.sort(x[start:])
    assert same_bits(out.cpu().numpy(), ref)
