"""Pins of the oracle's sample-range policy (reading R14: the bins span the
alpha samples' range; keys outside it take the end bins).  (TEST
INFRASTRUCTURE: CPU only.)"""
import numpy as np

import oracle
from paper_2405_07122_gb300 import workloads as W

from test_oracle_pins import KINDS, gen, is_total_order_sorted


def ordk(x):
    b = np.ascontiguousarray(x).view(np.uint64)
    if x.dtype == np.uint64:
        return b
    return np.where(b >> np.uint64(63), ~b, b | np.uint64(2**63))


def pol(model=oracle.MODEL_PCF, tau=100):
    return oracle.paper_policy(tau=tau, model=model, range_mode=oracle.RANGE_SAMPLE)


def test_range_is_the_samples_range():
    for kind in ("uniform", "normal", "lognormal", "u64", "mixture"):
        x = gen(kind, 100000, 13)
        L = oracle.level0(x, seed=4, policy=pol())
        s = x[L["sample_idx"].astype(np.int64)]
        o = ordk(s)
        assert ordk(np.array([L["lo_bits"]], dtype=np.uint64).view(x.dtype))[0] == o.min(), kind
        assert ordk(np.array([L["hi_bits"]], dtype=np.uint64).view(x.dtype))[0] == o.max(), kind
        # the sample's range lies inside the array's
        assert o.min() >= ordk(x).min() and o.max() <= ordk(x).max()


def test_keys_outside_the_sample_range_take_the_end_buckets():
    x = W.f64_keys("normal", 200000, 21)
    L = oracle.level0(x, seed=8, policy=pol())
    lo = np.array([L["lo_bits"]], dtype=np.uint64).view(np.float64)[0]
    hi = np.array([L["hi_bits"]], dtype=np.uint64).view(np.float64)[0]
    kb = L["keys"]
    ends = np.cumsum(L["counts"].astype(np.int64))
    bucket = np.searchsorted(ends, np.arange(x.size), side="right")
    below, above = kb < lo, kb > hi
    assert below.any() and above.any()  # the tails lie outside the sample's range
    assert np.all(bucket[below] == bucket[kb == lo][0])
    assert np.all(bucket[above] >= bucket[kb == hi].max())
    # ordered buckets (Sec. 3.2) over the whole array
    o = ordk(kb)
    for j in range(len(ends) - 1):
        a, b, c = (ends[j - 1] if j else 0), ends[j], ends[j + 1]
        if b > a and c > b:
            assert o[a:b].max() <= o[b:c].min()


def test_equal_samples_fall_back_to_the_array_range():
    # one value holds almost every key: all alpha samples see it, the array
    # has others, and the array's own range is used
    x = np.full(20000, 5.0)
    x[[17, 9000, 19999]] = [-1.0, 3.0, 11.0]
    L = oracle.level0(x, seed=1, policy=pol())
    s = x[L["sample_idx"].astype(np.int64)]
    assert np.all(s == 5.0)
    lo = np.array([L["lo_bits"]], dtype=np.uint64).view(np.float64)[0]
    hi = np.array([L["hi_bits"]], dtype=np.uint64).view(np.float64)[0]
    assert (lo, hi) == (-1.0, 11.0) and L["status"] == 0


def test_sample_range_sort_matches_insertion_sort():
    for n in list(range(2, 300)) + [1000, 2000]:
        kind = KINDS[n % len(KINDS)]
        x = gen(kind, n, n + 31)
        v = np.arange(n, dtype=np.uint32)
        rk, rv = oracle.insertion_sort(x, v)
        for model in (oracle.MODEL_PCF, oracle.MODEL_SPLINE):
            k, vv = oracle.sort(x, v, seed=n, policy=pol(model, tau=4))
            assert np.array_equal(k.view(np.uint64), rk.view(np.uint64)), (kind, n, model)
            assert np.array_equal(vv, rv), (kind, n, model)


def test_sample_range_sort_large_stable():
    for kind in ("uniform", "lognormal", "u64wide", "dups", "inf", "zeros"):
        x = gen(kind, 200000, 41)
        v = np.arange(x.size, dtype=np.uint32)
        k, vv = oracle.sort(x, v, seed=6, policy=pol())
        assert np.array_equal(vv, np.argsort(ordk(x), kind="stable").astype(np.uint32)), kind
        if x.dtype == np.float64:
            assert is_total_order_sorted(k)
