"""Pins of the oracle's Spline Learned Sort (App. A.5): the spline model's
buckets against the PCF model's at the points where the definition ties
them together, the ordered-bucket property, and the final output against
brute force.  (TEST INFRASTRUCTURE: CPU only.)"""
import math
from fractions import Fraction

import numpy as np

import oracle

from test_oracle_pins import KINDS, gen, is_total_order_sorted

SPLINE = oracle.MODEL_SPLINE


def spline_policy(tau=100):
    return oracle.paper_policy(tau=tau, model=SPLINE)


def bucket_of_each(L):
    """Bucket index of every position of the bucketed keys."""
    ends = np.cumsum(L["counts"].astype(np.int64))
    return np.searchsorted(ends, np.arange(int(ends[-1])), side="right")


def test_spline_at_bin_edges_equals_pcf_of_the_previous_bin():
    # n = 256: alpha = beta = gamma = 64; lo = 0, hi = 64, so s = 1 and p = x
    # exactly.  A key on the left edge of bin k has f = 0 and
    # F = b_{k-1} / alpha, which is the PCF table of bin k - 1; a key in the
    # middle of bin k lies between the PCF values of bins k - 1 and k.
    g = np.random.Generator(np.random.PCG64(3))
    edges = np.arange(0, 65, dtype=np.float64)                # 0, 1, ..., 64
    mids = np.arange(0, 64, dtype=np.float64) + 0.5
    rest = g.uniform(0.0, 64.0, 256 - edges.size - mids.size)
    x = np.concatenate([edges, mids, rest])
    g.shuffle(x)
    L = oracle.level0(x, seed=11, policy=spline_policy())
    assert (L["alpha"], L["beta"], L["gamma"]) == (64, 64, 64)
    assert L["status"] == 0
    T = L["T"].astype(np.int64)                               # PCF: floor(b_k g / a) = b_k
    keys, bk = L["keys"], bucket_of_each(L)
    where = {float(v): i for i, v in enumerate(keys)}
    b = L["b"].astype(np.int64)
    assert np.array_equal(T, b)
    for k in range(1, 65):
        assert bk[where[float(k)]] == T[k - 1], k
    assert bk[where[0.0]] == 0
    for k in range(0, 64):
        j = bk[where[k + 0.5]]
        lo = T[k - 1] if k else 0
        assert lo <= j <= T[k], k
        # f = 1/2: y = (b_{k-1} + b_k) / 2, exact in binary64
        assert j == (lo + T[k]) // 2, k


def test_spline_buckets_are_ordered_and_count_every_key():
    for kind in ("uniform", "normal", "lognormal", "mixture", "u64", "dups", "edges"):
        x = gen(kind, 50000, 7)
        L = oracle.level0(x, seed=5, policy=spline_policy())
        if L["status"] != 0:
            continue
        assert int(L["counts"].sum()) == x.size
        kb = L["keys"]
        ends = np.cumsum(L["counts"].astype(np.int64))
        starts = ends - L["counts"].astype(np.int64)
        prev = None
        for s0, e0 in zip(starts, ends):
            if e0 == s0:
                continue
            seg = kb[s0:e0]
            o = np.sort(oracle._bits(seg) ^ np.where(oracle._bits(seg) >> np.uint64(63),
                                                     np.uint64(2**64 - 1), np.uint64(2**63))) \
                if kb.dtype == np.float64 else np.sort(seg)
            if prev is not None:
                assert prev <= o[0], kind
            prev = o[-1]


def test_spline_sort_matches_insertion_sort():
    for n in list(range(2, 300)) + [1000, 2000]:
        kind = KINDS[n % len(KINDS)]
        x = gen(kind, n, n + 17)
        v = np.arange(n, dtype=np.uint32)
        rk, rv = oracle.insertion_sort(x, v)
        k, vv = oracle.sort(x, v, seed=n, policy=oracle.Policy(3, 3, 3, 3, 4, 4, SPLINE))
        assert np.array_equal(k.view(np.uint64), rk.view(np.uint64)), (kind, n)
        assert np.array_equal(vv, rv), (kind, n)


def test_spline_sort_large_and_stats():
    for kind in ("uniform", "lognormal", "mixture", "u64wide", "dups"):
        x = gen(kind, 300000, 29)
        v = np.arange(x.size, dtype=np.uint32)
        k, vv, st = oracle.sort(x, v, seed=2, policy=spline_policy(), with_stats=True)
        assert is_total_order_sorted(k) if x.dtype == np.float64 else np.all(k[:-1] <= k[1:])
        ref = np.argsort(oracle._bits(x) if x.dtype == np.uint64 else
                         np.where(oracle._bits(x) >> np.uint64(63),
                                  ~oracle._bits(x), oracle._bits(x) | np.uint64(2**63)),
                         kind="stable")
        assert np.array_equal(vv, ref.astype(np.uint32)), kind
        assert st["n_bucketings"] >= 1


def test_spline_buckets_with_alpha_not_gamma_are_exact_rationals():
    # App. A.5 in exact reals: j = floor(F(x) gamma), F(x) = (b_{k-1} + f
    # (b_k - b_{k-1})) / alpha.  Policy a = 3/4, b = c = 1/2 at n = 256:
    # alpha = 64, beta = gamma = 16, so gamma / alpha = 1/4 (and beta / range
    # = 16 / 64) are exact in binary64.  With lo = 0 and hi = 64 a key x sits
    # at p = x / 4 in bin floor(x / 4) at f = (x mod 4) / 4; at the edges and
    # the quarter points of every bin each step of R13 is exact, so the
    # oracle's bucket must equal the rational floor.
    P = oracle.Policy(3, 2, 2, 3, 4, 100, SPLINE)
    g = np.random.Generator(np.random.PCG64(8))
    grid = np.arange(0, 65, dtype=np.float64)              # 0, 1, ..., 64
    rest = g.uniform(0.0, 64.0, 256 - grid.size)
    x = np.concatenate([grid, rest])
    g.shuffle(x)
    L = oracle.level0(x, seed=21, policy=P)
    assert (L["alpha"], L["beta"], L["gamma"]) == (64, 16, 16)
    assert L["status"] == 0
    a, c = L["alpha"], L["gamma"]
    b = [int(v) for v in L["b"]]
    keys, bk = L["keys"], bucket_of_each(L)
    where = {float(v): i for i, v in enumerate(keys)}

    def exact(k, f):
        lo = b[k - 1] if k else 0
        return min(math.floor((lo + f * (b[k] - lo)) / a * c), c)

    for xv in range(0, 65):
        k, f = (16, Fraction(0)) if xv == 64 else (xv // 4, Fraction(xv % 4, 4))
        assert bk[where[float(xv)]] == exact(k, f), xv
    assert max(bk) <= c
