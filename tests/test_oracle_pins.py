"""Pins the CPU oracle to facts fixed by the paper and by mathematics.

Each test checks the oracle against something other than itself: a
library routine, a brute-force reference, exact rational arithmetic, a
hand-derived fixture or a bound from the paper.
"""
import math
import os
from fractions import Fraction

import numpy as np
import pytest

import oracle
from paper_2405_07122_gb300 import workloads as W

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")
GOLDEN_GAMMA = 0x9E3779B97F4A7C15


def small_tau_policy():
    # same exponents as the paper policy, tau = 4: recursion on tiny inputs
    return oracle.Policy(3, 3, 3, 3, 4, 4)


def gen(kind, n, seed):
    """Inputs for the pins: the paper's distributions plus adversarial ones."""
    g = np.random.Generator(np.random.PCG64(seed))
    if kind in W.DISTRIBUTIONS:
        return W.f64_keys(kind, n, seed)
    if kind == "dups":
        return g.integers(0, 5, n).astype(np.float64) * 0.5
    if kind == "zeros":
        return np.where(g.random(n) < 0.5, -0.0, 0.0) * np.where(g.random(n) < 0.1, 0.0, 1.0) \
            + np.where(g.random(n) < 0.1, g.standard_normal(n) * 1e-310, 0.0)
    if kind == "inf":
        x = g.standard_normal(n)
        x[g.random(n) < 0.05] = np.inf
        x[g.random(n) < 0.05] = -np.inf
        return x
    if kind == "u64":
        return W.fmix64(g.integers(0, 1000, n, dtype=np.uint64))
    if kind == "u64wide":
        return g.integers(0, 2**64 - 1, n, dtype=np.uint64, endpoint=True)
    if kind == "sorted":
        return np.sort(g.standard_normal(n))
    if kind == "reversed":
        return np.sort(g.standard_normal(n))[::-1].copy()
    if kind == "edges":
        return np.arange(n, dtype=np.float64)[::-1].copy() * 0.25
    raise ValueError(kind)


KINDS = list(W.DISTRIBUTIONS) + ["dups", "zeros", "inf", "u64", "u64wide", "sorted", "reversed",
                                 "edges"]


def is_total_order_sorted(keys):
    """Non-decreasing under the IEEE total order, checked with float
    comparisons plus an explicit rule for signed zeros."""
    if keys.dtype == np.uint64:
        return bool(np.all(keys[:-1] <= keys[1:]))
    x = keys
    if not np.all(x[:-1] <= x[1:]):
        return False
    z = x == 0
    neg = np.signbit(x)
    # a -0 may not follow a +0
    bad = z[:-1] & z[1:] & ~neg[:-1] & neg[1:]
    return not bool(np.any(bad))


def same_multiset(a, b):
    return np.array_equal(np.sort(a.view(np.uint64)), np.sort(b.view(np.uint64)))


# --------------------------------------------------------------------------
# parameters, sampling and the bin function
# --------------------------------------------------------------------------

@pytest.mark.parametrize("n", [1, 2, 99, 100, 1000, 10**6, 10**8, 2**28, 2**10, 2**22, 2**12,
                               2**26, 2**32 - 1, 12345678901])
def test_root_floor_is_exact(n):
    # floor(n^{3/4}) by its definition: m^4 <= n^3 < (m+1)^4 (Python integers)
    m = oracle.root_floor(n, 3, 4)
    assert m**4 <= n**3 < (m + 1) ** 4


def test_paper_policy_values():
    # alpha = beta = gamma = delta = floor(n^{3/4}) (Thm. pcf nlogn); known integer roots
    assert oracle.params(10**8) == (10**6,) * 4          # (10^8)^{3/4} = 10^6 exactly
    assert oracle.params(2**28) == (2**21,) * 4          # (2^28)^{3/4} = 2^21 exactly
    assert oracle.params(2**12) == (512,) * 4            # 2^9
    assert oracle.params(10**6) == (31622,) * 4          # 10^{4.5} = 31622.78
    assert oracle.root_floor(1000, 1, 3) == 10
    assert oracle.root_floor(999, 1, 3) == 9
    assert oracle.root_floor(10**18, 1, 2) == 10**9


def test_splitmix64_known_answer():
    # SplitMix64 (Steele, Lea & Flood 2014): the first output from state 0 is
    # mix(0 + 0x9E3779B97F4A7C15) = 0xE220A8397B1DCDAF (reference splitmix64.c).
    assert oracle.splitmix64_mix(GOLDEN_GAMMA) == 0xE220A8397B1DCDAF


def test_splitmix64_is_a_bijection():
    # each step of the output function is invertible: xor-shift by >= 32/2 bits
    # and multiplication by an odd constant modulo 2^64
    M = 2**64 - 1
    inv1 = pow(0xBF58476D1CE4E5B9, -1, 2**64)
    inv2 = pow(0x94D049BB133111EB, -1, 2**64)

    def unxorshift(y, s):
        x = y
        for _ in range(64 // s + 1):
            x = y ^ (x >> s)
        return x & M

    g = np.random.Generator(np.random.PCG64(3))
    for z in [0, 1, M, *map(int, g.integers(0, 2**63, 200, dtype=np.uint64))]:
        y = oracle.splitmix64_mix(z)
        x = unxorshift(y, 31)
        x = (x * inv2) & M
        x = unxorshift(x, 27)
        x = (x * inv1) & M
        x = unxorshift(x, 30)
        assert x == z


def test_sample_indices_uniform():
    # with-replacement uniform sampling: chi-square over 50 cells
    n, alpha = 50, 200000
    idx = oracle.sample_indices(seed=7, depth=1, start=123, n=n, alpha=alpha)
    assert idx.max() < n
    cnt = np.bincount(idx.astype(np.int64), minlength=n)
    chi2 = float(((cnt - alpha / n) ** 2 / (alpha / n)).sum())
    assert chi2 < 100.0  # 49 dof: p ~ 3e-5 at 100
    # different sub-arrays draw different streams
    idx2 = oracle.sample_indices(seed=7, depth=1, start=124, n=n, alpha=64)
    assert not np.array_equal(idx[:64], idx2)


def _golden_bins():
    rows = []
    with open(os.path.join(GOLDEN, "bin_edges.txt")) as f:
        for line in f:
            if line.startswith("#") or not line.strip():
                continue
            kt, lo, hi, beta, x, exp = line.split()
            rows.append((kt, lo, hi, int(beta), x, int(exp)))
    return rows


@pytest.mark.parametrize("row", _golden_bins())
def test_bin_hand_derived(row):
    kt, lo, hi, beta, x, exp = row
    if kt == "f64":
        b = lambda s: np.array([float(s)]).view(np.uint64)
        got = oracle.bins(oracle.KEY_F64, int(b(lo)[0]), int(b(hi)[0]), beta, b(x))
    else:
        got = oracle.bins(oracle.KEY_U64, int(lo), int(hi), beta,
                          np.array([int(x)], dtype=np.uint64))
    assert int(got[0]) == exp


def test_bin_degenerate_ranges():
    f = lambda v: int(np.array([v]).view(np.uint64)[0])
    one = np.array([1.0]).view(np.uint64)
    assert oracle.bins(0, f(1.0), f(1.0), 10, one) is None           # zero range
    assert oracle.bins(0, f(-0.0), f(0.0), 10, one) is None          # -0/+0 only
    assert oracle.bins(0, f(0.0), f(np.inf), 10, one) is None        # infinite range
    assert oracle.bins(0, f(-1e308), f(1e308), 10, one) is None      # range overflows
    assert oracle.bins(0, f(0.0), f(5e-324), 10, one) is None        # scale overflows


@pytest.mark.parametrize("seed", range(4))
def test_bin_matches_exact_rational_formula(seed):
    # Sec. 3.3's formula in exact rational arithmetic; the binary64 reading may
    # only differ where the exact value lies within 2^-40 (relative) of an
    # integer, and then by one bin.
    g = np.random.Generator(np.random.PCG64(seed))
    x = g.standard_normal(4000) * 10.0 ** g.uniform(-3, 3)
    lo, hi = x.min(), x.max()
    beta = int(g.integers(1, 2**21))
    got = oracle.bins(0, int(np.array([lo]).view(np.uint64)[0]),
                      int(np.array([hi]).view(np.uint64)[0]), beta, x.view(np.uint64))
    r = Fraction(hi) - Fraction(lo)
    for xi, gi in zip(x, got):
        v = (Fraction(xi) - Fraction(lo)) * beta / r
        exact = min(beta, math.floor(v))
        if int(gi) != exact:
            near = abs(v - round(v)) <= abs(v) * Fraction(1, 2**40) + Fraction(1, 2**60)
            assert near and abs(int(gi) - exact) == 1


def test_bin_is_monotone():
    g = np.random.Generator(np.random.PCG64(11))
    x = np.sort(np.concatenate([g.standard_normal(20000), g.lognormal(0, 3, 2000), [0.0, -0.0]]))
    lo, hi = x[0], x[-1]
    got = oracle.bins(0, int(np.array([lo]).view(np.uint64)[0]),
                      int(np.array([hi]).view(np.uint64)[0]), 100000, x.view(np.uint64))
    assert np.all(np.diff(got.astype(np.int64)) >= 0)
    assert got[0] == 0 and got[-1] <= 100000


# --------------------------------------------------------------------------
# one bucketing level
# --------------------------------------------------------------------------

@pytest.mark.parametrize("kind,n", [("uniform", 3000), ("normal", 5000), ("lognormal", 2000),
                                    ("mixture", 4000), ("u64", 3000), ("dups", 1000)])
def test_level0_b_matches_definition(kind, n):
    x = gen(kind, n, 5)
    L = oracle.level0(x, seed=9)
    assert L["status"] == 0
    alpha, beta = L["alpha"], L["beta"]
    a = x.view(np.uint64)[L["sample_idx"].astype(np.int64)]
    kt = oracle.KEY_F64 if x.dtype == np.float64 else oracle.KEY_U64
    sbins = oracle.bins(kt, L["lo_bits"], L["hi_bits"], beta, a)
    # b_i = |{j : i(a_j) <= i}|, straight from the definition (O(alpha*beta))
    b_ref = oracle.brute_cumulative_counts(sbins, beta)
    assert np.array_equal(L["b"], b_ref)
    assert L["b"][-1] == alpha and np.all(np.diff(L["b"].astype(np.int64)) >= 0)


def test_level0_T_is_the_paper_bucket_formula():
    # j = floor(F(x) gamma) with F = b_{i(x)}/alpha, in exact rationals, for a
    # policy where alpha != gamma (a = 3/4, c = 1/2)
    P = oracle.Policy(3, 3, 2, 3, 4, 100)
    x = gen("normal", 5000, 2)
    L = oracle.level0(x, seed=1, policy=P)
    assert L["alpha"] != L["gamma"]
    for bk, tk in zip(L["b"], L["T"]):
        assert int(tk) == math.floor(Fraction(int(bk), L["alpha"]) * L["gamma"])
    # paper policy: alpha == gamma, so the bucket of bin k is b_k itself
    L = oracle.level0(x, seed=1)
    assert np.array_equal(L["T"], L["b"])


@pytest.mark.parametrize("kind", ["uniform", "normal", "exponential", "mixture", "dups", "u64",
                                  "zeros"])
def test_level0_buckets_ordered_and_stable(kind):
    x = gen(kind, 4000, 3)
    if kind == "zeros":
        x = np.concatenate([x, [1.0, -1.0]])
    idx = np.arange(x.size, dtype=np.uint32)
    L = oracle.level0(x, vals=idx, seed=4)
    if L["status"] != 0:
        pytest.skip("level not bucketed")
    counts = L["counts"].astype(np.int64)
    assert counts.sum() == x.size
    assert same_multiset(L["keys"], x)
    off = np.concatenate([[0], np.cumsum(counts)])
    ks, vs = L["keys"], L["vals"]
    prev_max = None
    for j in range(counts.size):
        if counts[j] == 0:
            continue
        seg = ks[off[j]:off[j + 1]]
        # Append keeps input order inside a bucket
        assert np.all(np.diff(vs[off[j]:off[j + 1]].astype(np.int64)) > 0)
        # p in c_j, q in c_k, j < k  =>  p <= q  (Sec. 3.2; equal only for +-0)
        if prev_max is not None:
            assert prev_max <= seg.min()
        prev_max = seg.max()


def test_failure_lemma_uniform():
    # Lemma pcf-divide-success-prob with sigma1 = sigma2 (uniform): at n = 10^6
    # under the paper policy K = gamma*delta/(2n) - 2 ~ 498 and the bound on
    # Pr[exists j: |c_j| > delta] is (2n/delta) exp(-(alpha K / 2 gamma)(1-1/K)^2),
    # about e^-244: no level-0 bucket may exceed delta.
    n = 10**6
    alpha, beta, gamma, delta = oracle.params(n)
    K = gamma * delta / (2 * n) - 2 * gamma / beta
    log_bound = math.log(2 * n / delta) - (alpha * K / (2 * gamma)) * (1 - 1 / K) ** 2
    assert K >= 1 and log_bound < -200
    for seed in range(6):
        x = W.f64_keys("uniform", n, 100 + seed)
        L = oracle.level0(x, seed=seed)
        assert int(L["counts"].max()) <= delta


# --------------------------------------------------------------------------
# the full sort
# --------------------------------------------------------------------------

def test_sort_matches_insertion_sort_every_n():
    # every n in 2..2000, generators rotating; paper policy and tau = 4
    for n in range(2, 2001):
        kind = KINDS[n % len(KINDS)]
        x = gen(kind, n, n)
        v = np.arange(n, dtype=np.uint32)
        ref_k, ref_v = oracle.insertion_sort(x, v)
        for P in (oracle.paper_policy(), small_tau_policy()):
            k, vv = oracle.sort(x, v, seed=n, policy=P)
            assert np.array_equal(k.view(np.uint64), ref_k.view(np.uint64)), (kind, n)
            assert np.array_equal(vv, ref_v), (kind, n)


@pytest.mark.parametrize("kind", KINDS)
def test_sort_matches_numpy(kind):
    n = 200000
    x = gen(kind, n, 17)
    v = np.arange(n, dtype=np.uint32)
    k, vv, st = oracle.sort(x, v, seed=3, with_stats=True)
    assert same_multiset(k, x)
    assert is_total_order_sorted(k)
    if x.dtype == np.float64:
        assert np.array_equal(k, np.sort(x))  # numerically (library sort)
    else:
        assert np.array_equal(k, np.sort(x))
        # stable: equal keys keep increasing payloads == numpy stable argsort
        assert np.array_equal(vv, np.argsort(x, kind="stable").astype(np.uint32))
    # payload follows its key
    assert np.array_equal(x.view(np.uint64)[vv.astype(np.int64)], k.view(np.uint64))


def test_pairs_stable_on_duplicates():
    x = W.zipf_u64(300000, seed=5, n_values=1000)
    v = np.arange(x.size, dtype=np.uint32)
    k, vv, st = oracle.sort(x, v, seed=1, with_stats=True)
    assert np.array_equal(vv, np.argsort(x, kind="stable").astype(np.uint32))
    assert st["n_single"] > 0 or st["n_fallback"] > 0


@pytest.mark.parametrize("n,dist", [(10**6, "uniform"), (10**6, "normal"), (300000, "lognormal")])
def test_depth_bound(n, dist):
    # proof of Lemma nlogn: a bucket at depth i has fewer than n^{d^i} keys, and
    # recursion stops below tau, so depth <= min{i : n^{(3/4)^i} <= tau}
    x = W.f64_keys(dist, n, 1)
    _, _, st = oracle.sort(x, seed=2, with_stats=True)
    bound = 0
    while n ** (0.75 ** bound) > 100:
        bound += 1
    assert st["max_depth"] <= bound
    assert st["recursed_violations"] == 0


def test_edge_cases():
    cases = [
        np.array([], dtype=np.float64),
        np.array([1.5]),
        np.array([2.0, 1.0]),
        np.full(500, 3.25),
        np.array([1.0, 2.0] * 300),
        np.array([0.0, -0.0] * 150 + [-0.0]),
        np.array([5e-324, -5e-324, 0.0, -0.0, 2.2250738585072014e-308] * 40),
        np.array([np.inf, -np.inf, 1.0, 0.0] * 50),
        np.arange(1000, dtype=np.float64),
        np.arange(1000, dtype=np.float64)[::-1].copy(),
        W.inject_duplicates(W.f64_keys("normal", 5000, 3), seed=4),
        np.array([0, 2**64 - 1, 1, 2**63] * 100, dtype=np.uint64),
        np.array([1e308, -1e308] * 200 + [0.0]),
    ]
    for x in cases:
        v = np.arange(x.size, dtype=np.uint32)
        for P in (oracle.paper_policy(), small_tau_policy()):
            k, vv = oracle.sort(x, v, seed=1, policy=P)
            rk, rv = oracle.insertion_sort(x, v)
            assert np.array_equal(k.view(np.uint64), rk.view(np.uint64))
            assert np.array_equal(vv, rv)


def test_nan_rejected():
    with pytest.raises(ValueError):
        oracle.sort(np.array([1.0, np.nan, 0.0] * 100))


def test_seed_independent_output():
    # the sorted output is unique, so the sampling seed cannot change it
    x = W.f64_keys("mixture", 100000, 9)
    a, _ = oracle.sort(x, seed=1)
    b, _ = oracle.sort(x, seed=2)
    assert np.array_equal(a.view(np.uint64), b.view(np.uint64))


def _total_order_u64(x):
    # IEEE-754 total order of binary64 bit patterns as unsigned integers
    b = np.ascontiguousarray(x).view(np.uint64)
    neg = (b >> np.uint64(63)) == 1
    return np.where(neg, ~b, b | np.uint64(1 << 63))


@pytest.mark.parametrize("n", [2, 17, 1000, 4097, 100003])
def test_std_sort_is_a_stable_sort(n):
    # Standard-Sort (R7) against numpy's stable argsort of the total-order
    # keys: heavy duplicates, signed zeros and infinities, values carried
    g = np.random.Generator(np.random.PCG64(n))
    x = np.round(g.normal(size=n) * 3.0)
    x[g.random(n) < 0.1] = -0.0
    x[g.random(n) < 0.1] = 0.0
    x[g.random(n) < 0.02] = np.inf
    x[g.random(n) < 0.02] = -np.inf
    v = np.arange(n, dtype=np.uint32)
    k, vv = oracle.std_sort(x, v)
    order = np.argsort(_total_order_u64(x), kind="stable")
    assert np.array_equal(k.view(np.uint64), x[order].view(np.uint64))
    assert np.array_equal(vv, v[order])
    # unsigned keys: plain unsigned order
    u = g.integers(0, 50, size=n, dtype=np.uint64) * np.uint64(2**58)
    ku, vu = oracle.std_sort(u, v)
    order = np.argsort(u, kind="stable")
    assert np.array_equal(ku, u[order]) and np.array_equal(vu, v[order])


def three_value_input(n_lo, n_mid, n_hi, seed):
    """n_lo copies of 1.0, n_mid of 2.0 and n_hi of 3.0, shuffled."""
    x = np.concatenate([np.full(n_lo, 1.0), np.full(n_mid, 2.0), np.full(n_hi, 3.0)])
    np.random.Generator(np.random.PCG64(seed)).shuffle(x)
    return x


def test_failure_guard_fires_at_exactly_delta():
    # Alg. 1 sends a bucket to Standard-Sort when |c_j| >= delta (reading R8),
    # with delta the parent's.  n = 10^4: alpha = beta = gamma = delta = 1000.
    # Three values 1, 2, 3: bins 0, beta/2 and beta; with alpha = gamma the
    # bucket of bin k is b_k, so the three values fall in three buckets (b_0,
    # b_{beta/2}, alpha) as long as 2 and 3 are each sampled (a 1000-draw
    # sample misses a value with over 10% of the keys with probability
    # below 1e-45).  Sizes 1000 (= delta), 999 (= delta - 1) and 8001: the
    # first and the last reach the guard, the middle one is recursed (one
    # value: sorted at once).
    n = 10**4
    assert oracle.params(n) == (1000, 1000, 1000, 1000)
    x = three_value_input(1000, 999, 8001, 11)
    k, _, st = oracle.sort(x, seed=4, with_stats=True)
    assert np.array_equal(k, np.sort(x))
    assert st["n_fallback"] == 2
    assert st["fallback_keys"] == 1000 + 8001
    assert st["n_bucketings"] == 1 and st["n_single"] == 1
    # one key fewer in the first bucket: below the guard, recursed instead
    x = three_value_input(999, 999, 8002, 12)
    _, _, st = oracle.sort(x, seed=4, with_stats=True)
    assert st["n_fallback"] == 1 and st["fallback_keys"] == 8002
    assert st["n_single"] == 2
