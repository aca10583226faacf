"""The bucketing-failure experiment of Sec. 4.2 on the CPU side: the exact
grid parameters, the closed form of Lemma pcf-divide-success-prob, and the
oracle's bucketing with given alpha, beta, gamma checked against the lemma
and against the oracle's own level-0 path."""
import math

import numpy as np

import oracle
from paper_2405_07122_gb300 import failsweep as F
from paper_2405_07122_gb300 import workloads as W


def test_floor_pow_exact():
    # 10^6 ^ (k/20) = 10^(0.3 k): integers at k = 10 (10^3), else irrational
    assert F.floor_pow(10**6, 10) == 1000
    assert F.floor_pow(10**6, 15) == 31622       # 10^4.5  = 31622.77...
    assert F.floor_pow(10**6, 19) == 501187      # 10^5.7  = 501187.23...
    assert F.floor_pow(10**6, 1) == 1            # 10^0.3  = 1.99...
    assert F.floor_pow(10**6, 5) == 31           # 10^1.5  = 31.62...
    assert F.floor_pow(2**20, 10) == 2**10
    for n in (7, 1000, 123457, 10**6):
        for k in range(1, 20):
            m = F.floor_pow(n, k)
            assert m ** 20 <= n ** k < (m + 1) ** 20
    # at exponent 3/4 the grid agrees with the policy's exact floor
    assert F.setting(10**6, .75, .75, .75, .75) == tuple(oracle.params(10**6))


def test_lemma_bound_closed_form():
    n = 10**6
    p = F.setting(n, .75, .75, .75, .75)
    # by hand: K = 31622^2 / 2e6 - 2 = 497.975; alpha K / (2 gamma) = 248.99;
    # (1 - 1/K)^2 = 0.995988; log(2n / delta) = log(63.246) = 4.147;
    # log bound = 4.147 - 248.99 * 0.995988 = -243.84
    assert math.isclose(math.log(F.lemma_bound(n, *p)), -243.84, abs_tol=0.01)
    # K < 1: the lemma does not apply
    assert F.lemma_bound(n, *F.setting(n, .75, .75, .3, .3)) is None
    # the bound falls as alpha grows (other parameters fixed)
    b1 = F.lemma_bound(n, *F.setting(n, .55, .75, .75, .75))
    b2 = F.lemma_bound(n, *F.setting(n, .65, .75, .75, .75))
    assert b1 is not None and b2 is not None and b2 < b1


def test_oracle_bucket_sizes_matches_level0():
    x = W.f64_keys("normal", 200003, 5)
    L = oracle.level0(x, seed=7)
    counts, status = oracle.bucket_sizes(x, 7, L["alpha"], L["beta"], L["gamma"])
    assert status == 0 and np.array_equal(counts, L["counts"])
    assert int(counts.sum()) == x.size
    c1, s1 = oracle.bucket_sizes(np.full(500, 2.5), 0, 10, 10, 10)
    assert s1 == 1 and int(c1.sum()) == 0


def test_oracle_failure_frequency_follows_the_lemma():
    n, R = 10**6, 4
    xs = [W.f64_keys("uniform", n, 300 + r) for r in range(R)]

    def freq(a, b, c, d):
        al, be, ga, de = F.setting(n, a, b, c, d)
        return sum(int(oracle.bucket_sizes(x, r, al, be, ga)[0].max()) > de
                   for r, x in enumerate(xs)) / R
    # the paper policy: bound e^-244, no failure
    assert freq(.75, .75, .75, .75) == 0.0
    # delta = n^0.2 = 15 below the mean bucket size n / gamma = 31.6: always
    assert freq(.75, .75, .75, .2) == 1.0
    # gamma = n^0.3 = 63 buckets of ~15,900 keys against delta = 1000
    assert freq(.75, .75, .3, .5) == 1.0
    # alpha = n^0.9: a bound of about 1e-4 once K >= 1, no failure
    al, be, ga, de = F.setting(n, .9, .75, .75, .75)
    assert F.lemma_bound(n, al, be, ga, de) < 1e-100
    assert freq(.9, .75, .75, .75) == 0.0
