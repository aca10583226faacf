"""GPU parity of the bucketing-only entry point (pcf_bucket_sizes) against
the oracle's bucketing with the same alpha, beta, gamma: every bucket size
of every array, bit for bit, and the failure frequency of the Sec. 4.2
experiment at settings where Lemma pcf-divide-success-prob decides it."""
import numpy as np
import pytest

import oracle
from paper_2405_07122_gb300 import failsweep as F
from paper_2405_07122_gb300 import workloads as W

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")


@pytest.fixture(scope="module")
def ctx():
    from paper_2405_07122_gb300 import build as pcf_build
    pcf_build.build()
    from paper_2405_07122_gb300 import pcfsort
    c = pcfsort.Context(0)
    yield c
    c.close()


def _dev(x):
    return torch.from_numpy(x if x.dtype == np.float64 else x.view(np.int64)).cuda()


def _check(ctx, arrays, alpha, beta, gamma, seed):
    offs = np.zeros(len(arrays) + 1, dtype=np.uint64)
    offs[1:] = np.cumsum([a.size for a in arrays])
    x = np.concatenate(arrays)
    counts = torch.zeros(len(arrays) * (gamma + 1), dtype=torch.int32, device="cuda")
    mx = ctx.bucket_sizes(_dev(x), offs, alpha, beta, gamma, seed=seed, counts_out=counts)
    got = counts.cpu().numpy().view(np.uint32).reshape(len(arrays), gamma + 1)
    for s, a in enumerate(arrays):
        ref, status = oracle.bucket_sizes(a, seed + s, alpha, beta, gamma)
        if status == 0:
            assert np.array_equal(got[s].astype(np.uint64), ref), (s, alpha, beta, gamma)
            assert int(mx[s]) == int(ref.max())
        else:
            assert int(mx[s]) == a.size and not got[s].any()
    return mx


@pytest.mark.parametrize("abc", [(31622, 31622, 31622), (1, 1, 1), (7, 3, 5000),
                                 (501187, 1000, 63), (1000, 501187, 501187),
                                 (100, 100000, 8191), (100, 100000, 8192)])
def test_counts_match_oracle_f64(ctx, abc):
    # gamma + 1 up to 8192 counts in shared memory first, above that directly
    arrays = [W.f64_keys(d, n, i + 11) for i, (d, n) in
              enumerate([("uniform", 10**6), ("normal", 300001), ("lognormal", 2),
                         ("mixture", 77777), ("exponential", 5000)])]
    _check(ctx, arrays, *abc, seed=3)


def test_counts_match_oracle_u64_and_degenerate(ctx):
    g = np.random.Generator(np.random.PCG64(8))
    arrays = [g.integers(0, 2**64 - 1, size=200000, dtype=np.uint64, endpoint=True),
              np.full(1000, 12345, dtype=np.uint64),          # one value
              W.zipf_u64(100000, seed=9, n_values=500)]
    mx = _check(ctx, arrays, 4000, 4000, 4000, seed=1)
    assert int(mx[1]) == 1000
    inf = np.full(3000, np.inf)
    inf[::2] = -np.inf                                        # degenerate range
    mx = _check(ctx, [W.f64_keys("normal", 4000, 2), inf], 300, 300, 300, seed=0)
    assert int(mx[1]) == 3000


def test_failure_frequency_matches_the_lemma(ctx):
    n, R = 10**6, 20
    arrays = [W.f64_keys("uniform", n, 500 + r) for r in range(R)]
    offs = np.arange(R + 1, dtype=np.uint64) * n
    keys = _dev(np.concatenate(arrays))
    for e, expect in [((.75, .75, .75, .75), 0.0), ((.9, .75, .75, .75), 0.0),
                      ((.75, .75, .75, .2), 1.0), ((.75, .75, .3, .5), 1.0)]:
        al, be, ga, de = F.setting(n, *e)
        mx = ctx.bucket_sizes(keys, offs, al, be, ga)
        assert float((mx > de).mean()) == expect, e
    # a setting in between: the GPU's per-array decisions equal the oracle's
    al, be, ga, de = F.setting(n, .45, .75, .75, .75)
    mx = ctx.bucket_sizes(keys, offs, al, be, ga)
    for r in (0, 7, 19):
        ref, _ = oracle.bucket_sizes(arrays[r], r, al, be, ga)
        assert int(mx[r]) == int(ref.max())
