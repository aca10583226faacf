"""GPU parity of Spline Learned Sort (the spline CDF model of App. A.5 in
every bucketing step) against the oracle run with the same model: level-0
bucket sizes bit for bit, and whole sorts (unique output; stable pairs)
through the global levels and both on-chip kernels."""
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


@pytest.fixture(scope="module", params=[1024, 4096])
def ctx(P, request):
    c = P.Context(0, tuning=dict(leaf_cap=request.param))
    c.set_policy(model="spline")
    yield c
    c.close()


def _dev(x):
    return torch.from_numpy(x if x.dtype == np.float64 else x.view(np.int64)).cuda()


def _bits(a):
    return np.ascontiguousarray(a).view(np.uint64)


SPLINE = oracle.paper_policy(model=oracle.MODEL_SPLINE)


@pytest.mark.parametrize("abc", [(31622, 31622, 31622), (1000, 5000, 8191), (5000, 300, 20000),
                                 (7, 3, 64)])
def test_level0_counts_match_oracle(ctx, abc):
    arrays = [W.f64_keys(d, n, i + 3) for i, (d, n) in
              enumerate([("uniform", 10**6), ("normal", 200003), ("lognormal", 50000),
                         ("mixture", 3)])]
    g = np.random.Generator(np.random.PCG64(4))
    u = g.integers(0, 2**64 - 1, size=100000, dtype=np.uint64, endpoint=True)
    for group in (arrays, [u, W.zipf_u64(70000, seed=2, n_values=3000)]):
        offs = np.zeros(len(group) + 1, dtype=np.uint64)
        offs[1:] = np.cumsum([a.size for a in group])
        x = np.concatenate(group)
        counts = torch.zeros(len(group) * (abc[2] + 1), dtype=torch.int32, device="cuda")
        mx = ctx.bucket_sizes(_dev(x), offs, *abc, seed=9, counts_out=counts)
        got = counts.cpu().numpy().view(np.uint32).reshape(len(group), abc[2] + 1)
        for s, a in enumerate(group):
            ref, st = oracle.bucket_sizes(a, 9 + s, *abc, model=oracle.MODEL_SPLINE)
            assert st == 0
            assert np.array_equal(got[s].astype(np.uint64), ref), (s, abc)
            assert int(mx[s]) == int(ref.max())


@pytest.mark.parametrize("n", [150, 1000, 4000, 100003, 10**6])
@pytest.mark.parametrize("dist", ["uniform", "normal", "lognormal", "exponential", "mixture"])
def test_sort_keys(ctx, n, dist):
    x = W.f64_keys(dist, n, n + 5)
    t = _dev(x)
    out = torch.empty_like(t)
    ctx.sort_keys(t, out, key_type="f64", seed=1)
    torch.cuda.synchronize()
    ref, _ = oracle.sort(x, seed=1, policy=SPLINE)
    assert np.array_equal(out.cpu().numpy().view(np.uint64), _bits(ref))


def test_sort_u64_and_pairs_stable(ctx):
    x = W.zipf_u64(600000, seed=12, n_values=20000)
    v = np.arange(x.size, dtype=np.uint32)
    t, tv = _dev(x), torch.from_numpy(v.view(np.int32)).cuda()
    ko, vo = torch.empty_like(t), torch.empty_like(tv)
    ctx.sort_pairs(t, tv, ko, vo, key_type="u64", seed=3)
    torch.cuda.synchronize()
    rk, rv = oracle.sort(x, v, seed=3, policy=SPLINE)
    assert np.array_equal(ko.cpu().numpy().view(np.uint64), rk)
    assert np.array_equal(vo.cpu().numpy().view(np.uint32), rv)


def test_segmented(ctx):
    keys, offs, _ = W.batched_f64(60, seed=8, lo_exp=6.0, hi_exp=17.0)
    t = _dev(keys)
    out = torch.empty_like(t)
    ctx.sort_segmented(t, offs, keys_out=out, key_type="f64", seed=2)
    torch.cuda.synchronize()
    got = out.cpu().numpy().view(np.uint64)
    for s in range(len(offs) - 1):
        a, b = int(offs[s]), int(offs[s + 1])
        ref, _ = oracle.sort(keys[a:b], seed=2 + s, policy=SPLINE)
        assert np.array_equal(got[a:b], _bits(ref)), s
