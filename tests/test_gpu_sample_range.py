"""GPU parity of the sample-range policy (the bins span the alpha samples'
range, reading R14) against the oracle run with the same policy: level-0
bucket sizes bit for bit (keys outside the samples' range included), and
whole sorts through the global levels and both on-chip kernels, with both
CDF models; NaN keys are still rejected with the output untouched."""
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


@pytest.fixture(scope="module", params=[("pcf", 1024), ("pcf", 4096), ("spline", 4096)])
def setup(P, request):
    model, cap = request.param
    c = P.Context(0, tuning=dict(leaf_cap=cap))
    c.set_policy(model=model, range_mode="sample")
    pol = oracle.paper_policy(model=oracle.MODEL_SPLINE if model == "spline" else oracle.MODEL_PCF,
                              range_mode=oracle.RANGE_SAMPLE)
    yield c, pol
    c.close()


def _dev(x):
    return torch.from_numpy(x if x.dtype == np.float64 else x.view(np.int64)).cuda()


def _bits(a):
    return np.ascontiguousarray(a).view(np.uint64)


def test_level0_counts_match_oracle(setup):
    ctx, pol = setup
    g = np.random.Generator(np.random.PCG64(6))
    arrays = [W.f64_keys("normal", 10**6, 1), W.f64_keys("lognormal", 200003, 2),
              np.where(g.random(50000) < 0.999, 5.0, g.normal(size=50000)),  # equal samples
              W.f64_keys("mixture", 7, 3)]
    for abc in [(31622, 31622, 31622), (300, 5000, 20000), (50, 64, 64)]:
        offs = np.zeros(len(arrays) + 1, dtype=np.uint64)
        offs[1:] = np.cumsum([a.size for a in arrays])
        x = np.concatenate(arrays)
        counts = torch.zeros(len(arrays) * (abc[2] + 1), dtype=torch.int32, device="cuda")
        mx = ctx.bucket_sizes(_dev(x), offs, *abc, seed=5, counts_out=counts)
        got = counts.cpu().numpy().view(np.uint32).reshape(len(arrays), abc[2] + 1)
        for s, a in enumerate(arrays):
            ref, st = oracle.bucket_sizes(a, 5 + s, *abc, model=pol.model,
                                          range_mode=oracle.RANGE_SAMPLE)
            if st == 0:
                assert np.array_equal(got[s].astype(np.uint64), ref), (s, abc)
                assert int(mx[s]) == int(ref.max())


@pytest.mark.parametrize("n", [120, 3000, 200001, 10**6])
@pytest.mark.parametrize("dist", ["uniform", "normal", "lognormal", "exponential", "mixture"])
def test_sort_keys(setup, n, dist):
    ctx, pol = setup
    x = W.f64_keys(dist, n, n + 3)
    t = _dev(x)
    out = torch.empty_like(t)
    ctx.sort_keys(t, out, key_type="f64", seed=2)
    torch.cuda.synchronize()
    ref, _ = oracle.sort(x, seed=2, policy=pol)
    assert np.array_equal(out.cpu().numpy().view(np.uint64), _bits(ref))


def test_u64_pairs_and_edges(setup):
    ctx, pol = setup
    g = np.random.Generator(np.random.PCG64(9))
    cases = [W.zipf_u64(400000, seed=3, n_values=5000),
             g.integers(0, 2**64 - 1, size=300000, dtype=np.uint64, endpoint=True)]
    for x in cases:
        v = np.arange(x.size, dtype=np.uint32)
        t, tv = _dev(x), torch.from_numpy(v.view(np.int32)).cuda()
        ko, vo = torch.empty_like(t), torch.empty_like(tv)
        ctx.sort_pairs(t, tv, ko, vo, key_type="u64", seed=1)
        torch.cuda.synchronize()
        rk, rv = oracle.sort(x, v, seed=1, policy=pol)
        assert np.array_equal(ko.cpu().numpy().view(np.uint64), rk)
        assert np.array_equal(vo.cpu().numpy().view(np.uint32), rv)
    # infinities, signed zeros, a heavy value: sample ranges that need the array's
    y = W.f64_keys("normal", 300000, 4)
    y[::1000] = np.inf
    y[7::1000] = -np.inf
    y[::3] = -0.0
    t = _dev(y)
    out = torch.empty_like(t)
    ctx.sort_keys(t, out, key_type="f64")
    torch.cuda.synchronize()
    ref, _ = oracle.sort(y, policy=pol)
    assert np.array_equal(out.cpu().numpy().view(np.uint64), _bits(ref))


def test_nan_rejected_output_untouched(setup, P):
    ctx, _ = setup
    for n, where in [(10**6, 123457), (10**6, 0), (5000, 4999)]:
        x = W.f64_keys("normal", n, 5)
        x[where] = np.nan
        t = _dev(x)
        out = torch.zeros_like(t)
        with pytest.raises(P.PcfError) as ei:
            ctx.sort_keys(t, out, key_type="f64")
        assert ei.value.code == 2
        torch.cuda.synchronize()
        assert int(torch.count_nonzero(out)) == 0
