"""pcf_sort_segmented_static, the allocation-free batched sort of small
arrays: two calls in a row, each equal to pcf_sort_segmented on the same
input and to the oracle, no change in free device memory across them, and
the documented rejections.  (Collected last: it must pass both alone and
after every other GPU test.)"""
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


def _batch(seed, S, max_len, kt):
    g = np.random.Generator(np.random.PCG64(seed))
    lens = g.integers(0, max_len + 1, size=S)
    # the degenerate and boundary sizes: empty, one key, tau - 1, tau, the cap
    lens[:5] = [0, 1, 99, 100, max_len]
    offs = np.zeros(S + 1, dtype=np.uint64)
    offs[1:] = np.cumsum(lens)
    n = int(offs[-1])
    dist = W.DISTRIBUTIONS[seed % len(W.DISTRIBUTIONS)]
    x = W.request_keys(n, kt, dist, seed=seed)
    return x, offs


def _dev(x, kt):
    return torch.from_numpy(x if kt == "f64" else x.view(np.int64)).cuda()


@pytest.mark.parametrize("kt", ["f64", "u64"])
def test_two_calls_match_segmented_and_oracle(P, kt):
    ctx = P.Context(0)
    batches = [_batch(71, 900, 1024, kt), _batch(72, 3000, 700, kt)]
    free = []
    for i, (x, offs) in enumerate(batches):
        n = int(offs[-1])
        d_in = _dev(x, kt)
        d_offs = torch.from_numpy(offs.view(np.int64)).cuda()
        got = torch.empty_like(d_in)
        torch.cuda.synchronize()
        free.append(torch.cuda.mem_get_info()[0])
        P.sort_segmented_static(d_in, d_offs, n, keys_out=got, key_type=kt, seed=5 + i)
        torch.cuda.synchronize()
        free.append(torch.cuda.mem_get_info()[0])
        ref_dev = torch.empty_like(d_in)
        ctx.sort_segmented(d_in, offs, keys_out=ref_dev, key_type=kt, seed=5 + i)
        torch.cuda.synchronize()
        g = got.cpu().numpy().view(np.uint64)
        assert np.array_equal(g, ref_dev.cpu().numpy().view(np.uint64))
        for s in range(len(offs) - 1):
            a, b = int(offs[s]), int(offs[s + 1])
            ref, _ = oracle.sort(x[a:b])
            assert np.array_equal(g[a:b], ref.view(np.uint64)), s
        # in place gives the same
        P.sort_segmented_static(d_in, d_offs, n, key_type=kt, seed=5 + i)
        torch.cuda.synchronize()
        assert np.array_equal(d_in.cpu().numpy().view(np.uint64), g)
    ctx.close()
    # the second call (the first may load the module) allocates nothing
    assert free[2] == free[3]


def test_rejections(P):
    x = np.sort(W.f64_keys("normal", 4096, 3))
    d = torch.from_numpy(x).cuda()
    out = torch.zeros_like(d)

    def run(offs, n_total):
        o = torch.from_numpy(np.asarray(offs, dtype=np.int64)).cuda()
        with pytest.raises(P.PcfError) as ei:
            P.sort_segmented_static(d, o, n_total, keys_out=out, key_type="f64")
        torch.cuda.synchronize()
        return ei.value.code

    assert run([0, 1025], 1025) == 1                      # an array above the cap
    assert run([0, 10, 5, 20], 20) == 1                   # decreasing offsets
    assert run([0, 10, 20], 30) == 1                      # last offset != n_total
    assert run([3, 10, 20], 20) == 1                      # first offset != 0
    assert int(torch.count_nonzero(out)) == 0  # nothing written
    big = torch.zeros(P.STATIC_MAX_ARRAYS + 2, dtype=torch.int64, device="cuda")
    with pytest.raises(P.PcfError):
        P.sort_segmented_static(d, big, 0, keys_out=out, key_type="f64")
    huge = torch.zeros(P.STATIC_MAX_KEYS + 1, dtype=torch.float64, device="cuda")
    with pytest.raises(P.PcfError):
        P.sort_segmented_static(huge, torch.tensor([0, 1], device="cuda"), P.STATIC_MAX_KEYS + 1,
                                key_type="f64")
    # arguments the binding checks before calling in: n_total beyond the
    # buffers, 4-byte offsets, a non-contiguous tensor
    o2 = torch.tensor([0, 2048, 4096], device="cuda")
    with pytest.raises(ValueError):
        P.sort_segmented_static(d, o2, 4097, keys_out=out, key_type="f64")
    with pytest.raises(ValueError):
        P.sort_segmented_static(d[:100], o2, 4096, keys_out=out, key_type="f64")
    with pytest.raises(ValueError):
        P.sort_segmented_static(d, o2.to(torch.int32), 4096, keys_out=out, key_type="f64")
    with pytest.raises(ValueError):
        P.sort_segmented_static(d[::2], torch.tensor([0, 2048], device="cuda"), 2048,
                                keys_out=out[:2048], key_type="f64")
    # NaN: rejected, output untouched
    y = x[:2000].copy()
    y[777] = np.nan
    dn = torch.from_numpy(y).cuda()
    on = torch.zeros_like(dn)
    with pytest.raises(P.PcfError) as ei:
        P.sort_segmented_static(dn, torch.tensor([0, 1000, 2000], device="cuda"), 2000,
                                keys_out=on, key_type="f64")
    assert ei.value.code == 2
    torch.cuda.synchronize()
    assert int(torch.count_nonzero(on)) == 0
