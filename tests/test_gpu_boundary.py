"""The C-ABI boundary on the GPU: the segmented sort with device offsets,
stream ordering of its inputs, the workspace bound against what a context
really allocates, and the status returned by pcf_ctx_sync.

The problem the interface carries out is the paper's (Sec. 3.1: keys in,
the same keys ascending out), for S arrays at once; every output is
compared with the oracle."""
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


def _check_segments(got, x, offs, seed, vals=None, got_v=None):
    for s in range(offs.size - 1):
        a, b = int(offs[s]), int(offs[s + 1])
        if vals is None:
            ref, _ = oracle.sort(x[a:b], seed=seed + s)
        else:
            ref, rv = oracle.sort(x[a:b], vals[a:b], seed=seed + s)
            assert np.array_equal(got_v[a:b], rv), s
        assert np.array_equal(got[a:b], np.ascontiguousarray(ref).view(np.uint64)), s


def test_device_offsets_made_on_the_stream(P):
    # the offsets are produced by a kernel on a side stream and the sort is
    # issued on that stream at once: the library reads them in stream order
    ctx = P.Context(0)
    x, offs, _ = W.batched_f64(60, seed=21, lo_exp=2.0, hi_exp=17.0)
    t = torch.from_numpy(x).cuda()
    out = torch.empty_like(t)
    lens = torch.from_numpy(np.diff(offs).astype(np.int64)).cuda()
    side = torch.cuda.Stream()
    torch.cuda.synchronize()
    with torch.cuda.stream(side):
        torch.cuda._sleep(2_000_000)  # a slow producer ahead of the offsets
        d_offs = torch.zeros(lens.numel() + 1, dtype=torch.int64, device="cuda")
        d_offs[1:] = torch.cumsum(lens, 0)
        ctx.sort_segmented_dev(t, d_offs, keys_out=out, key_type="f64", seed=5, stream=side)
    torch.cuda.synchronize()
    _check_segments(out.cpu().numpy().view(np.uint64), x, offs, 5)
    assert ctx.sync(side) == 0
    ctx.close()


def test_device_offsets_pairs_and_equality_with_host_offsets(P):
    ctx = P.Context(0)
    x, offs, _ = W.batched_f64(40, seed=22, lo_exp=3.0, hi_exp=16.0)
    x = np.round(x, 2)
    v = np.arange(x.size, dtype=np.uint32)
    t, tv = torch.from_numpy(x).cuda(), torch.from_numpy(v.view(np.int32)).cuda()
    ko, vo = torch.empty_like(t), torch.empty_like(tv)
    d_offs = torch.from_numpy(offs.astype(np.int64)).cuda()
    ctx.sort_segmented_dev(t, d_offs, vals_in=tv, keys_out=ko, vals_out=vo, key_type="f64",
                           seed=1)
    torch.cuda.synchronize()
    k1, v1 = ko.cpu().numpy().view(np.uint64).copy(), vo.cpu().numpy().view(np.uint32).copy()
    ctx.sort_segmented(t, offs, vals_in=tv, keys_out=ko, vals_out=vo, key_type="f64", seed=1)
    torch.cuda.synchronize()
    assert np.array_equal(k1, ko.cpu().numpy().view(np.uint64))
    assert np.array_equal(v1, vo.cpu().numpy().view(np.uint32))
    _check_segments(k1, x, offs, 1, vals=v, got_v=v1)
    ctx.close()


def test_device_offsets_rejected_with_nothing_written(P):
    ctx = P.Context(0)
    x = W.f64_keys("normal", 5000, 3)
    t = torch.from_numpy(x).cuda()
    out = torch.zeros_like(t)
    for bad in ([0, 3000, 2000, 5000], [1, 2000, 5000], [0, 2000, 6000]):
        d = torch.tensor(bad, dtype=torch.int64, device="cuda")
        with pytest.raises(P.PcfError) as ei:
            ctx.sort_segmented_dev(t, d, keys_out=out, key_type="f64")
        assert ei.value.code == 1
    torch.cuda.synchronize()
    assert int(torch.count_nonzero(out)) == 0
    with pytest.raises(ValueError):  # 4-byte offsets
        ctx.sort_segmented_dev(t, torch.tensor([0, 5000], dtype=torch.int32, device="cuda"),
                               keys_out=out, key_type="f64")
    ctx.close()


def test_sync_reports_the_last_status(P):
    ctx = P.Context(0)
    assert ctx.sync() == 0
    x = W.f64_keys("uniform", 100000, 2)
    x[500] = np.nan
    t = torch.from_numpy(x).cuda()
    with pytest.raises(P.PcfError):
        ctx.sort_keys(t, torch.empty_like(t), key_type="f64")
    assert ctx.sync() == 2
    ctx.sort_keys(t[:400], torch.empty_like(t[:400]), key_type="f64")
    assert ctx.sync() == 0
    ctx.close()


CASES = [("normal", 10**7, 1, False), ("lognormal", 10**7, 1, False),
         ("mixture", 3 * 10**6, 1, True), ("zipf", 2**22, 1, True),
         ("batched", 0, 300, False), ("small", 0, 5000, False)]


@pytest.mark.parametrize("case", CASES, ids=[c[0] for c in CASES])
def test_workspace_bound_holds(P, case):
    # a fresh context holds no more than pcf_workspace_bytes after the sort
    kind, n, S, pairs = case
    ctx = P.Context(0)
    if kind == "batched":
        x, offs, _ = W.batched_f64(S, seed=31, lo_exp=8.0, hi_exp=19.0)
    elif kind == "small":
        x, offs, _ = W.batched_f64(S, seed=32, lo_exp=4.0, hi_exp=12.0)
    elif kind == "zipf":
        x = W.zipf_u64(n, seed=33, n_values=5000)
        offs = np.array([0, n], dtype=np.int64)
    else:
        x = W.f64_keys(kind, n, 34)
        offs = np.array([0, n], dtype=np.int64)
    kt = "u64" if x.dtype == np.uint64 else "f64"
    t = torch.from_numpy(x if kt == "f64" else x.view(np.int64)).cuda()
    out = torch.empty_like(t)
    if pairs:
        v = torch.arange(x.size, dtype=torch.int32, device="cuda")
        ctx.sort_segmented(t, offs, vals_in=v, keys_out=out, vals_out=torch.empty_like(v),
                           key_type=kt)
    else:
        ctx.sort_segmented(t, offs, keys_out=out, key_type=kt)
    torch.cuda.synchronize()
    held = ctx.workspace_held()
    bound = ctx.workspace_bytes(int(offs[-1]), offs.size - 1, key_type=kt, pairs=pairs)
    assert 0 < held <= bound, (held, bound)
    ctx.close()
