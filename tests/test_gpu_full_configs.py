"""GPU parity at the benchmark configurations' full sizes.

Every configuration is compared element by element with the oracle (a
sequential PCF Learned Sort, Alg. 1 with the Sec. 3.3 model):
  - four arrays of 10^8 float64 keys (Normal, LogNormal, Exponential, a
    5-Gaussian mixture), keys only;
  - 2^28 Zipf(1.2) u64 keys with u32 payloads (the original index), stable:
    keys and payloads both;
  - 2048 float64 arrays of 2^U(10, 22) keys (about 10^9 in all), through the
    segmented call and through a CUDA-graph replay; the oracle sorts one
    array per host thread (ctypes releases the GIL around its C calls).
Key-value sorts append stably and take every step of Alg. 1 on the GPU too,
so their decision counters (buckets that reached the failure guard |c| >=
delta, their keys, and the Learned-Sort calls that bucketed) must equal the
oracle's.
"""
import concurrent.futures as cf
import os

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


def _bits(a):
    return np.ascontiguousarray(a).view(np.uint64)


SEEDS = {"normal": 1, "lognormal": 2, "exponential": 3, "mixture": 4}


@pytest.mark.parametrize("dist", ["normal", "lognormal", "exponential", "mixture"])
def test_plain_1e8(ctx, dist):
    x = W.f64_keys(dist, 10**8, SEEDS[dist])
    t = torch.from_numpy(x).cuda()
    out = torch.empty_like(t)
    ctx.sort_keys(t, out, key_type="f64", seed=0)
    torch.cuda.synchronize()
    got = out.cpu().numpy().view(np.uint64)
    del t, out
    ref, _ = oracle.sort(x, seed=0)
    assert np.array_equal(got, _bits(ref))


def _decisions(st):
    return st["guard_buckets"], st["guard_keys"], st["bucketings"]


def _oracle_decisions(st):
    return st["n_fallback"], st["fallback_keys"], st["n_bucketings"]


def test_zipf_pairs_2p28(ctx):
    n = 1 << 28
    k = W.zipf_u64(n, seed=5)
    v = np.arange(n, dtype=np.uint32)
    tk = torch.from_numpy(k.view(np.int64)).cuda()
    tv = torch.from_numpy(v.view(np.int32)).cuda()
    ko, vo = torch.empty_like(tk), torch.empty_like(tv)
    ctx.sort_pairs(tk, tv, ko, vo, key_type="u64", seed=0)
    torch.cuda.synchronize()
    st = ctx.last_stats()
    gk = ko.cpu().numpy().view(np.uint64)
    gv = vo.cpu().numpy().view(np.uint32)
    del tk, tv, ko, vo
    rk, rv, ost = oracle.sort(k, v, seed=0, with_stats=True)
    assert np.array_equal(gk, rk)
    assert np.array_equal(gv, rv)
    assert _decisions(st) == _oracle_decisions(ost)
    assert st["guard_buckets"] > 0  # the heavy values reach the guard


def _oracle_segments(x, offs, seed):
    """Oracle sort of every segment, one per host thread."""
    S = offs.size - 1

    def one(s):
        a, b = int(offs[s]), int(offs[s + 1])
        r, _ = oracle.sort(x[a:b], seed=seed + s)
        return s, _bits(r)

    with cf.ThreadPoolExecutor(max_workers=os.cpu_count() or 4) as ex:
        yield from ex.map(one, range(S))


def test_batched_2048_segments(ctx, P):
    x, offs, _ = W.batched_f64(2048, seed=6)
    offs = offs.astype(np.uint64)
    assert x.size > 9 * 10**8
    t = torch.from_numpy(x).cuda()
    out = torch.empty_like(t)
    ctx.sort_segmented(t, offs, keys_out=out, key_type="f64", seed=0)
    torch.cuda.synchronize()
    got_seg = out.cpu().numpy().view(np.uint64)
    # the same batch as a CUDA graph: recorded, then replayed on the same data
    g = P.SortGraph(ctx, t, offs, out, key_type="f64", seed=0)
    out.zero_()
    assert g.launch(), "graph not replayed"
    torch.cuda.synchronize()
    got_graph = out.cpu().numpy().view(np.uint64)
    g.close()
    del t, out
    bad = []
    for s, ref in _oracle_segments(x, offs, 0):
        a, b = int(offs[s]), int(offs[s + 1])
        if not (np.array_equal(got_seg[a:b], ref) and np.array_equal(got_graph[a:b], ref)):
            bad.append(s)
    assert not bad, bad[:10]


@pytest.mark.parametrize("case", ["normal", "lognormal", "mixture", "zipf", "rounded"])
def test_pair_sorts_take_the_oracles_decisions(ctx, case):
    n = 3 * 10**6 + 7
    if case == "zipf":
        k = W.zipf_u64(n, seed=9, n_values=20000)
    elif case == "rounded":
        k = np.round(W.f64_keys("exponential", n, 10) * 100.0) / 100.0
    else:
        k = W.f64_keys(case, n, 11)
    v = np.arange(n, dtype=np.uint32)
    kt = "f64" if k.dtype == np.float64 else "u64"
    tk = torch.from_numpy(k if kt == "f64" else k.view(np.int64)).cuda()
    tv = torch.from_numpy(v.view(np.int32)).cuda()
    ko, vo = torch.empty_like(tk), torch.empty_like(tv)
    ctx.sort_pairs(tk, tv, ko, vo, key_type=kt, seed=7)
    torch.cuda.synchronize()
    st = ctx.last_stats()
    rk, rv, ost = oracle.sort(k, v, seed=7, with_stats=True)
    assert np.array_equal(ko.cpu().numpy().view(np.uint64), _bits(rk))
    assert np.array_equal(vo.cpu().numpy().view(np.uint32), rv)
    assert _decisions(st) == _oracle_decisions(ost), (st, ost)
