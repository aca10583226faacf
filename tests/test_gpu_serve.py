"""Served form on the GPU: concurrent requests, batched on several streams;
every result equals the oracle's sort and the same request sorted alone.
Keys produced asynchronously right before submission are read in stream
order, and under memory pressure requests wait for released results."""
import threading

import numpy as np
import pytest

import oracle
from paper_2405_07122_gb300 import workloads as W

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")


@pytest.fixture(scope="module")
def mods():
    from paper_2405_07122_gb300 import build as pcf_build
    pcf_build.build()
    from paper_2405_07122_gb300 import pcfsort, serve
    return pcfsort, serve


def _reqs(seed, count, lo, hi):
    g = np.random.Generator(np.random.PCG64(seed))
    out = []
    for i in range(count):
        n = int(2 ** g.uniform(lo, hi))
        kt = "f64" if i % 2 == 0 else "u64"
        out.append((W.request_keys(n, kt, W.DISTRIBUTIONS[i % 5], seed=seed * 1000 + i), kt))
    return out


def _check(pcfsort, reqs, results):
    ctx = pcfsort.Context(0)
    for (x, kt), got in zip(reqs, results):
        ref, _ = oracle.sort(x)
        assert np.array_equal(got, ref.view(np.uint64))
        t = torch.from_numpy(x if kt == "f64" else x.view(np.int64)).cuda()
        alone = torch.empty_like(t)
        ctx.sort_keys(t, alone, key_type=kt)
        torch.cuda.synchronize()
        assert np.array_equal(alone.cpu().numpy().view(np.uint64), got)
    ctx.close()


def test_results_same_alone_and_in_the_mix(mods):
    pcfsort, serve = mods
    reqs = _reqs(11, 48, 6, 17)
    srv = serve.SortServer(device=0, workers=3, mem_budget=1 << 30, batch_keys=1 << 20,
                           headroom=0)
    handles = [None] * len(reqs)

    def client(k):
        for i in range(k, len(reqs), 4):
            x, kt = reqs[i]
            t = torch.from_numpy(x if kt == "f64" else x.view(np.int64)).cuda()
            torch.cuda.synchronize()
            handles[i] = srv.submit(t, kt)

    ths = [threading.Thread(target=client, args=(k,)) for k in range(4)]
    for t in ths:
        t.start()
    for t in ths:
        t.join()
    results = []
    for h in handles:
        assert h.done.wait(120)
        assert h.error is None, h.error
        results.append(h.out.cpu().numpy().view(np.uint64).copy())
        h.release()
    srv.close()
    _check(pcfsort, reqs, results)
    lat = serve.latency_summary(handles)
    assert lat["count"] == len(reqs) and lat["p99_ms"] >= lat["p50_ms"]


def test_async_producer_without_synchronisation(mods):
    # each request's keys are written by a kernel on the client's own stream
    # behind a slow kernel and submitted at once: the server must wait for
    # that stream, not for the host
    pcfsort, serve = mods
    reqs = _reqs(12, 16, 8, 16)
    srv = serve.SortServer(device=0, workers=2, mem_budget=1 << 30, batch_keys=1 << 20,
                           headroom=0)
    side = torch.cuda.Stream()
    handles, keep = [], []
    with torch.cuda.stream(side):
        for x, kt in reqs:
            src = torch.from_numpy(x if kt == "f64" else x.view(np.int64)).pin_memory()
            dst = torch.empty(src.shape, dtype=src.dtype, device="cuda")
            torch.cuda._sleep(1_000_000)
            dst.copy_(src, non_blocking=True)
            keep.append((src, dst))
            handles.append(srv.submit(dst, kt))
    results = []
    for h in handles:
        assert h.done.wait(120)
        assert h.error is None, h.error
        results.append(h.out.cpu().numpy().view(np.uint64).copy())
        h.release()
    srv.close()
    _check(pcfsort, reqs, results)


def test_admission_under_memory_pressure(mods):
    # a result pool of 2^16 keys: requests beyond it wait for the client to
    # release earlier results, then complete correctly
    pcfsort, serve = mods
    reqs = _reqs(13, 12, 13, 15)   # 8K-32K keys each, more than the pool in all
    srv = serve.SortServer(device=0, workers=2, mem_budget=8 << 16, batch_keys=1 << 16,
                           headroom=0)
    assert srv.pool_keys == 1 << 16
    handles = []
    for x, kt in reqs:
        t = torch.from_numpy(x if kt == "f64" else x.view(np.int64)).cuda()
        handles.append(srv.submit(t, kt))
    assert sum(h.n for h in handles) > srv.pool_keys
    results = []
    for h in handles:
        # a later request can only be admitted once earlier ones are released
        assert h.done.wait(120)
        assert h.error is None, h.error
        results.append(h.out.cpu().numpy().view(np.uint64).copy())
        h.release()
    assert srv.adm.reserved == 0 and srv.adm.pool.free_keys() == srv.pool_keys
    srv.close()
    _check(pcfsort, reqs, results)
