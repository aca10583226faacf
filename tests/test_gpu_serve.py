"""Served form on the GPU: concurrent requests, batched on several streams;
every result equals the oracle's sort and the same request sorted alone."""
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


def test_results_same_alone_and_in_the_mix(mods):
    pcfsort, serve = mods
    g = np.random.Generator(np.random.PCG64(11))
    reqs = []
    for i in range(48):
        n = int(2 ** g.uniform(6, 17))
        kt = "f64" if i % 2 == 0 else "u64"
        x = W.request_keys(n, kt, W.DISTRIBUTIONS[i % 5], seed=100 + i)
        reqs.append((x, kt))
    srv = serve.SortServer(device=0, workers=3, mem_budget=1 << 30, batch_keys=1 << 20)
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
    for h in handles:
        assert h.done.wait(120)
        assert h.error is None, h.error
    srv.close()
    ctx = pcfsort.Context(0)
    for (x, kt), h in zip(reqs, handles):
        got = h.out.cpu().numpy().view(np.uint64)
        ref, _ = oracle.sort(x)
        assert np.array_equal(got, ref.view(np.uint64))
        t = torch.from_numpy(x if kt == "f64" else x.view(np.int64)).cuda()
        alone = torch.empty_like(t)
        ctx.sort_keys(t, alone, key_type=kt)
        torch.cuda.synchronize()
        assert np.array_equal(alone.cpu().numpy().view(np.uint64), got)
    ctx.close()
    lat = serve.latency_summary(handles)
    assert lat["count"] == len(reqs) and lat["p99_ms"] >= lat["p50_ms"]
