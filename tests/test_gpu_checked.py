"""The index-checked build (-DPCF_CHECKED; compute-sanitizer is not
available): every computed store position of the scatters, the bucket
decision's small sorts and the on-chip finish is tested against its buffer
before the access, and one out of bounds would fail the call with
PCF_ERR_INTERNAL instead of writing.  The checked library sorts a spread of
inputs, policies and entry points (the CUDA-graph form included) in a
subprocess (one library per process) and must match the oracle everywhere
with no check firing."""
import os
import subprocess
import sys
import textwrap

import pytest

pytestmark = pytest.mark.gpu

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))

SCRIPT = textwrap.dedent('''
    import sys
    import numpy as np
    import torch
    sys.path.insert(0, ROOT)
    sys.path.insert(0, ROOT + "/tests")
    from paper_2405_07122_gb300 import build as B, pcfsort, workloads as W
    import oracle
    pcfsort.LIB_PATH = B.build(checked=True)

    def dev(x):
        return torch.from_numpy(x if x.dtype == np.float64 else x.view(np.int64)).cuda()

    def bits(a):
        return np.ascontiguousarray(a).view(np.uint64)

    def check_keys(ctx, x, pol=None, seed=0):
        t = dev(x)
        o = torch.empty_like(t)
        ctx.sort_keys(t, o, key_type="f64" if x.dtype == np.float64 else "u64", seed=seed)
        torch.cuda.synchronize()
        ref, _ = oracle.sort(x, seed=seed, policy=pol)
        assert np.array_equal(o.cpu().numpy().view(np.uint64), bits(ref))

    ctx = pcfsort.Context(0)
    for dist in W.DISTRIBUTIONS:
        for n in (100, 5000, 300001, 2 * 10**6):
            check_keys(ctx, W.f64_keys(dist, n, n + 1))
    check_keys(ctx, W.inject_duplicates(W.f64_keys("normal", 500000, 3), seed=3))
    x = W.zipf_u64(10**6, seed=4, n_values=20000)
    v = np.arange(x.size, dtype=np.uint32)
    t, tv = dev(x), torch.from_numpy(v.view(np.int32)).cuda()
    ko, vo = torch.empty_like(t), torch.empty_like(tv)
    ctx.sort_pairs(t, tv, ko, vo, key_type="u64")
    torch.cuda.synchronize()
    rk, rv = oracle.sort(x, v)
    assert np.array_equal(ko.cpu().numpy().view(np.uint64), rk)
    assert np.array_equal(vo.cpu().numpy().view(np.uint32), rv)
    keys, offs, _ = W.batched_f64(40, seed=5, lo_exp=6.0, hi_exp=18.0)
    t = dev(keys)
    o = torch.empty_like(t)
    ctx.sort_segmented(t, offs, keys_out=o, key_type="f64", seed=1)
    torch.cuda.synchronize()
    got = o.cpu().numpy().view(np.uint64)
    for s in range(len(offs) - 1):
        a, b = int(offs[s]), int(offs[s + 1])
        ref, _ = oracle.sort(keys[a:b], seed=1 + s)
        assert np.array_equal(got[a:b], bits(ref)), s
    # the same batch, and a duplicate-heavy array (standard-sort rounds),
    # captured in a CUDA graph and replayed
    o2 = torch.empty_like(t)
    g = pcfsort.SortGraph(ctx, t, offs, o2, key_type="f64", seed=1)
    assert g.info()["captured"]
    for _ in range(2):
        o2.zero_()
        assert g.launch()
        torch.cuda.synchronize()
        assert torch.equal(o2.view(torch.int64), o.view(torch.int64))
    g.close()
    xd = W.inject_duplicates(W.f64_keys("normal", 300000, 6), seed=6)
    td = dev(xd)
    od = torch.empty_like(td)
    g = pcfsort.SortGraph(ctx, td, [0, xd.size], od, key_type="f64")
    assert g.info()["captured"]
    od.zero_()
    assert g.launch()
    torch.cuda.synchronize()
    ref, _ = oracle.sort(xd)
    assert np.array_equal(od.cpu().numpy().view(np.uint64), bits(ref))
    g.close()
    for model, rng in (("spline", "array"), ("pcf", "sample")):
        c = pcfsort.Context(0, tuning=dict(leaf_cap=1024))
        c.set_policy(model=model, range_mode=rng)
        pol = oracle.paper_policy(
            model=oracle.MODEL_SPLINE if model == "spline" else oracle.MODEL_PCF,
            range_mode=oracle.RANGE_SAMPLE if rng == "sample" else oracle.RANGE_ARRAY)
        for dist in ("normal", "lognormal"):
            check_keys(c, W.f64_keys(dist, 400000, 9), pol=pol)
        c.close()
    print("checked ok")
''').replace("ROOT", repr(ROOT))


def test_checked_build_matches_oracle_without_bounds_errors():
    r = subprocess.run([sys.executable, "-c", SCRIPT], capture_output=True, text=True,
                       timeout=1200, cwd=ROOT)
    assert r.returncode == 0 and "checked ok" in r.stdout, r.stdout[-2000:] + r.stderr[-4000:]
