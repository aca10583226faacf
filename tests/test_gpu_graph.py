"""GPU parity of the batched sort captured in a CUDA graph (pcf_graph_*).

Creating a graph sorts the buffers once (recording the host's decision at
each global level's end) and captures the same sort.  A launch replays the
graph on the current contents of the input; a guard kernel at each level's
end checks that the device computed the recorded plan, and otherwise the
call sorts again without the graph.  Every output is compared bit for bit
with the oracle, and the tests check which way each launch went.
"""
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


def _dev(x):
    return torch.from_numpy(x if x.dtype == np.float64 else x.view(np.int64)).cuda()


def _bits(a):
    return np.ascontiguousarray(a).view(np.uint64)


def _check(out, x, offs, seed, v=None, vout=None):
    got = out.cpu().numpy().view(np.uint64)
    gv = None if vout is None else vout.cpu().numpy().view(np.uint32)
    for s in range(len(offs) - 1):
        a, b = int(offs[s]), int(offs[s + 1])
        rk, rv = oracle.sort(x[a:b], None if v is None else v[a:b], seed=seed + s)
        assert np.array_equal(got[a:b], _bits(rk)), s
        if v is not None:
            assert np.array_equal(gv[a:b], rv), s


def _offsets(lens):
    offs = np.zeros(len(lens) + 1, dtype=np.uint64)
    offs[1:] = np.cumsum(lens)
    return offs


def _mixed(seed, lens, dists=("uniform", "normal", "lognormal", "exponential", "mixture")):
    g = np.random.Generator(np.random.PCG64(seed))
    parts = [W.f64_keys(dists[int(g.integers(len(dists)))], int(n), seed * 1000 + i)
             for i, n in enumerate(lens)]
    return np.concatenate(parts) if parts else np.zeros(0)


def test_replay_mixed_lengths(P, ctx):
    # small arrays (on chip at level 0), one- and two-level large ones
    lens = [0, 1, 100, 4096, 4097, 70000, 2**20, 3, 2**18 + 5, 9000]
    offs = _offsets(lens)
    x = _mixed(1, lens)
    t = _dev(x)
    o = torch.full_like(t, -1)
    g = P.SortGraph(ctx, t, offs, o, key_type="f64", seed=7)
    _check(o, x, offs, 7)
    assert g.info()["captured"]
    for _ in range(3):
        o.fill_(-1)
        assert g.launch() is True
        torch.cuda.synchronize()
        _check(o, x, offs, 7)
    info = g.info()
    assert info["replays"] == 3 and info["eager_runs"] == 1
    # the input is never written
    assert np.array_equal(t.cpu().numpy().view(np.uint64), _bits(x))
    g.close()


def test_new_data_same_plan_replays(P, ctx):
    # Uniform arrays finish at level 0 with no standard-sort bucket: any
    # Uniform input takes the recorded plan, so the graph sorts it
    lens = [300000, 123457, 2**19]
    offs = _offsets(lens)
    x0 = np.concatenate([W.f64_keys("uniform", n, 10 + i) for i, n in enumerate(lens)])
    t = _dev(x0)
    o = torch.empty_like(t)
    g = P.SortGraph(ctx, t, offs, o, key_type="f64")
    for rep in range(3):
        x = np.concatenate([W.f64_keys("uniform", n, 100 * rep + i) for i, n in enumerate(lens)])
        t.copy_(_dev(x))
        assert g.launch() is True
        torch.cuda.synchronize()
        _check(o, x, offs, 0)
    g.close()


def test_new_data_mixed_batch_replays(P):
    # arrays of five distributions whose densest buckets exceed leaf_cap
    # (2048 here, as the autotuner picks for the batched workload): their
    # Learned-Sort calls run in k_mid within the level, so the plan (one
    # global level, no standard-sort item) depends on the lengths only, and
    # fresh keys of the same lengths replay
    lens = [5000, 2**17, 70001, 2**18 + 3, 9000, 2**16, 300000, 2**12]
    offs = _offsets(lens)
    x0 = _mixed(3, lens)
    ctx = P.Context(0, tuning=dict(leaf_cap=2048))
    tmp = torch.empty(int(offs[-1]), dtype=torch.float64, device="cuda")
    ctx.sort_segmented(_dev(x0), offs, keys_out=tmp, key_type="f64")
    assert ctx.last_stats()["levels"] == 1 and ctx.last_stats()["fallback_keys"] == 0
    t = _dev(x0)
    o = torch.empty_like(t)
    g = P.SortGraph(ctx, t, offs, o, key_type="f64", seed=1)
    for rep in range(3):
        x = _mixed(40 + rep, lens)
        t.copy_(_dev(x))
        o.zero_()
        assert g.launch() is True
        torch.cuda.synchronize()
        _check(o, x, offs, 1)
    g.close()
    ctx.close()


def test_new_data_other_plan_sorts_again(P):
    n = 2**22
    offs = _offsets([n])
    xu = W.f64_keys("uniform", n, 3)
    # a dense cluster of 50000 distinct keys inside one level-0 bin: a bucket
    # larger than one CTA's Learned-Sort call takes (kMidCap = 32768 keys),
    # below delta (92,681), so it takes a second global level
    xl = W.f64_keys("uniform", n, 4)
    rng = np.random.default_rng(4)
    xl[rng.choice(n, 50000, replace=False)] = 0.5 + rng.random(50000) * 1e-9
    # precondition: these keys take a second global level, Uniform none
    ctx = P.Context(0, tuning=dict(leaf_cap=2048))
    tmp = torch.empty_like(_dev(xl))
    ctx.sort_keys(_dev(xl), tmp, key_type="f64")
    assert ctx.last_stats()["levels"] >= 2
    ctx.sort_keys(_dev(xu), tmp, key_type="f64")
    assert ctx.last_stats()["levels"] == 1
    t = _dev(xu)
    o = torch.empty_like(t)
    g = P.SortGraph(ctx, t, offs, o, key_type="f64", seed=5)
    t.copy_(_dev(xl))
    assert g.launch() is False  # the guard saw another plan: sorted again
    torch.cuda.synchronize()
    _check(o, xl, offs, 5)
    assert g.info()["eager_runs"] == 2
    # The graph keeps its capture after one miss, and captures a missed plan
    # when it comes back on the next launch, or at once when the miss moved
    # a workspace buffer (its nodes would point at freed memory).  Either
    # way the same input replays within two more launches, and every output
    # is the sorted input.
    def settle(x):
        t.copy_(_dev(x))
        seen = []
        for _ in range(3):
            o.zero_()
            seen.append(g.launch())
            torch.cuda.synchronize()
            _check(o, x, offs, 5)
            if seen[-1]:
                break
        assert seen[-1] is True, seen
        return seen

    settle(xl)
    assert settle(xu)[0] is False  # the LogNormal plan is held: Uniform misses first
    assert settle(xu) == [True]
    assert settle(xl)[0] is False
    g.close()
    ctx.close()


@pytest.mark.parametrize("kt", ["f64", "u64"])
def test_pairs_stable(P, ctx, kt):
    lens = [5000, 2**20 + 3, 77, 2**17]
    offs = _offsets(lens)
    if kt == "f64":
        x = np.round(_mixed(2, lens) * 64.0) / 64.0  # ties
    else:
        gen = np.random.Generator(np.random.PCG64(2))
        x = gen.integers(0, 2**20, size=int(offs[-1]), dtype=np.uint64) << np.uint64(40)
    v = np.arange(x.size, dtype=np.uint32)[::-1].copy()
    t, tv = _dev(x), torch.from_numpy(v.view(np.int32)).cuda()
    o, ov = torch.empty_like(t), torch.empty_like(tv)
    g = P.SortGraph(ctx, t, offs, o, vals_in=tv, vals_out=ov, key_type=kt, seed=11)
    _check(o, x, offs, 11, v, ov)
    assert g.info()["captured"]
    o.zero_()
    ov.zero_()
    assert g.launch() is True
    torch.cuda.synchronize()
    _check(o, x, offs, 11, v, ov)
    g.close()


def test_nan_leaves_output_and_graph(P, ctx):
    lens = [2**20, 1000, 2**16]
    offs = _offsets(lens)
    x = _mixed(3, lens)
    t = _dev(x)
    o = torch.empty_like(t)
    g = P.SortGraph(ctx, t, offs, o, key_type="f64")
    for where in (5, int(offs[1]) + 3, int(offs[2]) + 100):  # a large and a small array
        y = x.copy()
        y[where] = np.nan
        t.copy_(_dev(y))
        o.fill_(7)
        with pytest.raises(P.PcfError) as e:
            g.launch()
        assert e.value.code == 2  # PCF_ERR_INVALID_KEY
        torch.cuda.synchronize()
        assert bool((o == 7).all()), "output written after a NaN"
    t.copy_(_dev(x))
    assert g.launch() is True  # the graph is intact
    torch.cuda.synchronize()
    _check(o, x, offs, 0)
    g.close()


def test_standard_sort_rounds_replay(P, ctx):
    # Buckets sent to the standard sort: their split rounds and merge sort
    # are captured too, each read-back replaced by a guard
    x = W.inject_duplicates(W.f64_keys("normal", 2**19, 8), seed=8)
    offs = _offsets([x.size])
    t = _dev(x)
    o = torch.empty_like(t)
    g = P.SortGraph(ctx, t, offs, o, key_type="f64")
    _check(o, x, offs, 0)
    assert g.info()["captured"]
    o.zero_()
    assert g.launch() is True
    torch.cuda.synchronize()
    _check(o, x, offs, 0)
    # other duplicates: other rounds, so the guards send it back to the host
    y = W.inject_duplicates(W.f64_keys("normal", 2**19, 9), seed=9)
    t.copy_(_dev(y))
    assert g.launch() is False
    torch.cuda.synchronize()
    _check(o, y, offs, 0)
    g.close()


def test_many_split_rounds_pairs(P, ctx):
    # heavy value k holds n >> (k + 1) keys, all in one bucket: more split
    # rounds than the limit, then the merge sort; stable values
    n = 1 << 20
    gen = np.random.Generator(np.random.PCG64(4))
    parts, used = [], 0
    for k in range(20):
        c = n >> (k + 1)
        parts.append(np.full(c, (1 << 63) + 3 * k, dtype=np.uint64))
        used += c
    parts.append(gen.integers(0, 2**64 - 1, size=n - used, dtype=np.uint64, endpoint=True))
    x = np.concatenate(parts)
    gen.shuffle(x)
    lens = [n // 2, n - n // 2]
    offs = _offsets(lens)
    v = np.arange(n, dtype=np.uint32)
    t, tv = _dev(x), torch.from_numpy(v.view(np.int32)).cuda()
    o, ov = torch.empty_like(t), torch.empty_like(tv)
    g = P.SortGraph(ctx, t, offs, o, vals_in=tv, vals_out=ov, key_type="u64", seed=2)
    _check(o, x, offs, 2, v, ov)
    assert g.info()["captured"]
    for _ in range(2):
        o.zero_()
        ov.zero_()
        assert g.launch() is True
        torch.cuda.synchronize()
        _check(o, x, offs, 2, v, ov)
    g.close()


def test_zipf_pairs_three_levels(P, ctx):
    # duplicate-heavy u64 pairs: several global levels and many split rounds,
    # all captured; the replay is stable and matches the oracle
    k = W.zipf_u64(1 << 22, seed=5, n_values=200000)
    v = np.arange(k.size, dtype=np.uint32)
    offs = _offsets([k.size])
    t, tv = _dev(k), torch.from_numpy(v.view(np.int32)).cuda()
    o, ov = torch.empty_like(t), torch.empty_like(tv)
    g = P.SortGraph(ctx, t, offs, o, vals_in=tv, vals_out=ov, key_type="u64", seed=1)
    assert g.info()["captured"]
    o.zero_()
    ov.zero_()
    assert g.launch() is True
    torch.cuda.synchronize()
    _check(o, k, offs, 1, v, ov)
    g.close()


def test_small_arrays_only(P, ctx):
    g0 = np.random.Generator(np.random.PCG64(9))
    lens = g0.integers(0, 4097, size=300)
    offs = _offsets(lens)
    x = _mixed(9, lens)
    for kt in ("f64", "u64"):
        xx = x if kt == "f64" else W.f64_to_u64_fixed(x)
        t = _dev(xx)
        o = torch.empty_like(t)
        g = P.SortGraph(ctx, t, offs, o, key_type=kt, seed=3)
        assert g.info()["captured"]
        o.zero_()
        assert g.launch() is True
        torch.cuda.synchronize()
        _check(o, xx, offs, 3)
        g.close()


def test_no_keys(P, ctx):
    # no segments, or only empty ones: nothing to sort, every launch returns
    t = torch.empty(0, dtype=torch.float64, device="cuda")
    o = torch.empty(0, dtype=torch.float64, device="cuda")
    for offs in ([0], [0, 0, 0]):
        g = P.SortGraph(ctx, t, offs, o, key_type="f64")
        assert not g.info()["captured"]
        assert g.launch() is False
        g.close()


def test_rejects_in_place_and_overlap(P, ctx):
    x = W.f64_keys("normal", 10000, 1)
    t = _dev(x)
    with pytest.raises(P.PcfError) as e:
        P.SortGraph(ctx, t, [0, x.size], t, key_type="f64")
    assert e.value.code == 1  # PCF_ERR_INVALID_ARG
    big = torch.empty(2 * x.size, dtype=torch.float64, device="cuda")
    with pytest.raises(P.PcfError) as e:
        P.SortGraph(ctx, big[:x.size], [0, x.size], big[100:100 + x.size], key_type="f64")
    assert e.value.code == 1  # PCF_ERR_INVALID_ARG


@pytest.mark.parametrize("model,rng", [("spline", "array"), ("pcf", "sample")])
def test_policy_and_tuning_follow_the_context(P, model, rng):
    c = P.Context(0, tuning=dict(leaf_cap=1024))
    c.set_policy(model=model, range_mode=rng)
    lens = [2**20, 3000, 50000]
    offs = _offsets(lens)
    x = np.concatenate([W.f64_keys(d, n, 12 + i) for i, (d, n) in
                        enumerate(zip(("exponential", "normal", "mixture"), lens))])
    t = _dev(x)
    o = torch.empty_like(t)
    g = P.SortGraph(c, t, offs, o, key_type="f64")
    _check(o, x, offs, 0)
    o.zero_()
    assert g.launch() is True
    torch.cuda.synchronize()
    _check(o, x, offs, 0)
    # a NaN (with the samples' range it is found by the bucketing pass)
    y = x.copy()
    y[777] = np.nan
    t.copy_(_dev(y))
    o.fill_(7)
    with pytest.raises(P.PcfError) as e:
        g.launch()
    assert e.value.code == 2  # PCF_ERR_INVALID_KEY
    torch.cuda.synchronize()
    assert bool((o == 7).all())
    g.close()
    c.close()
