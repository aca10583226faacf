"""GPU parity of the mid-size Learned-Sort calls (k_mid): a next-level
bucket of leaf_cap < n <= 32768 keys takes its own call of Alg. 1 in one
CTA, and its buckets are finished by the block-local leaf sort.  Every
output is compared bit for bit with the oracle; the paths where k_mid
leaves a bucket to the next global level (one of its own buckets is too
large, or its range is degenerate) and where a bucket holds one value are
exercised with constructed inputs."""
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


def _dev(x):
    if x.dtype == np.float64:
        return torch.from_numpy(np.ascontiguousarray(x)).cuda()
    return torch.from_numpy(np.ascontiguousarray(x).view(np.int64)).cuda()


def _sort(ctx, x, seed=0):
    t = _dev(x)
    o = torch.empty_like(t)
    ctx.sort_keys(t, o, key_type="f64" if x.dtype == np.float64 else "u64", seed=seed)
    torch.cuda.synchronize()
    a = o.cpu().numpy()
    return (a if x.dtype == np.float64 else a.view(np.uint64)), ctx.last_stats()


def _bits(a):
    return a.view(np.uint64)


@pytest.mark.parametrize("dist", ["lognormal", "mixture", "exponential"])
def test_mid_calls_match_oracle(P, dist):
    # leaf_cap 2048: the densest level-0 buckets (a few thousand keys) go to
    # k_mid and every one of them finishes there, so one global level
    x = W.f64_keys(dist, 1 << 21, 11)
    ctx = P.Context(0, tuning=dict(leaf_cap=2048))
    got, st = _sort(ctx, x, seed=3)
    ref, _ = oracle.sort(x, seed=3)
    assert np.array_equal(_bits(got), _bits(ref))
    ctx.close()


def test_mid_call_on_lognormal_default_tuning(P):
    # the default leaf_cap (8192): LogNormal's densest level-0 buckets exceed
    # it at 2^23 keys and are finished by k_mid in the same level
    x = W.f64_keys("lognormal", 1 << 23, 12)
    ctx = P.Context(0)
    got, st = _sort(ctx, x, seed=1)
    assert st["levels"] == 1
    ref, _ = oracle.sort(x, seed=1)
    assert np.array_equal(_bits(got), _bits(ref))
    ctx.close()


def test_mid_leaves_a_too_large_inner_bucket_to_the_next_level(P):
    # a cluster of 20000 keys inside one level-0 bin (a mid-size bucket), and
    # inside it 5000 keys within 1e-15: one of k_mid's own buckets exceeds
    # leaf_cap, so the bucket goes to the next global level instead
    n = 1 << 21
    rng = np.random.default_rng(5)
    x = W.f64_keys("uniform", n, 13)
    pos = rng.choice(n, 20000, replace=False)
    x[pos] = 0.25 + rng.random(20000) * 1e-9
    x[pos[:5000]] = 0.25 + 5e-10 + rng.random(5000) * 1e-15
    ctx = P.Context(0, tuning=dict(leaf_cap=2048))
    got, st = _sort(ctx, x, seed=2)
    assert st["levels"] >= 2
    ref, _ = oracle.sort(x, seed=2)
    assert np.array_equal(_bits(got), _bits(ref))
    ctx.close()


def test_mid_single_value_bucket(P):
    # a mid-size bucket of one value: 20000 copies of 5.0 above keys in
    # [-1, 1) fill the last level-0 bin alone; k_mid copies it as it is
    n = 1 << 21
    rng = np.random.default_rng(6)
    x = W.f64_keys("uniform", n, 14) * 2.0 - 1.0
    x[rng.choice(n, 20000, replace=False)] = 5.0
    ctx = P.Context(0, tuning=dict(leaf_cap=2048))
    got, st = _sort(ctx, x, seed=4)
    assert st["levels"] == 1
    ref, _ = oracle.sort(x, seed=4)
    assert np.array_equal(_bits(got), _bits(ref))
    ctx.close()


def test_mid_signed_zero_bucket(P):
    # a mid-size bucket of -0.0 and +0.0 below keys in [1, 2): its range is
    # degenerate, so k_mid leaves it to the next level, whose standard sort
    # orders it (-0.0 before +0.0)
    n = 1 << 21
    rng = np.random.default_rng(8)
    x = W.f64_keys("uniform", n, 15) + 1.0
    pos = rng.choice(n, 20000, replace=False)
    x[pos[:10000]] = -0.0
    x[pos[10000:]] = 0.0
    ctx = P.Context(0, tuning=dict(leaf_cap=2048))
    got, st = _sort(ctx, x, seed=6)
    assert st["levels"] >= 2 and st["fallback_keys"] >= 20000
    ref, _ = oracle.sort(x, seed=6)
    assert np.array_equal(_bits(got), _bits(ref))
    ctx.close()


def test_mid_u64_keys(P):
    # unsigned keys through the mid calls: 20000 distinct values spread over
    # 2^48 around 2^62 (one or two level-0 bins of uniform u64 keys)
    n = 1 << 21
    rng = np.random.default_rng(7)
    x = rng.integers(0, 2**64 - 1, size=n, dtype=np.uint64)
    pos = rng.choice(n, 20000, replace=False)
    x[pos] = np.uint64(1 << 62) + rng.integers(0, 1 << 48, size=20000, dtype=np.uint64)
    ctx = P.Context(0, tuning=dict(leaf_cap=2048))
    got, st = _sort(ctx, x, seed=5)
    assert st["levels"] == 1
    ref, _ = oracle.sort(x, seed=5)
    assert np.array_equal(got, ref)
    ctx.close()


@pytest.mark.parametrize("start", [1, 3])
def test_mid_calls_with_buffers_at_8_byte_offsets(P, start):
    # input and output 8 bytes past a 16-byte boundary: the mid calls read
    # one buffer and append into the other, and their buckets are staged for
    # the leaf sort from a buffer at either alignment
    x = W.f64_keys("lognormal", (1 << 21) + 5, 16 + start)
    t = _dev(x)
    src = t[start:]
    out = torch.empty(src.numel() + 1, dtype=torch.float64, device="cuda")[1:]
    ctx = P.Context(0, tuning=dict(leaf_cap=2048))
    ctx.sort_keys(src, out, key_type="f64", seed=2)
    torch.cuda.synchronize()
    ref, _ = oracle.sort(x[start:], seed=2)
    assert np.array_equal(_bits(out.cpu().numpy()), _bits(ref))
    ctx.close()
