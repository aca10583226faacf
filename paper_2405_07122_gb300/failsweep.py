"""The bucketing-failure experiment of Sec. 4.2 (Confirmation of Lemma
pcf-divide-success-prob) on the GPU.

alpha = floor(n^a), beta = floor(n^b), gamma = floor(n^c), delta = floor(n^d)
with a, b, c, d on the grid 0.05, 0.10, ..., 0.95; for each setting, R
arrays of n uniform keys are bucketed once (level 0 of Algorithm 1 with the
PCF model) and the setting's failure frequency is the share of arrays with
a bucket of more than delta keys.  The paper plots six heat maps, each
varying two of a, b, c, d with the other two at 0.75, against the line where
the lemma's bound equals 0.5.

The bucketing runs in the library (`Context.bucket_sizes`, one call per
setting over all R arrays); this module only chooses the parameters and
evaluates the lemma's closed form.
"""
import itertools
import math

GRID = [k / 20 for k in range(1, 20)]  # 0.05 .. 0.95
AXES = "abcd"
MAPS = [("a", "b"), ("a", "c"), ("a", "d"), ("b", "c"), ("b", "d"), ("c", "d")]


def floor_pow(n: int, k: int, q: int = 20) -> int:
    """floor(n^(k/q)) exactly: the largest m with m^q <= n^k (integers)."""
    if k == 0:
        return 1
    target = n ** k
    lo, hi = 1, 1
    while hi ** q <= target:
        hi *= 2
    while lo < hi:  # largest m with m^q <= target lies in [lo, hi)
        mid = (lo + hi + 1) // 2
        if mid ** q <= target:
            lo = mid
        else:
            hi = mid - 1
    return lo


def setting(n: int, a: float, b: float, c: float, d: float):
    """(alpha, beta, gamma, delta) of exponents on the 1/20 grid."""
    return tuple(max(1, floor_pow(n, round(e * 20))) for e in (a, b, c, d))


def lemma_bound(n: int, alpha: int, beta: int, gamma: int, delta: int, ratio: float = 1.0):
    """The right side of Lemma pcf-divide-success-prob,
    (2n/delta) exp(-(alpha K / (2 gamma)) (1 - 1/K)^2) with
    K = gamma delta / (2n) - 2 ratio gamma / beta (ratio = sigma2 / sigma1,
    1 for uniform keys); None where K < 1 (the lemma says nothing)."""
    K = gamma * delta / (2 * n) - 2 * ratio * gamma / beta
    if K < 1:
        return None
    log_b = math.log(2 * n / delta) - (alpha * K / (2 * gamma)) * (1 - 1 / K) ** 2
    return math.exp(min(log_b, 700.0))


def heat_map(ctx, keys, offsets, n: int, axes, fixed: float = 0.75, seed: int = 0,
             grid=GRID, stream=None):
    """Failure frequency over the (axes[0], axes[1]) grid, the other two
    exponents at `fixed`.  Returns {(x, y): (freq, bound)}."""
    R = len(offsets) - 1
    out = {}
    for x, y in itertools.product(grid, grid):
        e = {k: fixed for k in AXES}
        e[axes[0]], e[axes[1]] = x, y
        alpha, beta, gamma, delta = setting(n, e["a"], e["b"], e["c"], e["d"])
        mx = ctx.bucket_sizes(keys, offsets, alpha, beta, gamma, key_type="f64", seed=seed,
                              stream=stream)
        freq = float((mx > delta).sum()) / R
        out[(x, y)] = (freq, lemma_bound(n, alpha, beta, gamma, delta))
    return out


def agreement(points):
    """Where the bound is at most 0.5 the paper expects failure to be rare:
    (settings with bound <= 0.5, of those with frequency > 0.5)."""
    inside = [(f, b) for f, b in points.values() if b is not None and b <= 0.5]
    return len(inside), sum(1 for f, _ in inside if f > 0.5)
