"""Seeded synthetic inputs for the sort workloads.

This module only draws inputs; it holds none of the sorting method's
arithmetic and is the one module that both the CUDA path's tests/benchmark
and the CPU oracle consume.  All draws use numpy's PCG64 so that a
(workload, seed) pair names one exact array on any machine.

Distributions follow the paper's synthetic setup (Sec. 4: Uniform[0,1),
Normal(0,1), Exponential(1), LogNormal(0,1)) plus a 5-component Gaussian
mixture (means U[-100,100], sd U[0.1,10], equal weights) and a duplicate-heavy
truncated Zipf(1.2) over 10^7 ranks hashed into 64-bit keys.  The adversarial
input of the paper's appendix (n extra copies of one value drawn inside
[x_min, x_max]) is `inject_duplicates`.
"""
import numpy as np

DISTRIBUTIONS = ("uniform", "normal", "lognormal", "exponential", "mixture")

_M64 = np.uint64(0xFFFFFFFFFFFFFFFF)


def _rng(seed: int) -> np.random.Generator:
    return np.random.Generator(np.random.PCG64(seed))


def f64_keys(dist: str, n: int, seed: int) -> np.ndarray:
    """n float64 keys i.i.d. from `dist`."""
    g = _rng(seed)
    if dist == "uniform":
        return g.random(n)
    if dist == "normal":
        return g.standard_normal(n)
    if dist == "lognormal":
        return g.lognormal(0.0, 1.0, n)
    if dist == "exponential":
        return g.exponential(1.0, n)
    if dist == "mixture":
        means = g.uniform(-100.0, 100.0, 5)
        sds = g.uniform(0.1, 10.0, 5)
        comp = g.integers(0, 5, n)
        return means[comp] + sds[comp] * g.standard_normal(n)
    raise ValueError("unknown distribution %r" % dist)


def fmix64(x: np.ndarray) -> np.ndarray:
    """MurmurHash3's 64-bit finaliser (Appleby): a bijection on uint64."""
    x = np.asarray(x, dtype=np.uint64).copy()
    with np.errstate(over="ignore"):
        x ^= x >> np.uint64(33)
        x *= np.uint64(0xFF51AFD7ED558CCD)
        x ^= x >> np.uint64(33)
        x *= np.uint64(0xC4CEB9FE1A85EC53)
        x ^= x >> np.uint64(33)
    return x


def zipf_u64(n: int, seed: int, s: float = 1.2, n_values: int = 10**7) -> np.ndarray:
    """n uint64 keys: Zipf(s) ranks truncated to [1, n_values] (redrawn when
    larger), each rank hashed to 64 bits by a seeded bijection."""
    g = _rng(seed)
    out = np.empty(n, dtype=np.uint64)
    filled = 0
    while filled < n:
        z = g.zipf(s, size=max(1024, int((n - filled) * 1.05)))
        z = z[z <= n_values][: n - filled]
        out[filled:filled + z.size] = z.astype(np.uint64)
        filled += z.size
    salt = np.uint64(fmix64(np.array([seed], dtype=np.uint64))[0])
    with np.errstate(over="ignore"):
        return fmix64(out ^ salt)


def f64_to_u64_fixed(x: np.ndarray) -> np.ndarray:
    """uint64 keys of the same distribution shape: 32 fractional bits of
    fixed point, offset by 2^63 (x within +-2^31)."""
    v = np.round(np.asarray(x, dtype=np.float64) * 4294967296.0)
    return (v.astype(np.int64).view(np.uint64) + np.uint64(1 << 63))


def inject_duplicates(x: np.ndarray, seed: int) -> np.ndarray:
    """Appendix 'adversarial' input: append len(x) copies of one value drawn
    uniformly in [min x, max x], then shuffle."""
    g = _rng(seed)
    if x.dtype == np.float64:
        v = g.uniform(float(x.min()), float(x.max()))
    else:
        v = np.uint64(g.integers(int(x.min()), int(x.max()), endpoint=True, dtype=np.uint64))
    y = np.concatenate([x, np.full(x.size, v, dtype=x.dtype)])
    g.shuffle(y)
    return y


def segment_lengths(n_segments: int, seed: int, lo_exp: float = 10.0, hi_exp: float = 22.0):
    """floor(2^U(lo_exp, hi_exp)) lengths (log-uniform)."""
    g = _rng(seed)
    return np.floor(np.exp2(g.uniform(lo_exp, hi_exp, n_segments))).astype(np.int64)


def segment_seed(seed: int, i: int) -> int:
    return int(fmix64(np.array([(seed << 20) + i + 1], dtype=np.uint64))[0] >> np.uint64(1))


def batched_f64(n_segments: int, seed: int, lo_exp: float = 10.0, hi_exp: float = 22.0):
    """Segmented batch: (keys, offsets[S+1], dists).  Segment i has length
    floor(2^U(lo_exp,hi_exp)) and a distribution drawn uniformly from
    DISTRIBUTIONS, with its own derived seed."""
    lens = segment_lengths(n_segments, seed, lo_exp, hi_exp)
    g = _rng(seed + 1)
    dists = [DISTRIBUTIONS[i] for i in g.integers(0, len(DISTRIBUTIONS), n_segments)]
    offs = np.zeros(n_segments + 1, dtype=np.int64)
    offs[1:] = np.cumsum(lens)
    keys = np.empty(int(offs[-1]), dtype=np.float64)
    for i in range(n_segments):
        keys[offs[i]:offs[i + 1]] = f64_keys(dists[i], int(lens[i]), segment_seed(seed, i))
    return keys, offs, dists


def request_stream(rate_hz: float, duration_s: float, seed: int, lo_exp: float = 12.0,
                   hi_exp: float = 26.0):
    """Poisson arrivals: list of (arrival_time_s, n, key_type 'f64'|'u64',
    dist, seed) with sizes floor(2^U(lo_exp, hi_exp))."""
    g = _rng(seed)
    t, out, i = 0.0, [], 0
    while True:
        t += g.exponential(1.0 / rate_hz)
        if t > duration_s:
            break
        n = int(np.floor(np.exp2(g.uniform(lo_exp, hi_exp))))
        kt = "f64" if g.random() < 0.5 else "u64"
        dist = DISTRIBUTIONS[int(g.integers(0, len(DISTRIBUTIONS)))]
        out.append((t, n, kt, dist, segment_seed(seed, i)))
        i += 1
    return out


def request_keys(n: int, kt: str, dist: str, seed: int) -> np.ndarray:
    x = f64_keys(dist, n, seed)
    return x if kt == "f64" else f64_to_u64_fixed(x)
